"""Helpers shared by the GPU parity tests: moving cubes between the oracle's
float64 (n1, n2, n3) arrays and the library's flat float32 device tensors."""
import numpy as np


def dev(cube):
    """(n1, n2, n3) array -> flat float32 CUDA tensor in i + n1*(j + n2*k) order."""
    import torch
    flat = np.ascontiguousarray(np.asarray(cube).reshape(-1, order="F").astype(np.float32))
    return torch.from_numpy(flat).cuda()


def dev3(cubes):
    """(3, n1, n2, n3) -> flat 3N float32 CUDA tensor (mode-n blocks back to back)."""
    import torch
    return torch.cat([dev(c) for c in cubes])


def host(t, shape):
    """Flat CUDA tensor -> float64 (n1, n2, n3) array."""
    return t.detach().cpu().numpy().astype(np.float64).reshape(shape, order="F")


def host3(t, shape):
    a = t.detach().cpu().numpy().astype(np.float64)
    N = int(np.prod(shape))
    return np.stack([a[n * N:(n + 1) * N].reshape(shape, order="F") for n in range(3)])


def f32(x):
    """Rounds an oracle array to the float32 values the GPU sees."""
    return np.asarray(x, np.float64).astype(np.float32).astype(np.float64)


def maxabs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))


STATE_NAMES = ("Y", "L", "Z", "S", "G1", "G2", "F", "E", "G3", "G4")
TRIPLE = ("F", "E", "G3", "G4")


def load_oracle_state(plan, st):
    """Copies an oracle State (rounded to float32) into a GPU plan, including
    mu and the iteration counter.  Returns the rounded copy of the state the
    oracle should continue from."""
    st32 = st.copy()
    st32.buf = f32(st.buf)
    for name in STATE_NAMES:
        if name in TRIPLE:
            plan.set(name, dev3([st32.get(name, n) for n in range(3)]))
        else:
            plan.set(name, dev(st32.get(name)))
    plan.set_mu(st32.mu, st.iters)
    return st32
