"""Pins of the FP64 adjoint of the unrolled iteration (oracle/adjoint.py).

The adjoint is checked against things it does not compute itself: torch's
autograd of a complex SVD (for the singular value thresholding), and central
finite differences of the C oracle's forward iteration (for the t-SVT, one
whole iteration and a chain of iterations with free per-iteration scalars).
The numpy forward it differentiates is checked against the C oracle.
"""
import numpy as np
import pytest

from oracle import adjoint as adj

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

KEYS = ("L", "Z", "S", "G1", "G2", "F", "E", "G3", "G4")


def _rand_state(shape, seed, scale=0.3):
    """A mid-run-like state: every block random (multipliers included), so
    that every term of the iteration is exercised."""
    rng = np.random.default_rng(seed)
    Y = rng.uniform(0.0, 1.0, shape)
    st = adj.initial_state(Y)
    for k in KEYS:
        st[k] = st[k] + scale * rng.standard_normal(st[k].shape)
    return st


def _c_state(orc, st, theta):
    c = orc.State(st["Y"], orc.Params(n1=st["Y"].shape[0], n2=st["Y"].shape[1]))
    for k in KEYS:
        if st[k].ndim == 4:
            for n in range(3):
                c.set(k, st[k][n], n)
        else:
            c.set(k, st[k])
    return c


def _c_step(orc, st, theta):
    """One iteration through the C oracle; returns the new state as a dict."""
    c = _c_state(orc, st, theta)
    c.step_theta(*theta)
    out = {"Y": st["Y"]}
    for k in KEYS:
        out[k] = np.stack([c.get(k, n) for n in range(3)]) if st[k].ndim == 4 else c.get(k)
    return out


def _dot(a, b, keys):
    return sum(float(np.sum(a[k] * b[k])) for k in keys if k in a and k in b)


THETA = (0.02, 0.35, 0.08, 1.3)


def test_forward_matches_c_oracle(orc):
    st = _rand_state((7, 6, 5), 1)
    new, _ = adj.forward_iteration(st, THETA)
    ref = _c_step(orc, st, THETA)
    for k in KEYS:
        assert np.max(np.abs(new[k] - ref[k])) < 1e-10, k


def _svt_torch(A, t, C):
    torch = pytest.importorskip("torch")
    At = torch.tensor(A, dtype=torch.complex128, requires_grad=True)
    U, s, Vh = torch.linalg.svd(At, full_matrices=False)
    R = (U * torch.clamp(s - t, min=0.0).to(U.dtype)) @ Vh
    loss = (torch.tensor(C).conj() * R).real.sum()
    loss.backward()
    return At.grad.numpy()


def _rand_complex(rng, m, n):
    return rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))


@pytest.mark.parametrize("m,n", [(7, 5), (5, 7), (6, 6)])
def test_svt_backward_matches_torch_autograd(m, n):
    rng = np.random.default_rng(10 + m + 3 * n)
    A = _rand_complex(rng, m, n)
    s = np.linalg.svd(A, compute_uv=False)
    t = 0.5 * (s[1] + s[2])  # two values kept, the rest cut
    C = _rand_complex(rng, m, n)
    gA, _ = adj.svt_backward(A, t, C)
    ref = _svt_torch(A, t, C)
    # torch returns d loss / d conj(A) scaled so that its real and imaginary
    # parts are the partial derivatives along Re A and Im A
    assert np.max(np.abs(gA - ref)) < 1e-10


def _fd_svt(A, t, C, dA, dt, h=1e-6):
    f = lambda a, tt: float(np.real(np.sum(np.conj(C) * adj.svt(a, tt))))
    return (f(A + h * dA, t + h * dt) - f(A - h * dA, t - h * dt)) / (2 * h)


def _svt_cases():
    rng = np.random.default_rng(7)
    cases = []
    A = _rand_complex(rng, 8, 5)
    cases.append(("tall", A, 0.7 * np.linalg.svd(A, compute_uv=False)[2]))
    A = _rand_complex(rng, 4, 9)
    cases.append(("wide", A, 0.9 * np.linalg.svd(A, compute_uv=False)[1]))
    # exactly rank 2 (zero singular values below a positive threshold)
    A = _rand_complex(rng, 6, 2) @ _rand_complex(rng, 2, 6)
    cases.append(("rank2", A, 0.3 * np.linalg.svd(A, compute_uv=False)[1]))
    # a repeated kept singular value and a repeated cut one
    U, _ = np.linalg.qr(_rand_complex(rng, 6, 6))
    V, _ = np.linalg.qr(_rand_complex(rng, 6, 6))
    A = (U * np.array([3.0, 2.0, 2.0, 0.4, 0.4, 0.1])) @ V.conj().T
    cases.append(("repeated", A, 1.0))
    # all values cut, and none cut
    A = _rand_complex(rng, 5, 5)
    cases.append(("allcut", A, 2.0 * np.linalg.svd(A, compute_uv=False)[0]))
    cases.append(("nonecut", A, 0.5 * np.linalg.svd(A, compute_uv=False)[-1]))
    return cases


@pytest.mark.parametrize("name,A,t", _svt_cases(), ids=lambda x: x if isinstance(x, str) else "")
def test_svt_backward_matches_finite_differences(name, A, t):
    rng = np.random.default_rng(sum(map(ord, name)))
    C = _rand_complex(rng, *A.shape)
    gA, gt = adj.svt_backward(A, t, C)
    for trial in range(3):
        dA = _rand_complex(rng, *A.shape)
        dt = rng.standard_normal()
        want = _fd_svt(A, t, C, dA, dt)
        got = float(np.real(np.sum(np.conj(gA) * dA))) + gt * dt
        assert abs(got - want) <= 1e-7 * max(1.0, abs(want)), (name, got, want)


@pytest.mark.parametrize("shape", [(6, 5, 4), (5, 7, 5)])
def test_tsvt_backward_matches_c_oracle_fd(orc, shape):
    rng = np.random.default_rng(sum(shape))
    B = rng.standard_normal(shape)
    t = 1.5
    G = rng.standard_normal(shape)
    gB, gt = adj.tsvt_backward(B, t, G)
    for trial in range(2):
        dB = rng.standard_normal(shape)
        dt = rng.standard_normal()
        h = 1e-6
        f = lambda b, tt: float(np.sum(G * orc.tsvt(b, tt)[0]))
        want = (f(B + h * dB, t + h * dt) - f(B - h * dB, t - h * dt)) / (2 * h)
        got = float(np.sum(gB * dB)) + gt * dt
        assert abs(got - want) <= 1e-6 * max(1.0, abs(want)), (got, want)


def _rand_like(st, rng):
    return {k: rng.standard_normal(st[k].shape) for k in ("Y",) + KEYS}


def test_iteration_backward_matches_c_oracle_fd(orc):
    shape = (6, 5, 4)
    st = _rand_state(shape, 3)
    rng = np.random.default_rng(4)
    W = _rand_like(st, rng)            # loss = <W, new state>
    new, inter = adj.forward_iteration(st, THETA)
    g_state, g_theta = adj.backward_iteration(st, inter, THETA, {k: W[k] for k in KEYS})

    def loss(s, th):
        return _dot(W, _c_step(orc, s, th), KEYS)

    h = 1e-6
    # state directions
    for trial in range(2):
        dS = _rand_like(st, rng)
        sp = {k: st[k] + h * dS[k] for k in st}
        sm = {k: st[k] - h * dS[k] for k in st}
        want = (loss(sp, THETA) - loss(sm, THETA)) / (2 * h)
        got = _dot(g_state, dS, ("Y",) + KEYS)
        assert abs(got - want) <= 1e-6 * max(1.0, abs(want)), (got, want)
    # each scalar on its own
    for i in range(4):
        e = np.zeros(4)
        e[i] = h * THETA[i]
        want = (loss(st, np.add(THETA, e)) - loss(st, np.subtract(THETA, e))) / (2 * e[i])
        assert abs(g_theta[i] - want) <= 1e-6 * max(1.0, abs(want)), (i, g_theta[i], want)


def test_unrolled_gradient_matches_c_oracle_fd(orc):
    from synthetic import Recipe, make_cube
    clean, noisy = make_cube(Recipe(8, 8, 6, 3, 5, (0.1, 0.1), 0.1), 11)
    thetas = np.array([[1e-3, 0.2, 0.125, 1e-2 * 1.5 ** k] for k in range(3)])
    thetas[1, 0] = 3e-3
    loss, g_theta, g_Y = adj.unrolled_loss_grad(noisy, clean, thetas)

    def c_loss(Y, th):
        c = orc.State(Y, orc.Params(n1=8, n2=8))
        for row in th:
            c.step_theta(*row)
        return float(np.mean((c.X - clean) ** 2))

    assert abs(c_loss(noisy, thetas) - loss) < 1e-12
    for k in range(3):
        for i in range(4):
            h = 1e-5 * thetas[k, i]
            tp, tm = thetas.copy(), thetas.copy()
            tp[k, i] += h
            tm[k, i] -= h
            want = (c_loss(noisy, tp) - c_loss(noisy, tm)) / (2 * h)
            # floor: the rounding noise of a central difference of the loss
            noise = 64 * np.finfo(float).eps * loss / h
            assert abs(g_theta[k, i] - want) <= 1e-5 * abs(want) + noise, (k, i, g_theta[k, i], want)
    rng = np.random.default_rng(5)
    dY = rng.standard_normal(noisy.shape)
    h = 1e-6
    want = (c_loss(noisy + h * dY, thetas) - c_loss(noisy - h * dY, thetas)) / (2 * h)
    assert abs(float(np.sum(g_Y * dY)) - want) <= 1e-6 * max(abs(want), 1e-9)


# -------------------------------------------------- planted mistakes ---
def _mutated_adjoint(old, new):
    """A copy of oracle/adjoint.py with one planted mistake."""
    import types
    src = open(adj.__file__).read()
    assert old in src, old
    mod = types.ModuleType("adjoint_mutated")
    mod.__file__ = adj.__file__
    exec(compile(src.replace(old, new, 1), adj.__file__, "exec"), mod.__dict__)
    return mod


_ADJ_MUTATIONS = {
    # the SVD differential's off-diagonal coefficients exchanged
    "svt_ab_swapped": ("M = a * H + b * H.conj().T", "M = b * H + a * H.conj().T",
                       lambda orc: test_svt_backward_matches_torch_autograd(7, 5)),
    # the directions outside the column space left out (a tall matrix has them)
    "svt_range_term": ("Abar = Abar + Pu @ G", "Abar = Abar + 0.0 * Pu @ G",
                       lambda orc: test_svt_backward_matches_finite_differences(*_svt_cases()[0])),
    # the threshold's gradient with the wrong sign
    "svt_threshold_sign": ("tbar = -float(np.sum(fp * d.real))", "tbar = float(np.sum(fp * d.real))",
                           lambda orc: test_svt_backward_matches_finite_differences(*_svt_cases()[0])),
    # the adjoint of Re ifft without its 1/n3
    "tsvt_scale": ("Gh = np.fft.fft(Ebar, axis=2) / n3", "Gh = np.fft.fft(Ebar, axis=2)",
                   lambda orc: test_tsvt_backward_matches_c_oracle_fd(orc, (6, 5, 4))),
    # the F-update's one half dropped on the path to E
    "f_half": ('out["E"] += 0.5 * ba', 'out["E"] += ba',
               lambda orc: test_iteration_backward_matches_c_oracle_fd(orc)),
    # the S threshold's derivative in mu dropped
    "s_threshold_mu": ("dmu += np.sum(bS * sgn) * lam / mu ** 2", "dmu += 0.0",
                       lambda orc: test_iteration_backward_matches_c_oracle_fd(orc)),
}


@pytest.mark.parametrize("name", sorted(_ADJ_MUTATIONS))
def test_pins_catch_planted_mistakes(orc, monkeypatch, name):
    import sys
    old, new, pin = _ADJ_MUTATIONS[name]
    monkeypatch.setattr(sys.modules[__name__], "adj", _mutated_adjoint(old, new))
    with pytest.raises(AssertionError):
        pin(orc)
