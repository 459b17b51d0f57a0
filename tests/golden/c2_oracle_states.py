"""FP64 oracle states of the 200x200x80 benchmark cube, for the full-size
parity tests of the benchmarked path (tests/test_gpu_fullsize.py).

Runs Algorithm 1 (plain LRSTV, the library's default scalars) on the c2
mixed-noise cube, seed 2, with the oracle alone (oracle/ and the seeded
generator in synthetic/; nothing from the CUDA path), and keeps:
 - the whole state after EARLY_LOAD iterations (rounded to float32, the
   values a plan is loaded with), for the step-by-step comparison;
 - L, S, F, E after each of EARLY_COMPARE iterations of the uninterrupted run,
   for a warm-started plan run from lrstv_init;
 - the whole state after LATE_LOAD iterations, rounded to float32, and, from
   that rounded state, L, S, F, E, Gamma1, Gamma2 after each of
   LATE_COMPARE, for a warm-started plan loaded with it (late iterations,
   where the Jacobi runs one or two sweeps under the threshold-aware
   tolerance).

One oracle run of LATE_COMPARE[-1] iterations: about 20 s an iteration on 8
x86 cores, 5 s on 16 Grace cores.  The states are cached by key (a SHA-256
of the float32 cube, the oracle's scalars, the iteration lists and the
sources of the oracle and the generator) when LRSTV_ORACLE_CACHE names a
directory; a cache whose key does not match is recomputed.

    python tests/golden/c2_oracle_states.py [cache_dir]   # writes the cache
"""
from __future__ import annotations

import hashlib
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

EARLY_LOAD = 2
EARLY_COMPARE = (3, 4, 5, 6)
LATE_LOAD = 30
LATE_COMPARE = (31, 32, 33)
COMPARE_BLOCKS = ("L", "S", "F", "E", "G1", "G2")
SEED = 2


def cube():
    """(shape, float32-rounded noisy cube as float64) of the c2 recipe."""
    from synthetic import RECIPES, make_cube
    r = RECIPES["c2"]
    _, noisy = make_cube(r, SEED)
    return r.shape, noisy.astype(np.float32).astype(np.float64)


def key(Y, params_vec) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(Y.astype(np.float32)).tobytes())
    h.update(np.asarray(params_vec, np.float64).tobytes())
    h.update(repr((EARLY_LOAD, EARLY_COMPARE, LATE_LOAD, LATE_COMPARE, COMPARE_BLOCKS)).encode())
    for rel in ("oracle/lrstv_oracle.c", "oracle/lrstv_oracle.h", "oracle/oracle.py",
                "synthetic/hsi.py"):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _snapshot(st, names):
    out = {}
    for name in names:
        if name in ("F", "E", "G3", "G4"):
            out[name] = np.stack([st.get(name, n) for n in range(3)]).astype(np.float32)
        else:
            out[name] = st.get(name).astype(np.float32)
    return out


def _rounded(st):
    """A copy of the state rounded to float32 (what a plan holds once loaded)."""
    c = st.copy()
    c.buf = c.buf.astype(np.float32).astype(np.float64)
    return c


def compute(orc):
    """Runs the oracle; returns a dict of arrays (see the module docstring)."""
    shape, Y = cube()
    st = orc.State(Y, orc.Params(n1=shape[0], n2=shape[1]))
    out = {"shape": np.array(shape), "key": np.array(key(Y, st.p))}
    done = 0

    def run_to(k):
        nonlocal done
        if k > done:
            st.iterate(k - done)
            done = k

    run_to(EARLY_LOAD)
    out["early_state"] = st.buf.astype(np.float32)
    out["early_mu"] = np.array([st.mu, st.iters], np.float64)
    for k in EARLY_COMPARE:
        run_to(k)
        for name, v in _snapshot(st, COMPARE_BLOCKS).items():
            out[f"early_{k}_{name}"] = v
    run_to(LATE_LOAD)
    st = _rounded(st)
    out["late_state"] = st.buf.astype(np.float32)
    out["late_mu"] = np.array([st.mu, st.iters], np.float64)
    for k in LATE_COMPARE:
        run_to(k)
        for name, v in _snapshot(st, COMPARE_BLOCKS).items():
            out[f"late_{k}_{name}"] = v
        out[f"late_{k}_mu"] = np.array([st.mu], np.float64)
    return out


def load_or_compute(orc, cache_dir=None):
    """The states from cache_dir (or LRSTV_ORACLE_CACHE) when its key matches,
    else computed (and written there when a directory is named)."""
    cache_dir = cache_dir or os.environ.get("LRSTV_ORACLE_CACHE")
    shape, Y = cube()
    want = key(Y, orc.Params(n1=shape[0], n2=shape[1]).vector())
    path = os.path.join(cache_dir, "c2_oracle_states.npz") if cache_dir else None
    if path and os.path.exists(path):
        with np.load(path) as z:
            if str(z["key"]) == want:
                return {k: z[k] for k in z.files}
    out = compute(orc)
    assert str(out["key"]) == want
    if path:
        os.makedirs(cache_dir, exist_ok=True)
        tmp = path + f".tmp{os.getpid()}.npz"
        np.savez(tmp, **out)
        os.replace(tmp, path)
    return out


if __name__ == "__main__":
    import oracle
    oracle.build_oracle()
    d = sys.argv[1] if len(sys.argv) > 1 else os.environ.get("LRSTV_ORACLE_CACHE")
    if not d:
        sys.exit("usage: c2_oracle_states.py CACHE_DIR (or set LRSTV_ORACLE_CACHE)")
    s = load_or_compute(oracle, d)
    print(f"{d}: key {s['key']}, {len(s)} arrays")
