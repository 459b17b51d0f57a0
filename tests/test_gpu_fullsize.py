"""Parity at the benchmark's full size and in its own configuration: the
200x200x80 Pavia-shaped synthetic cube with the mixed-noise recipe, through
the plan / lrstv_iterate path that bench.py times, against the FP64 oracle.

The oracle states come from tests/golden/c2_oracle_states.py (one oracle run
of 33 iterations, cached by key when LRSTV_ORACLE_CACHE is set).  Compared:
 - a warm-started plan (LRSTV_FLAG_WARM_START, the benchmark's default) run
   from lrstv_init: iterations 0 and 1 cut every singular value (every
   Fourier slice's Frobenius norm is below the threshold alpha/mu, so the
   t-SVT is exactly zero and no Jacobi sweep runs); iterations 2-5 run 9-12
   sweeps; L (= X), S, F and E are compared after each of iterations 2-5;
 - each ADMM step on its own from the oracle's state after two iterations
   (the cold E-step of iteration 2, 12 sweeps on 200 x 200 slices);
 - a warm-started plan loaded with the oracle's state after 30 iterations:
   iteration 30's E-step starts cold (the first after lrstv_state_set),
   31 and 32 warm, in the late regime where the threshold is far below the
   columns' norms and the Jacobi runs one or two sweeps under its
   threshold-aware tolerance.
Whole iterations are held to 1e-4 max-abs (multipliers relative to mu)."""
import numpy as np
import pytest

from tests.gpu_util import dev, host, host3, load_oracle_state, maxabs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def c2(orc):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_12879_gb300 import lrstv
    from tests.golden import c2_oracle_states as cs
    states = cs.load_or_compute(orc)
    shape, Y = cs.cube()
    return lrstv, tuple(int(x) for x in states["shape"]), Y, states


def _state(orc, Y, shape, buf, mu_iters):
    st = orc.State(Y, orc.Params(n1=shape[0], n2=shape[1]))
    st.buf = np.asarray(buf, np.float64).copy()
    st.mu, st.iters = float(mu_iters[0]), int(mu_iters[1])
    return st


def _compare(pl, shape, snap, prefix, mu):
    for name in ("L", "S"):
        err = maxabs(host(pl.get(name), shape), snap[f"{prefix}_{name}"])
        assert err <= 1e-4, (prefix, name, err)
    for name in ("F", "E"):
        got = host3(pl.get(name), shape)
        for n in range(3):
            err = maxabs(got[n], snap[f"{prefix}_{name}"][n])
            assert err <= 1e-4, (prefix, name, n, err)
    for name in ("G1", "G2"):
        err = maxabs(host(pl.get(name), shape), snap[f"{prefix}_{name}"])
        assert err <= 1e-4 * max(1.0, mu), (prefix, name, err)


def test_warm_start_from_init_full_size(c2):
    lrstv, shape, Y, states = c2
    from tests.golden import c2_oracle_states as cs
    n1, n2, n3 = shape
    params = lrstv.Params.make(n1, n2, max_iter=50, flags=lrstv.FLAG_WARM_START)
    with lrstv.Plan(n1, n2, n3, params) as pl:
        pl.init(dev(Y))
        pl.iterate(cs.EARLY_LOAD)
        st = pl.stats()
        assert st.iters == 2 and st.jacobi_max_sweeps == 0  # all-cut: the t-SVT is zero
        for k in cs.EARLY_COMPARE:
            pl.iterate(1)
            st = pl.stats()
            assert st.iters == k and st.jacobi_unconverged == 0
            assert st.jacobi_max_sweeps > 0, k  # this E-step ran Jacobi sweeps
            _compare(pl, shape, states, f"early_{k}", st.mu)


def test_each_step_full_size(c2, orc):
    lrstv, shape, Y, states = c2
    n1, n2, n3 = shape
    ost = _state(orc, Y, shape, states["early_state"], states["early_mu"])
    with lrstv.Plan(n1, n2, n3, lrstv.Params.make(n1, n2)) as pl:
        s = load_oracle_state(pl, ost)
        pl.step_l_tz()
        s.step_l()
        assert maxabs(host(pl.get("L"), shape), s.get("L")) <= 1e-6
        pl.step_z()
        s.step_z()
        assert maxabs(host(pl.get("Z"), shape), s.get("Z")) <= 2e-5
        # continue from the oracle's Z so each step is compared on equal inputs
        s = load_oracle_state(pl, s)
        pl.step_fs_dual()
        s.step_f()
        s.step_s()
        Fg = host3(pl.get("F"), shape)
        for n in range(3):
            assert maxabs(Fg[n], s.get("F", n)) <= 1e-6
        assert maxabs(host(pl.get("S"), shape), s.get("S")) <= 1e-6
        # step 4 reads F and Gamma4 only (Algorithm 1's order: E before the multipliers)
        pl.step_e()
        s.step_e()
        Eg = host3(pl.get("E"), shape)
        for n in range(3):
            assert maxabs(Eg[n], s.get("E", n)) <= 2e-5
        st = pl.stats()
        assert st.jacobi_unconverged == 0 and st.jacobi_max_sweeps > 0
        s.step_dual()
        tol = 2e-6 * max(1.0, s.mu)
        for name in ("G1", "G2"):
            assert maxabs(host(pl.get(name), shape), s.get(name)) <= tol, name
        for name in ("G3", "G4"):
            got = host3(pl.get(name), shape)
            for n in range(3):
                assert maxabs(got[n], s.get(name, n)) <= 2e-5 * max(1.0, s.mu), (name, n)


def test_late_warm_iterations_full_size(c2, orc):
    lrstv, shape, Y, states = c2
    from tests.golden import c2_oracle_states as cs
    n1, n2, n3 = shape
    ost = _state(orc, Y, shape, states["late_state"], states["late_mu"])
    params = lrstv.Params.make(n1, n2, max_iter=50, flags=lrstv.FLAG_WARM_START)
    sweeps = []
    with lrstv.Plan(n1, n2, n3, params) as pl:
        load_oracle_state(pl, ost)  # the stored state is float32 already
        for k in cs.LATE_COMPARE:
            pl.iterate(1)
            st = pl.stats()
            assert st.iters == k and st.jacobi_unconverged == 0
            assert st.jacobi_max_sweeps > 0, k
            sweeps.append(st.jacobi_max_sweeps)
            _compare(pl, shape, states, f"late_{k}", float(states[f"late_{k}_mu"][0]))
    print("late sweeps (cold, warm, warm):", sweeps)
