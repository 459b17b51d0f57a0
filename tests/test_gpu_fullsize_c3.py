"""Parity of the E-update (eq. E_solution, the t-SVT of Theorem 4.2 on each
gradient tensor) at the mixed-precision workload's full size, 256x256x191,
in the configuration bench.py times there (warm start, 3xBF16 tensor-core
GEMMs and mode-3 DFTs, the default Jacobi schedule), and in the FP32-accurate
3xTF32 configuration, against the FP64 oracle's E-step on the same state.

The state is synthetic: the seeded 256x256x191 mixed-noise cube as Y, F_n =
c D_n Y (c = 0.05, so that the threshold alpha/mu at mu = mu0 rho^4 sits
inside each Fourier slice's spectrum: about 44% of the singular values
of the 288 slices of 256 x 256 are kept) and Gamma4_n = 0.01 mu xi_n with
seeded standard normal xi_n, so the E-step's input F - Gamma4/mu carries
the multiplier term.  Every slice runs cold Jacobi sweeps (the first E-step
after a state is loaded).  E is held to the 1e-4 max-abs bound of the
iteration, and Gamma4 = Gamma4 + mu (E - F) to 1e-4 mu.  One oracle E-step
at this size takes about a minute of host time."""
import numpy as np
import pytest

from tests.gpu_util import host3, load_oracle_state, maxabs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

C_F = 0.05
K_MU = 4


@pytest.fixture(scope="module")
def c3(orc):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_12879_gb300 import lrstv
    from synthetic import RECIPES, make_cube
    r = RECIPES["c3"]
    _, Y = make_cube(r, 3)
    Y = Y.astype(np.float32).astype(np.float64)
    shape = r.shape
    p = lrstv.Params.make(shape[0], shape[1])
    mu = float(p.mu0) * float(p.rho) ** K_MU
    st = orc.State(Y, orc.Params(n1=shape[0], n2=shape[1]))
    rng = np.random.default_rng(31)
    for n in range(3):
        st.set("F", C_F * (np.roll(Y, -1, axis=n) - Y), n)
        st.set("G4", 0.01 * mu * rng.standard_normal(shape), n)
    st.mu, st.iters = mu, K_MU
    # the oracle's E-step (and Gamma4) on the float32-rounded state, once
    s32 = st.copy()
    s32.buf = s32.buf.astype(np.float32).astype(np.float64)
    s32.step_e()
    E = np.stack([s32.get("E", n) for n in range(3)])
    s32.step_dual()
    G4 = np.stack([s32.get("G4", n) for n in range(3)])
    return lrstv, shape, st, E, G4, mu


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3"])
def test_e_step_256x256x191(c3, precision):
    lrstv, shape, st, E_ref, G4_ref, mu = c3
    n1, n2, n3 = shape
    flags = lrstv.FLAG_WARM_START | (lrstv.FLAG_BF16X3 if precision == "bf16x3" else 0)
    with lrstv.Plan(n1, n2, n3, lrstv.Params.make(n1, n2, flags=flags)) as pl:
        load_oracle_state(pl, st)
        pl.step_e()
        s = pl.stats()
        E = host3(pl.get("E"), shape)
        G4 = host3(pl.get("G4"), shape)
    assert s.jacobi_unconverged == 0 and s.jacobi_max_sweeps > 0
    errs = [maxabs(E[n], E_ref[n]) for n in range(3)]
    print(f"{precision}: E max-abs {errs}, |E| max {np.abs(E_ref).max():.3f}, "
          f"sweeps {s.jacobi_max_sweeps}")
    for n in range(3):
        # the threshold keeps part of the spectrum and cuts part of it
        B = st.get("F", n) - st.get("G4", n) / mu
        assert np.abs(E_ref[n]).max() > 0.05 * np.abs(B).max()
        assert maxabs(E_ref[n], B) > 0.05 * np.abs(B).max()
    for n in range(3):
        assert errs[n] <= 1e-4, (n, errs[n])
        assert maxabs(G4[n], G4_ref[n]) <= 1e-4 * mu, n
