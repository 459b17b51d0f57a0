"""GPU parity of the mixed-precision mode (LRSTV_FLAG_BF16X3): the tensor-core
GEMMs split each FP32 operand into two BF16 halves and form three products
with FP32 accumulation.

Bound.  A BF16 half carries 8 significant bits (unit roundoff 2^-9), so
|x - hi - lo| <= 2^-18 |x| and the dropped lo*lo term is at most 2^-18 |a b|:
about 3 * 2^-18 ~ 1.1e-5 relative error per product term, against 2^-21 for
3xTF32.  A DFT pass of length n sums n terms of random phase, so a transformed
value carries ~1e-5 of its magnitude; over a whole denoise these errors are
damped by the thresholds like the FP32 path's rounding.  Steps are held to
2e-4 and whole runs to 1e-3 max-abs and 0.01 dB MPSNR against the FP64
oracle (the FP32 path's bounds are 2e-5 / 1e-4 / 0.01 dB); the measured
errors are printed.
"""
import numpy as np
import pytest

from tests.gpu_util import dev, f32, host, host3, load_oracle_state, maxabs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_12879_gb300 import lrstv
    lrstv.load()
    return lrstv


def _noisy(shape, seed):
    from synthetic import Recipe, make_cube
    clean, noisy = make_cube(Recipe(*shape, 4, 12, (0.1, 0.1), 0.1), seed)
    return clean, f32(noisy)


def test_bf16x3_steps_match_oracle(L, orc):
    """One Z-step and one E-step from an oracle state after 4 iterations."""
    shape = (32, 32, 16)
    _, Y = _noisy(shape, 11)
    st = orc.State(Y, orc.Params(n1=32, n2=32))
    st.iterate(4)
    with L.Plan(*shape, L.Params.make(32, 32, flags=L.FLAG_BF16X3)) as pl:
        s = load_oracle_state(pl, st)
        pl.step_l_tz()
        pl.step_z()
        s.step_l()
        s.step_z()
        ez = maxabs(host(pl.get("Z"), shape), s.get("Z"))
        # the plan fuses F, S and Gamma1..3 ahead of E (Gamma4 moves with E);
        # the oracle's E reads the same F and Gamma4
        pl.step_fs_dual()
        s.step_f()
        pl.step_e()
        s.step_e()
        E = host3(pl.get("E"), shape)
        ee = max(maxabs(E[n], s.get("E", n)) for n in range(3))
    print("bf16x3 step errors: Z", ez, "E", ee)
    assert ez <= 2e-4
    assert ee <= 2e-4


@pytest.mark.parametrize("shape,iters,flags", [((32, 32, 16), 20, 0), ((37, 29, 11), 15, 0),
                                                ((64, 64, 31), 50, 32)])
def test_bf16x3_run_matches_oracle(L, orc, shape, iters, flags):
    from synthetic import mpsnr
    clean, Y = _noisy(shape, 1)
    n1, n2, _ = shape
    p = L.Params.make(n1, n2, max_iter=iters, flags=L.FLAG_BF16X3 | flags)
    with L.Plan(*shape, p) as pl:
        X, S, stats = pl.run(dev(Y), stats=True)
        X, S = host(X, shape), host(S, shape)
    ost = orc.State(Y, orc.Params(n1=n1, n2=n2))
    ost.iterate(iters)
    d = mpsnr(X, clean) - mpsnr(ost.X, clean)
    print(shape, iters, "bf16x3 max-abs", maxabs(X, ost.X), "S", maxabs(S, ost.get("S")), "dMPSNR", d)
    assert stats.iters == iters and stats.jacobi_unconverged == 0 and stats.gemm_errors == 0
    assert maxabs(X, ost.X) <= 1e-3
    assert maxabs(S, ost.get("S")) <= 1e-3
    assert abs(d) <= 0.01


def test_bf16x3_full_size_equal_quality(L):
    """256x256x191 mixed-noise cube, 60 iterations: the mixed-precision run
    against the FP32-accurate (3xTF32) run of the same plan, which the oracle
    pins at smaller sizes: same MPSNR to 0.01 dB."""
    import torch
    from synthetic import RECIPES, make_cube, mpsnr
    r = RECIPES["c3"]
    clean, Y = make_cube(r, 3)
    Y = f32(Y)
    shape = r.shape
    out = {}
    for name, flags in (("tf32x3", L.FLAG_WARM_START), ("bf16x3", L.FLAG_WARM_START | L.FLAG_BF16X3)):
        p = L.Params.make(shape[0], shape[1], max_iter=60, flags=flags)
        with L.Plan(*shape, p) as pl:
            X, _ = pl.run(dev(Y))
            torch.cuda.synchronize()
            out[name] = host(X, shape)
    d = mpsnr(out["bf16x3"], clean) - mpsnr(out["tf32x3"], clean)
    diff = maxabs(out["bf16x3"], out["tf32x3"])
    print("256x256x191: MPSNR tf32x3", mpsnr(out["tf32x3"], clean), "bf16x3",
          mpsnr(out["bf16x3"], clean), "max-abs between them", diff)
    assert abs(d) <= 0.01
    assert diff <= 5e-3


def test_bf16x3_needs_the_tensor_core_path(L):
    with pytest.raises(L.LrstvError, match="status 1"):
        L.Plan(8, 8, 4, L.Params.make(8, 8, flags=L.FLAG_BF16X3 | L.FLAG_SIMT_GEMM))


def test_bf16x3_differs_from_tf32x3(L):
    """The flag reaches the kernels: the two splits round differently."""
    import torch
    shape = (32, 32, 16)
    _, Y = _noisy(shape, 2)
    outs = []
    for flags in (0, L.FLAG_BF16X3):
        with L.Plan(*shape, L.Params.make(32, 32, max_iter=3, flags=flags)) as pl:
            X, _ = pl.run(dev(Y))
            torch.cuda.synchronize()
            outs.append(host(X, shape))
    assert 0 < maxabs(outs[0], outs[1]) <= 1e-3
