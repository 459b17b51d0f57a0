"""The plan autotuner (lrstv_plan_autotune): it times whole short denoises
for each combination of the allowed flags (GEMM and mode-3 DFT engines,
Jacobi schedule, warm start), keeps the fastest, and leaves a plan that still
meets the FP32 parity bound against the FP64 oracle."""
import numpy as np
import pytest

from tests.gpu_util import dev, f32, host, maxabs

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


@pytest.mark.parametrize("shape", [(32, 32, 16), (64, 64, 31)])
def test_autotune_keeps_a_candidate_and_parity(L, orc, shape):
    clean, Y = _noisy(shape, 3)
    n1, n2, _ = shape
    # the default search: GEMM engine, mode-3 DFT engine, Jacobi schedule and
    # panel width, warm start
    allowed = (L.FLAG_SIMT_GEMM | L.FLAG_SIMT_DFT | L.FLAG_JACOBI_PER_SLICE |
               L.FLAG_JACOBI_PANEL16 | L.FLAG_WARM_START)
    with L.Plan(*shape, L.Params.make(n1, n2, max_iter=20, flags=L.FLAG_GRAPH)) as pl:
        flags, ms = pl.autotune(dev(Y), iters=10)
        assert (flags & ~allowed) == L.FLAG_GRAPH  # only the allowed bits move
        assert ms > 0.0
        X, S = pl.run(dev(Y))
        X = host(X, shape)
    print(shape, "autotune kept flags", flags, "in", ms, "ms")
    ost = orc.State(Y, orc.Params(n1=n1, n2=n2))
    ost.iterate(20)
    assert maxabs(X, ost.X) <= 1e-4


def test_autotune_with_nothing_allowed_keeps_the_flags(L):
    shape = (16, 16, 8)
    _, Y = _noisy(shape, 4)
    with L.Plan(*shape, L.Params.make(16, 16, max_iter=4, flags=L.FLAG_WARM_START)) as pl:
        flags, ms = pl.autotune(dev(Y), allowed=0)
        assert flags == L.FLAG_WARM_START and ms > 0.0


def test_autotune_skips_rejected_combinations(L):
    """With the split-BF16 GEMMs on, the SIMT engine is not a candidate."""
    shape = (16, 16, 8)
    _, Y = _noisy(shape, 5)
    with L.Plan(*shape, L.Params.make(16, 16, max_iter=4, flags=L.FLAG_BF16X3)) as pl:
        flags, _ = pl.autotune(dev(Y))
        assert flags & L.FLAG_BF16X3 and not flags & L.FLAG_SIMT_GEMM


def test_autotune_may_choose_the_bf16_split(L, orc):
    """With LRSTV_FLAG_BF16X3 allowed the tuner times both splits (never with
    the SIMT GEMMs), and the plan it leaves meets the 3xBF16 bound (1e-3
    against the FP64 oracle, as the mixed-precision tests hold it)."""
    shape = (24, 20, 9)
    clean, Y = _noisy(shape, 7)
    allowed = L.FLAG_BF16X3 | L.FLAG_SIMT_GEMM | L.FLAG_WARM_START
    with L.Plan(*shape, L.Params.make(24, 20, max_iter=6)) as pl:
        flags, ms = pl.autotune(dev(Y), allowed=allowed)
        assert ms > 0.0 and (flags & ~allowed) == 0
        assert not (flags & L.FLAG_BF16X3 and flags & L.FLAG_SIMT_GEMM)
        X, _ = pl.run(dev(Y))
        X = host(X, shape)
    ost = orc.State(Y, orc.Params(n1=24, n2=20))
    ost.iterate(6)
    assert maxabs(X, ost.X) <= 1e-3


def test_autotune_argument_errors(L):
    shape = (8, 8, 4)
    _, Y = _noisy(shape, 6)
    with L.Plan(*shape, L.Params.make(8, 8)) as pl:
        with pytest.raises(L.LrstvError, match="status 1"):
            pl.autotune(dev(Y), allowed=L.FLAG_GRAPH)
        with pytest.raises(L.LrstvError, match="status 1"):
            pl.autotune(dev(Y), iters=-1)
