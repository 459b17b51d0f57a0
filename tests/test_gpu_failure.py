"""Failure detection on the GPU without a fault: the tensor-core GEMM's
bounded barrier wait is made to run out (an mbarrier that nothing arrives
at), and the probe must record the timeout, free its tensor memory and leave
the context usable for a tensor-core plan that follows."""
import time

import numpy as np
import pytest

from tests.gpu_util import dev, f32, host, maxabs

pytestmark = pytest.mark.gpu

# the tensor-core GEMM's bound on a barrier wait, in tries (include/lrstv.h,
# lrstv_check_bounded_wait)
GEMM_WAIT_TRIES = 250000


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_12879_gb300 import lrstv
    lrstv.load()
    return lrstv


def test_bounded_wait_completes_when_the_phase_completes(L):
    assert L.lrstv_check_bounded_wait(1000, arrive=True) == (0, 32)


def test_bounded_wait_runs_out_and_frees_tensor_memory(L, orc):
    t0 = time.perf_counter()
    assert L.lrstv_check_bounded_wait(100) == (1, 32)
    t1 = time.perf_counter()
    if t1 - t0 < 0.5:
        # a longer wait, to time one try of the wait (allocation and launch
        # overheads cancel in the difference)
        assert L.lrstv_check_bounded_wait(10000) == (1, 32)
        t2 = time.perf_counter()
        per_try = max((t2 - t1) - (t1 - t0), 0.0) / 9900
        print("bounded wait: %.3g us per try; the GEMM's %d tries last %.3g s"
              % (per_try * 1e6, GEMM_WAIT_TRIES, per_try * GEMM_WAIT_TRIES))
        # a wait that ran out ends within seconds, not minutes
        assert per_try * GEMM_WAIT_TRIES <= 5.0
    # the context is usable and the tensor memory free: a tensor-core plan
    # runs and matches the oracle
    from synthetic import Recipe, make_cube
    shape = (16, 16, 8)
    _, noisy = make_cube(Recipe(*shape, 3, 6, (0.1, 0.1), 0.1), 1)
    Y = f32(noisy)
    with L.Plan(*shape, L.Params.make(16, 16, max_iter=3)) as pl:
        X, _, st = pl.run(dev(Y), stats=True)
        X = host(X, shape)
    assert st.gemm_errors == 0 and st.jacobi_unconverged == 0
    ref = orc.State(Y, orc.Params(n1=16, n2=16))
    ref.iterate(3)
    assert maxabs(X, ref.X) <= 1e-4


def test_bounded_wait_arguments(L):
    for tries in (0, -5, GEMM_WAIT_TRIES + 1):
        with pytest.raises(L.LrstvError, match="status 1"):
            L.lrstv_check_bounded_wait(tries)
