"""The allocation-free t-SVT entry point, called through the C ABI.

lrstv_tsvt_noalloc exists for callers that cannot allocate device memory when
they call the library (a plug-in whose host application owns the device
memory pool, a process that reserves its device memory up front, a loop that
must not reach the allocator).  It takes its scratch from a fixed 16 MiB
device array inside the library.  These tests check it against the
workspace-taking lrstv_tsvt on the same input, on two calls in a row (the
second call finds the first call's contents in the shared array), and that a
cube too large for the array is refused.  This file is collected last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_12879_gb300 import lrstv
    return torch, lrstv, lrstv.load()


def _cube(torch, shape, seed):
    a = np.random.default_rng(seed).standard_normal(shape).astype(np.float32)
    return torch.from_numpy(np.ascontiguousarray(a.reshape(-1, order="F"))).cuda()


@pytest.mark.parametrize("shape,t", [((24, 20, 9), 1.5), ((20, 24, 8), 0.7), ((64, 64, 31), 4.0)])
def test_noalloc_matches_workspace_tsvt_on_two_calls(env, shape, t):
    torch, lrstv, lib = env
    A = _cube(torch, shape, 3)
    B = _cube(torch, shape, 4)
    n1, n2, n3 = shape
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    tol = 2e-5  # the t-SVT parity tolerance, relative to max |A|
    for X in (A, B):  # two calls in a row through the shared scratch array
        ref = lrstv.lrstv_tsvt(X, shape, t)
        out = torch.full_like(X, float("nan"))
        sw = ctypes.c_int(0)
        rc = lib.lrstv_tsvt_noalloc(ctypes.c_void_p(X.data_ptr()), n1, n2, n3, t,
                                    ctypes.c_void_p(out.data_ptr()), ctypes.byref(sw), stream)
        assert rc == 0, lrstv.status_string(rc)
        torch.cuda.synchronize()
        assert sw.value > 0
        err = float((out - ref).abs().max())
        assert err <= tol * float(X.abs().max())


def test_noalloc_refuses_cubes_beyond_its_scratch(env):
    torch, lrstv, lib = env
    shape = (200, 200, 80)  # needs about 39 MB of scratch
    A = torch.zeros(200 * 200 * 80, device="cuda")
    out = torch.zeros_like(A)
    rc = lib.lrstv_tsvt_noalloc(ctypes.c_void_p(A.data_ptr()), *shape, 1.0,
                                ctypes.c_void_p(out.data_ptr()), None, None)
    assert rc == 2  # LRSTV_ERR_SHAPE
    assert lib.lrstv_tsvt_noalloc(None, 8, 8, 4, 1.0, None, None, None) == 1
