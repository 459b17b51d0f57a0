"""The allocation-free t-SVT entry point, called through the C ABI.

lrstv_tsvt_noalloc exists for callers that cannot allocate device memory when
they call the library (a plug-in whose host application owns the device
memory pool, a process that reserves its device memory up front, a loop that
must not reach the allocator).  It takes its scratch from a fixed 16 MiB
device array inside the library.  These tests check it against the
workspace-taking lrstv_tsvt and against the FP64 oracle on the same input, on
two calls in a row (the second call finds the first call's contents in the
shared array), with and without the synchronising sweep count, that device
memory does not change across a call once the library is loaded, and that a
cube too large for the array is refused.  This file is collected last."""
import ctypes

import numpy as np
import pytest

from tests.gpu_util import host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_12879_gb300 import lrstv
    return torch, lrstv, lrstv.load()


def _data(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def _dev(torch, a):
    flat = np.ascontiguousarray(np.asarray(a, np.float32).reshape(-1, order="F"))
    return torch.from_numpy(flat).cuda()


def _call(torch, lib, X, shape, t, out, with_sweeps):
    n1, n2, n3 = shape
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    sw = ctypes.c_int(-12345)
    rc = lib.lrstv_tsvt_noalloc(ctypes.c_void_p(X.data_ptr()), n1, n2, n3, t,
                                ctypes.c_void_p(out.data_ptr()),
                                ctypes.byref(sw) if with_sweeps else None, stream)
    return rc, sw.value


@pytest.mark.parametrize("shape,t", [((24, 20, 9), 1.5), ((20, 24, 8), 0.7), ((64, 64, 31), 4.0)])
def test_noalloc_matches_workspace_tsvt_and_oracle_on_two_calls(env, orc, shape, t):
    torch, lrstv, lib = env
    tol = 2e-5  # the t-SVT parity tolerance, relative to max |A|
    for seed, with_sweeps in ((3, True), (4, False)):  # two calls in a row, shared array
        a = np.asarray(_data(shape, seed), np.float32).astype(np.float64)
        X = _dev(torch, a)
        ref, ref_sw = lrstv.lrstv_tsvt(X, shape, t, sweeps=True)
        out = torch.full_like(X, float("nan"))
        rc, sw = _call(torch, lib, X, shape, t, out, with_sweeps)
        assert rc == 0, lrstv.status_string(rc)
        torch.cuda.synchronize()  # the call without sweeps does not synchronise
        scale = float(np.abs(a).max())
        assert float((out - ref).abs().max()) <= tol * scale
        want, orc_sw = orc.tsvt(a, t)
        assert orc_sw > 0
        assert float(np.abs(host(out, shape) - want).max()) <= tol * scale
        if with_sweeps:
            assert sw == ref_sw and sw > 0  # same kernels, same count
        else:
            assert sw == -12345  # NULL sweeps_host: nothing written


def test_noalloc_all_cut_cube_runs_no_sweep(env, orc):
    torch, lrstv, lib = env
    shape = (16, 12, 6)
    a = np.asarray(0.01 * _data(shape, 9), np.float32).astype(np.float64)
    t = 10.0  # above every Fourier slice's Frobenius norm: the t-SVT is zero
    X = _dev(torch, a)
    out = torch.full_like(X, float("nan"))
    rc, sw = _call(torch, lib, X, shape, t, out, True)
    assert rc == 0 and sw == 0
    assert float(out.abs().max()) == 0.0
    want, _ = orc.tsvt(a, t)
    assert float(np.abs(want).max()) == 0.0


def test_noalloc_call_leaves_device_memory_unchanged(env):
    torch, lrstv, lib = env
    shape = (32, 32, 16)
    X = _dev(torch, _data(shape, 5))
    out = torch.empty_like(X)
    assert _call(torch, lib, X, shape, 1.0, out, True)[0] == 0  # modules loaded by now
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    rc, sw = _call(torch, lib, X, shape, 1.0, out, True)
    free1, _ = torch.cuda.mem_get_info()
    assert rc == 0 and sw > 0
    assert free1 == free0


def test_noalloc_refuses_cubes_beyond_its_scratch(env):
    torch, lrstv, lib = env
    shape = (200, 200, 80)  # needs about 39 MB of scratch
    A = torch.zeros(200 * 200 * 80, device="cuda")
    out = torch.zeros_like(A)
    rc = lib.lrstv_tsvt_noalloc(ctypes.c_void_p(A.data_ptr()), *shape, 1.0,
                                ctypes.c_void_p(out.data_ptr()), None, None)
    assert rc == 2  # LRSTV_ERR_SHAPE
    assert lib.lrstv_tsvt_noalloc(None, 8, 8, 4, 1.0, None, None, None) == 1
    # the scalar and shape checks of lrstv_tsvt
    p = ctypes.c_void_p(A.data_ptr())
    assert lib.lrstv_tsvt_noalloc(p, 8, 8, 4, float("inf"), p, None, None) == 1
    assert lib.lrstv_tsvt_noalloc(p, 8, 8, 4, -1.0, p, None, None) == 1
    assert lib.lrstv_tsvt_noalloc(p, 0, 8, 4, 1.0, p, None, None) == 1
    assert lib.lrstv_tsvt_noalloc(p, 8, 8, 5000, 1.0, p, None, None) == 2
