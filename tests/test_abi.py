"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/lrstv.h declares; argument checks that precede any CUDA call return
their status codes.  No GPU needed."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lrstv.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lrstv_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2204_12879_gb300 import builder, lrstv
    builder.build()
    return lrstv.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lrstv_denoise", "lrstv_plan_create", "lrstv_init", "lrstv_step_l_tz",
                 "lrstv_step_z", "lrstv_step_fs_dual", "lrstv_step_e", "lrstv_step_mu",
                 "lrstv_state_get", "lrstv_state_set", "lrstv_diff", "lrstv_diff_adjoint",
                 "lrstv_tsvt", "lrstv_soft_threshold", "lrstv_status_string"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2204_12879_gb300 import builder
    out = subprocess.run(["nm", "-D", "--defined-only", builder.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\b(lrstv_[a-z_0-9]+)\b", out))
    for name in declared_functions():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_binding_covers_the_header():
    from paper_2204_12879_gb300 import lrstv
    assert sorted(lrstv.EXPORTED) == declared_functions()


def test_build_targets_sm_103a_only():
    from paper_2204_12879_gb300 import builder
    assert builder.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings(lib):
    from paper_2204_12879_gb300 import lrstv
    assert lrstv.status_string(0) == "ok"
    assert "shape" in lrstv.status_string(2)
    assert lib.lrstv_max_spatial() == 512


def test_argument_errors_before_any_cuda_call(lib):
    from paper_2204_12879_gb300 import lrstv
    p = lrstv.Params.make(8, 8)
    h = ctypes.c_void_p()
    assert lib.lrstv_plan_create(0, 8, 8, ctypes.byref(p), ctypes.byref(h)) == 1
    assert lib.lrstv_plan_create(8, 600, 8, ctypes.byref(p), ctypes.byref(h)) == 2
    assert lib.lrstv_plan_create(8, 8, 5000, ctypes.byref(p), ctypes.byref(h)) == 2
    assert lib.lrstv_plan_create(8, 8, 8, None, ctypes.byref(h)) == 1
    bad = lrstv.Params.make(8, 8, mu0=-1.0)
    assert lib.lrstv_plan_create(8, 8, 8, ctypes.byref(bad), ctypes.byref(h)) == 1
    # LRSTV_FLAG_UNROLL_RECOMPUTE belongs to the unrolled form; 1 << 13 is no flag
    for f in (lrstv.FLAG_UNROLL_RECOMPUTE, 1 << 13):
        bad = lrstv.Params.make(8, 8, flags=f)
        assert lib.lrstv_plan_create(8, 8, 8, ctypes.byref(bad), ctypes.byref(h)) == 1
    # the unrolled form refuses the plan-only flags and unknown bits before any CUDA call
    w = (ctypes.c_float * 3)(1, 1, 1)
    for f in (lrstv.FLAG_ISO_TV, lrstv.FLAG_BF16X3, lrstv.FLAG_GRAPH, 1 << 13):
        assert lib.lrstv_unroll_create(8, 8, 4, 1, 2, w, f, ctypes.byref(h)) == 1, f
    # the split-BF16 GEMMs exist on the tensor-core path only
    bad = lrstv.Params.make(8, 8, flags=lrstv.FLAG_BF16X3 | lrstv.FLAG_SIMT_GEMM)
    assert lib.lrstv_plan_create(8, 8, 8, ctypes.byref(bad), ctypes.byref(h)) == 1
    assert lib.lrstv_plan_destroy(None) == 1
    assert lib.lrstv_plan_autotune(None, None, 0, 0, None, None, None) == 1
    assert lib.lrstv_step_z(None, None) == 1
    assert lib.lrstv_soft_threshold(None, 5, 0.1, None, None) == 1
    sz = ctypes.c_size_t()
    assert lib.lrstv_tsvt_workspace_size(200, 200, 80, ctypes.byref(sz)) == 0
    assert sz.value >= 41 * 200 * 200 * 8 * 3
    assert lib.lrstv_zsolve_workspace_size(7, 0, 3, ctypes.byref(sz)) == 1
    # the bounded-wait probe: tries within 1 .. the GEMM's limit, both outputs
    t, n = ctypes.c_int(), ctypes.c_int()
    assert lib.lrstv_check_bounded_wait(0, 0, ctypes.byref(t), ctypes.byref(n)) == 1
    assert lib.lrstv_check_bounded_wait(250001, 0, ctypes.byref(t), ctypes.byref(n)) == 1
    assert lib.lrstv_check_bounded_wait(10, 0, None, ctypes.byref(n)) == 1
    assert lib.lrstv_check_bounded_wait(10, 0, ctypes.byref(t), None) == 1
    assert lib.lrstv_plan_tucker_factor(None, 0, None, None) == 1
    # the throughput probe: a known unit, work in 1 .. 2^40, both outputs
    d = ctypes.c_double()
    assert lib.lrstv_peak_probe(4, 10, ctypes.byref(d), ctypes.byref(d)) == 1
    assert lib.lrstv_peak_probe(0, 0, ctypes.byref(d), ctypes.byref(d)) == 1
    assert lib.lrstv_peak_probe(0, 10, None, ctypes.byref(d)) == 1
    # one band above the largest n3 a plan takes
    assert lib.lrstv_plan_create(2, 2, 4097, ctypes.byref(p), ctypes.byref(h)) == 2


def test_flag_constants_match_header():
    """The binding's FLAG_* constants are the header's LRSTV_FLAG_* values."""
    import re
    from paper_2204_12879_gb300 import lrstv
    with open(os.path.join(ROOT, "include", "lrstv.h")) as f:
        flags = dict(re.findall(r"#define LRSTV_FLAG_(\w+) (\d+)u", f.read()))
    assert len(flags) >= 12
    for name, val in flags.items():
        assert getattr(lrstv, "FLAG_" + name) == int(val), name
