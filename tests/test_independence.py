"""The structure the parity claims rest on, checked on the CPU: the FP64
oracle and the CUDA path share no code and neither imports the other, the
seeded input generators import neither, and the product path has no CPU
fallback (without a CUDA device its entry points raise)."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_2204_12879_gb300"


def _py_imports(sub):
    """Top-level names of every module imported by the .py files under sub
    (relative imports resolve to sub itself)."""
    names = set()
    for dirpath, _, files in os.walk(os.path.join(ROOT, sub)):
        for f in files:
            if not f.endswith(".py"):
                continue
            tree = ast.parse(open(os.path.join(dirpath, f)).read())
            for node in ast.walk(tree):
                if isinstance(node, ast.Import):
                    names |= {a.name.split(".")[0] for a in node.names}
                elif isinstance(node, ast.ImportFrom):
                    names.add(sub if node.level else (node.module or "").split(".")[0])
    return names


def _includes(sub, exts, quoted_only=False):
    """Headers #included by the sources under sub (only the "quoted" ones,
    i.e. not system headers, with quoted_only)."""
    pat = r'#include\s+"([^"]+)"' if quoted_only else r'#include\s+[<"]([^>"]+)[>"]'
    inc = set()
    for dirpath, _, files in os.walk(os.path.join(ROOT, sub)):
        for f in files:
            if f.endswith(exts):
                inc |= set(re.findall(pat, open(os.path.join(dirpath, f)).read()))
    return inc


def test_oracle_does_not_import_the_package():
    assert PKG not in _py_imports("oracle")


def test_package_does_not_import_the_oracle():
    assert "oracle" not in _py_imports(PKG)


def test_generators_import_neither():
    names = _py_imports("synthetic")
    assert PKG not in names and "oracle" not in names


def test_c_sources_share_no_headers():
    # the C oracle includes its own header and system headers only
    assert _includes("oracle", (".c", ".h"), quoted_only=True) <= {"lrstv_oracle.h"}
    cuda_inc = _includes(os.path.join(PKG, "csrc"), (".cu", ".cuh", ".h"))
    assert not any("oracle" in i for i in cuda_inc), cuda_inc


def test_no_cpu_fallback():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2204_12879_gb300 import lrstv
    with pytest.raises(RuntimeError, match="CUDA"):
        lrstv.Plan(8, 8, 4, lrstv.Params.make(8, 8))
    with pytest.raises(RuntimeError, match="CUDA"):
        lrstv.lrstv_check_bounded_wait(10)


def test_stored_expected_values_come_from_the_oracle_only():
    # the scripts under tests/golden that write expected values call oracle/
    # (and the seeded generators), never the CUDA path
    names = _py_imports(os.path.join("tests", "golden"))
    assert PKG not in names and "torch" not in names, names
