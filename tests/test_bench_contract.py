"""The benchmark's JSON contract on the CPU: the reference arm's line for each
workload (the FP64 oracle on the host cores) carries the keys and the
metric, unit and direction of the GPU arm's line for the same workload."""
import json

import numpy as np
import pytest

import bench

KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
        "cpu_baseline", "e2e"}


def _check_line(line, metric, unit):
    assert KEYS <= set(line), KEYS - set(line)
    assert line["impl"] == "reference" and line["metric"] == metric and line["unit"] == unit
    assert line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["value"] > 0 and line["ms_per_step"] == pytest.approx(1e3 / line["value"])
    assert line["steps"] >= 1 and line["warmup"] == 0  # the units actually timed, no warm-up
    assert "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["unit"] == unit
    assert cb["cores"] >= 1 and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == unit
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def _args(**kw):
    a = dict(steps=1, warmup=0, cpu_budget=0.0, tucker=0, precision="auto")
    a.update(kw)
    return type("A", (), a)()


def test_reference_line_through_main(capsys):
    bench.main(["--impl", "reference", "--workload", "c1", "--steps", "1", "--warmup", "0",
                "--cpu-budget", "0"])
    out = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(out) == 1
    _check_line(json.loads(out[0]), bench.METRIC, bench.UNIT)


def test_metric_names_follow_the_workload():
    assert bench.metric_for(_args(), "c2") == bench.METRIC
    assert bench.metric_for(_args(), "c3") == bench.METRIC_BF16X3
    assert bench.metric_for(_args(precision="tf32x3"), "c3") == bench.METRIC
    assert bench.metric_for(_args(precision="bf16x3"), "c2") == bench.METRIC_BF16X3
    assert bench.metric_for(_args(tucker=8), "c2") == bench.METRIC_TUCKER
    assert bench.tucker_ranks(_args(), (200, 200, 80)) is None
    assert bench.tucker_ranks(_args(tucker=8), (200, 200, 80)) == (160, 160, 8)
    assert bench.tucker_ranks(_args(tucker=99), (10, 9, 4)) == (8, 7, 4)


def test_reference_tucker_line():
    line = bench.run_reference(_args(tucker=3), "c1")
    _check_line(line, bench.METRIC_TUCKER, bench.UNIT)
    assert line["config"]["tucker_ranks"] == [26, 26, 3]
    assert "TDLRSTV" in line["cpu_baseline"]["sample"]


def test_reference_batch_and_unrolled_lines(monkeypatch):
    """The batch (c4) and unrolled (c5) reference arms, on small stand-in
    recipes so that the CPU suite stays fast."""
    import synthetic
    from synthetic import Recipe
    small = [Recipe(8, 8, 4, 3, 5, (0.1, 0.1), 0.1), Recipe(6, 7, 3, 3, 5, (0.1, 0.1), 0.1)]
    monkeypatch.setattr(synthetic, "batch_recipes", lambda count, seed: small)
    line = bench.run_reference(_args(), "c4")
    _check_line(line, bench.METRIC_BATCH, bench.UNIT_BATCH)
    assert line["config"]["cubes_timed"] == 1

    monkeypatch.setitem(synthetic.RECIPES, "c5", Recipe(6, 5, 4, 3, 5, (0.1, 0.1), 0.1))
    monkeypatch.setitem(bench.UNROLL, "iters", 2)
    line = bench.run_reference(_args(), "c5")
    _check_line(line, bench.METRIC_UNROLL, bench.UNIT_UNROLL)
    assert line["config"]["pairs_timed"] == 1


def test_stage_bounds_closed_forms():
    """The per-stage bounds of a 200x200x80 iteration against their closed
    forms: stencil kernels at HBM bytes / bandwidth, the DFTs at the larger
    of FP32 ALU and HBM time, the GEMMs at three products per complex
    multiply-add at the TF32 (half of BF16) rate, the Jacobi's counted flops at
    the FP32 peak; a kernel without a stated bound is listed, not summed."""
    shape, steps = (200, 200, 80), 10
    n1, n2, n3 = shape
    N, P, h = n1 * n2 * n3, n1 * n2, n3 // 2 + 1
    per_it = {"l_tz": 1, "r2c_z": 1, "cgemm_z": 4, "c2r_z": 1, "fs_dual": 1, "r2c_e": 1,
              "jacobi": 1, "cgemm_e": 1, "c2r_e": 1, "warm_e": 5, "tucker": 1}
    kernels = {k: {"launches": v * steps, "ms_per_launch": 1.0} for k, v in per_it.items()}
    pk = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0, "sm_max_mhz": 2000.0}
    jac = 7.0e10 * steps
    peak = bench.derived_peaks(pk, "measured", None, 152)
    b = bench.stage_bounds(kernels, shape, steps, "tf32x3", jac, pk, peak)
    ms = b["ms_per_iteration"]
    fp32 = 152 * 128 * 2 * 2.0e9
    assert ms["l_tz"] == pytest.approx(13 * 4 * N / 6.0e12 * 1e3)
    assert ms["fs_dual"] == pytest.approx(23 * 4 * N / 6.0e12 * 1e3)
    assert ms["jacobi"] == pytest.approx(7.0e10 / fp32 * 1e3)
    # Z-step DFT: 4 flops per product, n3 x h products per pixel, on the ALUs
    assert ms["r2c_z"] == pytest.approx(max(4 * n3 * h * P / fp32, (4 * N + 8 * h * P) / 6.0e12) * 1e3)
    # four spatial passes of 8 P h (n1 + n2) / 2 flops, three split products, TF32 = 1e15
    assert ms["cgemm_z"] == pytest.approx(4 * 3 * 8 * P * h * (n1 + n2) // 2 / 1.0e15 * 1e3)
    assert b["without_bound"] == ["tucker"] and "tucker" not in ms
    assert b["sum_ms"] == pytest.approx(sum(ms.values()))
    # the BF16 split runs at the full BF16 rate
    b16 = bench.stage_bounds(kernels, shape, steps, "bf16x3", jac, pk, peak)["ms_per_iteration"]
    assert b16["cgemm_e"] == pytest.approx(ms["cgemm_e"] / 2)


def test_peaks_measured_or_derived():
    """Measured probes set the FP32 (larger of scalar and paired FMA) and TF32
    roofs; without them FP32 is derived from the SM count and TF32 is half of
    BF16.  The tensor fraction counts three split products per complex MAC."""
    pk = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0, "sm_max_mhz": 2000.0}
    d = bench.derived_peaks(pk, "measured", None, 148)
    assert d["fp32"] == pytest.approx(148 * 128 * 2 * 2.0e9 / 1e12)
    assert d["tf32"] == 1000.0 and "derived" in d["fp32_source"]
    probes = {u: {"tflops": v, "ms": 400.0, "clocks": {"sm_mhz": 1900.0, "reasons": []}}
              for u, v in (("fp32_fma", 70.0), ("fp32_fma2", 72.0), ("tf32_mma", 900.0),
                           ("bf16_mma", 1800.0))}
    m = bench.derived_peaks(pk, "measured", probes, 152)
    assert m["fp32"] == 72.0 and m["tf32"] == 900.0 and "fp32_fma2" in m["fp32_source"]
    shape = (200, 200, 80)
    kernels = {"cgemm_e": {"launches": 1, "ms_per_launch": 1.0},
               "cgemm_z": {"launches": 4, "ms_per_launch": 1.0}}
    fr = bench.tensor_fracs(kernels, shape, "tf32x3", m)
    assert "cgemm_z" not in fr  # side stream: its in-region time includes waits
    f = fr["cgemm_e"]
    useful = 8 * 200 * 200 * 200 * 3 * 41
    assert f["useful_tflops"] == pytest.approx(useful / 1e-3 / 1e12)
    assert f["frac"] == pytest.approx(3 * useful / 1e-3 / 1e12 / 900.0)


def test_profile_commands_parse():
    """Every `python bench.py ...` command a profile summary cites is one the
    committed benchmark accepts (the summaries' commands run committed files)."""
    import os
    import re
    import shlex
    root = os.path.dirname(bench.__file__)
    cmds = []
    for f in sorted(os.listdir(os.path.join(root, "profiles"))):
        if f.endswith(".md"):
            for line in open(os.path.join(root, "profiles", f)):
                m = re.search(r"python bench\.py([^#`\\]*)", line)
                if m:
                    cmds.append((f, shlex.split(m.group(1))))
    assert cmds
    parser = bench.build_parser()
    for f, argv in cmds:
        parser.parse_args(argv)  # exits (SystemExit) on an unknown flag or value
