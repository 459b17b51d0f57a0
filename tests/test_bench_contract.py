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
