"""bench.py's reference arm and CPU baseline (no GPU): the oracle timed on host cores
over bounded random item ranges, and the JSON line the reference arm prints."""
import argparse
import json

import bench
from paper_1406_1215_gb300 import inputs


def test_cpu_baseline_times_the_oracle_on_host_cores():
    w, seed = inputs.workload("pl_n1e5")
    cb = bench.cpu_baseline(w, seed, budget_s=2.0, cores=2)
    assert cb["kind"] == "oracle" and cb["unit"] == "edges/s" and cb["cores"] == 2
    assert cb["value"] > 0 and abs(cb["per_core"] * 2 - cb["value"]) < 1e-6 * cb["value"]
    assert "2 processes" in cb["sample"] and "random ranges" in cb["sample"]


def test_reference_line(monkeypatch, capsys):
    fake = {"value": 1.5e7, "unit": "edges/s", "cores": 3, "kind": "oracle", "per_core": 5e6,
            "sample": "3 processes x 1.0 s"}
    monkeypatch.setattr(bench, "cpu_baseline", lambda w, seed, budget_s=16.0, cores=None: dict(fake))
    args = argparse.Namespace(workload="pl_n1e7", steps=2, warmup=1)
    bench.run_reference(args, rank=1, world=2)  # other ranks print nothing
    assert capsys.readouterr().out == ""
    bench.run_reference(args, rank=0, world=1)
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["value"] == 1.5e7 and line["unit"] == "edges/s" and line["steps"] == 2 and line["warmup"] == 1
    assert line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["e2e"] == {"value": 1.5e7, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 3
    assert line["config"]["workload"].startswith("chung-lu power law n=1e7")
    assert line["metric"] == bench.METRIC
