"""bench.py's reference arm (the FP64 oracle timed on the host) prints the
JSON line the benchmark contract asks for, without loading the library; the
oracle's slice timing is replaced by fixed figures here so the test stays
quick."""
import json
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_reference_arm_json_line(monkeypatch, capsys):
    calls = []

    def stub(n_samples=1, first=0):
        calls.append(n_samples)
        flops = {"job": 256 * 1e12, "per_slice": 0.0, "invariant": 256 * 1e12}
        return [2.0] * n_samples, 256, flops, 8

    monkeypatch.setattr(bench, "oracle_slices", stub)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"])
    bench.main()
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert calls == [5]
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 8
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    # a step is one whole slice (2 s); the job is 256 of them
    assert line["ms_per_step"] == pytest.approx(2.0 * 1e3)
    assert line["value"] == pytest.approx(256e12 / (256 * 2.0) / 1e12)
    assert "workload" in line["config"]


def test_reference_arm_reads_the_recorded_plan():
    # the recorded path and flops exist and are consistent with the job
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    import dump_plan
    edges, leaves, steps, flops = dump_plan.read(bench.GRID30_PLAN, with_flops=True)
    assert len(edges) == 8 and len(steps) == len(leaves) - 1
    assert flops["job"] == pytest.approx(flops["per_slice"] * 256 + flops["invariant"])


def test_time_space_case_runs_on_the_host(monkeypatch, capsys):
    # the planner's time-space table needs no GPU: one line per workload and
    # cap, every plan within its cap, annealing no worse than its greedy start
    monkeypatch.setattr(sys, "argv", ["bench.py", "--case", "time_space", "--anneal-iters", "2000",
                                      "--path-trials", "1"])
    bench.main()
    rows = [json.loads(l) for l in capsys.readouterr().out.strip().splitlines()]
    assert len(rows) == 15
    assert {r["cap_log2"] for r in rows} == {24, 26, 28, 30, 32}
    for r in rows:
        for k in ("greedy", "annealed_flops", "annealed_roofline"):
            assert r[k]["max_log2_elems"] <= r["cap_log2"] and r[k]["flops"] > 0
        assert r["annealed_flops"]["flops"] <= 1.01 * r["greedy"]["flops"]
