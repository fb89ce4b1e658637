"""bench.py's reference arm (the FP64 oracle timed on the host) prints the
JSON line the benchmark contract asks for; the oracle timing itself is
replaced by a fixed figure here so the test stays quick."""
import json
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_reference_arm_json_line(monkeypatch, capsys):
    monkeypatch.setattr(bench, "oracle_sample",
                        lambda seconds_target=15.0, max_gates=None, one_core=True: (100.0, "stub sample", 8, None))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"])
    bench.main()
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 8
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["ms_per_step"] == pytest.approx(100.0 * 1e3)
    assert "workload" in line["config"]
