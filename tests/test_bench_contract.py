"""The benchmark's reference line (``bench.py --impl reference``) on the CPU.

The reference arm times the FP64 oracle on the host cores and prints one JSON line that the
GPU arm's line is divided by, so its keys, units and self-consistency are checked here on a
tiny sample (2 worker processes, 4 steps each) instead of the bounded sample of the real run.
"""
import argparse
import contextlib
import io
import json
import os
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _run(monkeypatch, env, jsonl=None):
    real = bench.oracle_throughput
    monkeypatch.setattr(bench, "oracle_throughput", lambda M_sample=200: real(cores=2, M_sample=4))
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    args = argparse.Namespace(steps=2, warmup=1, jsonl=jsonl)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args)
    return buf.getvalue().strip()


def test_reference_line_keys_and_consistency(monkeypatch):
    out = _run(monkeypatch, {"WORLD_SIZE": "1", "RANK": "0"})
    lines = out.splitlines()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0
    # the same workload as the GPU arm's line, with the precision and sample named
    cfg = d["config"]
    assert cfg["B"] == bench.B_FULL and cfg["M"] == bench.M_FULL and cfg["N"] == 64 and cfg["K"] == 12
    assert "workload" in cfg and "sample" in cfg
    assert abs(d["ms_per_step"] - bench.B_FULL * bench.M_FULL / d["value"] * 1e3) < 1e-6 * d["ms_per_step"]
    cb = d["cpu_baseline"]
    assert cb["value"] == d["value"] and cb["unit"] == d["unit"] and cb["kind"] == "oracle"
    assert cb["cores"] == 2 and "4 steps" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_line_only_on_rank_zero(monkeypatch):
    assert _run(monkeypatch, {"WORLD_SIZE": "2", "RANK": "1"}) == ""


def test_reference_line_appended_to_a_jsonl_file(monkeypatch, tmp_path):
    path = tmp_path / "runs.jsonl"
    path.write_text('{"earlier": 1}\n')
    out = _run(monkeypatch, {"WORLD_SIZE": "1", "RANK": "0"}, jsonl=str(path))
    lines = path.read_text().splitlines()
    assert len(lines) == 2 and json.loads(lines[0]) == {"earlier": 1}
    assert json.loads(lines[1]) == json.loads(out)
