"""The benchmark's reference arm (complete evaluations of the CPU oracle at
8^3 x 4) prints one JSON line with the benchmark contract's keys.  A complete
oracle evaluation takes minutes on a few cores, so the oracle's timing is
stubbed here (the line's arithmetic and keys are what is checked); the arm
itself needs no GPU."""
import io
import json
import os
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_json_line(monkeypatch):
    times = iter([40.0, 30.0, 34.0, 32.0, 31.0])
    monkeypatch.setattr(bench, "oracle_eval", lambda: (next(times), None))
    args = bench.argparse.Namespace(steps=20, warmup=3)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, 0, 1)
    lines = [ln for ln in buf.getvalue().splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in j, key
    # one warm-up, then REF_MAX_STEPS complete evaluations (30, 34, 32, 31 s): median 31.5 s
    assert j["steps"] == bench.REF_MAX_STEPS == 4 and j["steps_requested"] == 20 and j["warmup"] == 1
    assert abs(j["ms_per_step"] - 31500.0) < 1e-6 and abs(j["value"] - 1 / 31.5) < 1e-12
    assert j["unit"] == "evals/s" and j["higher_is_better"] is True
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == j["value"] and cb["cores"] >= 1
    assert "no extrapolation" in cb["sample"]
    e = j["e2e"]
    assert e["value"] == j["value"] and e["unit"] == j["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_silent(monkeypatch):
    monkeypatch.setattr(bench, "oracle_eval", lambda: (_ for _ in ()).throw(AssertionError("rank 1 ran work")))
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(bench.argparse.Namespace(steps=20, warmup=3), 1, 2)
    assert buf.getvalue() == ""
