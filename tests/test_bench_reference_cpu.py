"""bench.py's reference arm (the oracle on the host cores) at a tiny size:
it must print one JSON line with the keys the harness reads."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--ref-L", "3", "--steps", "2",
           "--warmup", "1"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "config", "cpu_baseline", "e2e"):
        assert key in rec, key
    assert rec["value"] > 0 and rec["unit"] == "solves/s"
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["cores"] >= 1
    assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["e2e"]["d2h_bytes_per_step"] == 0
    # complete solves only: the timed steps add up to the reported time
    assert rec["steps"] == 2 and len(rec["solve_stats"]["seconds"]) == 2
    assert abs(sum(rec["solve_stats"]["seconds"]) * 1e3 - rec["ms_per_step"] * rec["steps"]) <= 1.0
    assert rec["value"] == __import__("pytest").approx(rec["steps"] / sum(rec["solve_stats"]["seconds"]), rel=1e-2)
    assert "priced" not in json.dumps(rec) and "lower bound" not in json.dumps(rec)
