"""bench.py prints one JSON line with the keys its contract names; run on
the 4^4 preset so that it takes seconds."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                         capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_default_line_keys():
    d = _run("--config", "wilson_4x4x4x4", "--steps", "1", "--warmup", "3", "--no-cpu-baseline",
             "--no-mixed", "--no-eo-variant")
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "gpu_launches", "roofline", "clocks", "e2e"):
        assert key in d, key
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["value"] > 0 and d["unit"] == "solves/s" and d["gpu_launches"] > 0
    r = d["roofline"]
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in r, key
    assert r["bound"] == "alu" and 0 < r["frac"] < 1.2
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert d["counts"]["true_rel_res_max"] <= d["config"].get("tol", 1e-10) * 1.0000001


def test_row_lines_run():
    d = _run("--config", "wilson_4x4x4x4", "--even-odd", "--steps", "1", "--warmup", "3")
    assert d["value"] > 0 and d["counts"]["full_system_rel_res_max"] <= 1.05e-10
