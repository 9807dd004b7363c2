"""The single-kernel runner that the ncu summaries under profiles/ are taken
with: every mode runs on a small lattice and reports a finite result."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, "-m", "paper_0710_1988_gb300.kernel_case", *args],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("kernel,extra", [("f64", []), ("f32", []), ("f16", []),
                                          ("f64", ["--even-odd"]), ("f32", ["--even-odd"])])
def test_apply_modes(kernel, extra):
    d = _run("--kernel", kernel, "--lattice", "4", "4", "4", "8", "--nrhs", "3", "--reps", "2",
             *extra)
    assert d["finite"] and d["ms_per_apply"] > 0 and d["even_odd"] == bool(extra)


@pytest.mark.parametrize("extra", [[], ["--storage", "16"], ["--even-odd"]])
def test_mixed_mode(extra):
    d = _run("--kernel", "mixed", "--lattice", "4", "4", "4", "8", "--nrhs", "2", "--reps", "20",
             *extra)
    assert d["iters"] == [20, 20] and d["ms"] > 0


@pytest.mark.parametrize("extra", [[], ["--fp64-eig"]])
def test_gmresdr_cycle_end_mode(extra):
    """The cycle-end timing mode on the 4^4 workload (GMRES-DR(20,6)): both
    eigenvalue paths converge with the same counts."""
    d = _run("--kernel", "gmresdr", "--workload", "wilson_4x4x4x4", *extra)
    assert d["status"] == 0 and d["fp32_estimates"] == (not extra)
    assert d["cycle_end_launches"] == d["cycles"] and d["ms_per_cycle_end"] > 0
