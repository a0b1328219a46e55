"""The device timeline of the measurement build (OPAL_TIMELINE), run as the
command line uses it, in a process of its own (the build loaded is chosen
when the library is first loaded)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_timeline_build_reports_the_step_kernels_in_order():
    r = subprocess.run([sys.executable, "-m", "paper_2601_19654_gb300.run", "--workload", "planetesimals",
                        "--steps", "2", "--timeline", "3"], cwd=ROOT, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = r.stdout.splitlines()
    start = [k for k, line in enumerate(lines) if "device timeline" in line]
    assert start, r.stdout
    rows = {}
    for line in lines[start[0] + 1:]:
        f = line.split()
        if len(f) >= 3:
            rows[f[0]] = (float(f[1]), float(f[2]))
    for name in ("k_step_reset", "k_open", "k_scan_tiles", "k_kick", "k_close", "k_finish"):
        assert name in rows, (name, r.stdout)
    for name, (a, b) in rows.items():
        assert 0.0 <= a <= b, (name, a, b)
    # the step's serial chain: reset, open, the scan, then after the encounters the close and the undo check
    assert rows["k_step_reset"][0] == 0.0
    assert rows["k_open"][0] >= rows["k_step_reset"][1]
    assert rows["k_scan_tiles"][0] >= rows["k_open"][1]
    assert rows["k_close"][0] >= rows["k_kick"][1]
    assert rows["k_finish"][0] >= rows["k_close"][1]
