"""The leaf-size study script (Sec. V-A, Fig. 4) runs on a tiny sphere: one
line per leaf cap, and where every leaf pair is near (Z_F = 0) the series
equals the LU solution."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_leaf_size_study_runs():
    r = subprocess.run([sys.executable, "-m", "oracle.study_leaf_size", "--level", "2",
                        "--radius", "0.25", "--caps", "16", "1000", "--terms", "2", "3",
                        "--processes", "1"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    rows = [ln.split() for ln in r.stdout.splitlines() if not ln.startswith("#")]
    assert [int(x[0]) for x in rows] == [16, 1000]
    small, one_leaf = rows
    assert int(small[1]) > int(one_leaf[1]) == 1
    # a single leaf: no far field, the series is exact
    assert float(one_leaf[6]) < 1e-10 and float(one_leaf[7]) < 1e-10
