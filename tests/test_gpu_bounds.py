"""The range-checked build (every global and shared index of the GMM, PBAS,
fused, batched, frame-0 and flush kernels checked; a violation is recorded,
never a fault) on the odd frame sizes 1x1, 3x5, 17x13, 67x45, on vector-width
frames, with spatial propagation and forced conflicting draws, other tile
shapes, the all-frames GMM launch and mixed batches: no violation anywhere,
and the checked build still matches the oracle.  Its own check is exercised
first with a declared extent below the index (recorded, access redirected).
Runs in a child process so that the range-checked library is the one loaded."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu


def test_range_checked_build_has_no_violations():
    here = os.path.dirname(os.path.abspath(__file__))
    r = subprocess.run([sys.executable, os.path.join(here, "_bounds_child.py")], capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["selftest"] == [1, 99, 12]
    assert len(out["runs"]) >= 25
    for run in out["runs"]:
        assert run["violations"] == 0, run
        assert run["oracle_equal"], run
