"""Failure paths made on the host (no GPU fault is provoked).

Allocation failures are injected with FOS_FAIL_ALLOC_AFTER=n (every device
allocation of the library after the first n fails with
cudaErrorMemoryAllocation): creating a context must then fail cleanly with
FOS_ERR_OOM and a message, for every n short of the total, and the process
must stay usable.  Each case runs in a child process because the hook is
read when the library loads.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, torch
sys.path.insert(0, {root!r})
from paper_2002_00250_gb300 import fos
try:
    seg = fos.Segmenter(64, 48)
    print("CREATED")
    seg.close()
except fos.FosError as e:
    print("FAILED", e.status, str(e))
x = torch.ones(1000, device="cuda")
print("USABLE", float(x.sum()))
"""


def _run(n):
    env = dict(os.environ, FOS_FAIL_ALLOC_AFTER=str(n))
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout


def test_every_allocation_failure_is_reported_cleanly():
    # a 64x48 context with both methods makes 9 device allocations: the GMM
    # planes; samples, D, R, T, S, requests, previous values; counters
    for n in range(0, 9):
        out = _run(n)
        assert "FAILED 3" in out and "cudaErrorMemoryAllocation" in out, (n, out)
        assert "USABLE 1000.0" in out
    out = _run(9)
    assert "CREATED" in out and "USABLE 1000.0" in out
