"""The oracle's build: OpenMP is used whenever the compiler has it, so the
CPU baseline's reported thread count is the count its loops ran on (a loop
form OpenMP rejects would otherwise drop the whole oracle to one thread)."""
import os
import subprocess
import tempfile

import pytest


def _gcc_has_openmp() -> bool:
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        with open(src, "w") as f:
            f.write("#include <omp.h>\nint main(void){return omp_get_max_threads() > 0 ? 0 : 1;}\n")
        r = subprocess.run(["gcc", "-fopenmp", src, "-o", os.path.join(d, "t")], capture_output=True)
        return r.returncode == 0


def test_openmp_used_when_available(orc):
    if not _gcc_has_openmp():
        pytest.skip("gcc without OpenMP here")
    assert orc.openmp()
    assert orc.threads_used(3) == 3
    assert orc.threads_used(0) >= 1


def test_thread_count_does_not_change_results(orc):
    import numpy as np
    from _helpers import scene
    rgb, depth, _ = scene(33, 21, 6, seed=4)
    outs = []
    for n in (1, 4):
        g, p = orc.GMM(33, 21, nthreads=n), orc.PBAS(33, 21, nthreads=n)
        masks = [(g.step(rgb[t], depth[t]), p.step(rgb[t], depth[t])) for t in range(6)]
        outs.append((masks, g.w_rgb.copy(), p.sv.copy(), p.R.copy()))
    for a, b in zip(outs[0][0], outs[1][0]):
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])
    for a, b in zip(outs[0][1:], outs[1][1:]):
        np.testing.assert_array_equal(a, b)
