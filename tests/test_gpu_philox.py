"""Pins the oracle's Philox4x32-10 against cuRAND's device implementation."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_philox(tmp_path_factory):
    from paper_2002_00250_gb300.build import ARCH, nvcc
    so = str(tmp_path_factory.mktemp("curand") / "curand_philox.so")
    subprocess.run([nvcc(), "-shared", "-Xcompiler", "-fPIC", *ARCH, "-o", so,
                    os.path.join(HERE, "gpu_helpers", "curand_philox.cu")], check=True)
    lib = ctypes.CDLL(so)
    lib.curand_philox_many.argtypes = [ctypes.c_int] + [ctypes.c_void_p] * 3
    return lib


def test_oracle_philox_equals_curand(orc, curand_philox):
    n = 1 << 20
    rng = np.random.default_rng(9)
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[: n // 2, 1:] = 0  # the counters the segmentation uses: (pixel, frame, channel, 0)
    ctr[: n // 2, 0] = np.arange(n // 2)
    key = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    out = np.empty_like(ctr)
    assert curand_philox.curand_philox_many(n, ctr.ctypes.data, key.ctypes.data, out.ctypes.data) == 0
    np.testing.assert_array_equal(orc.philox4x32_10(ctr, key), out)
