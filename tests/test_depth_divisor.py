"""The depth rescale's quotient by the full scale fs (0 stays 0, else
clamp(round-half-up(d * 255 / fs), 1, 255)) is taken on the GPU as a
multiply-shift: with l = ceil(log2 fs), sh = 25 + l and m = ceil(2^sh / fs)
(the round-up multiplier of Granlund and Montgomery, PLDI 1994),
floor(x / fs) = (x * m) >> sh for every x < 2^25.  Checked here, for every
16-bit depth, against integer division over every full scale up to 4096, the
powers of two and their neighbours, and a random sample up to the largest
accepted value (65535 * 4)."""
import numpy as np


def divisor(fs: int):
    l = 0
    while (1 << l) < fs:
        l += 1
    sh = 25 + l
    return ((1 << sh) + fs - 1) // fs, sh


def test_multiply_shift_equals_division_for_every_depth():
    d = np.arange(65536, dtype=np.uint64)
    fss = set(range(1, 4097))
    for k in range(1, 19):
        fss |= {(1 << k) - 1, 1 << k, (1 << k) + 1}
    rng = np.random.default_rng(3)
    fss |= set(int(v) for v in rng.integers(4097, 65535 * 4 + 1, size=1500))
    fss.add(65535 * 4)
    for fs in sorted(f for f in fss if 1 <= f <= 65535 * 4):
        m, sh = divisor(fs)
        assert m < (1 << 32)
        x = d * np.uint64(255) + np.uint64(fs >> 1)
        assert int(x.max()) < (1 << 25)
        q = (x * np.uint64(m)) >> np.uint64(sh)
        np.testing.assert_array_equal(q, x // np.uint64(fs), err_msg=f"fs={fs}")
