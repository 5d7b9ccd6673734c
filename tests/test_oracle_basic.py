"""Pins for the oracle's building blocks: Philox, depth rescale, gradient, quality.

Each check compares the oracle with something other than itself: published
known-answer vectors, hand-computed values, a library routine (scipy), or a
property the definition fixes.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = orc.philox4x32_10([ctr], [key])[0]
        assert [int(x) for x in got] == want


def test_philox_counter_sensitivity(orc):
    # Distinct counters give distinct blocks; bits are balanced (a dropped round
    # or a swapped lane would not pass the known answers above either).
    n = 4096
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n)
    out = orc.philox4x32_10(ctr, [[7, 11]])
    assert len({tuple(r) for r in out.tolist()}) == n
    bits = np.unpackbits(out.view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.01


@pytest.mark.parametrize("d,want", [(0, 0), (1, 1), (39, 1), (59, 2), (2000, 51), (2100, 54),
                                    (5000, 128), (9999, 255), (10000, 255), (65535, 255)])
def test_depth_rescale_hand_values(orc, d, want):
    # Sec. 4.2: 0..10 m onto 8 bits; 0 stays invalid; values are worked by hand:
    # e.g. 5000 mm -> (5000*255 + 5000) // 10000 = 128.
    assert int(orc.depth_to_u8(np.array([d], np.uint16))[0]) == want


def test_depth_rescale_step_is_about_4cm(orc):
    # Sec. 4.2 states about 4 cm per level over the 10 m range.
    d = np.arange(1, 10001, dtype=np.uint16)
    q = orc.depth_to_u8(d).astype(int)
    assert q.min() == 1 and q.max() == 255
    assert np.all(np.diff(q) >= 0)
    runs = np.diff(np.flatnonzero(np.diff(q)))
    assert runs.min() >= 39 and runs.max() <= 40


def test_sobel_matches_scipy(orc):
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(3)
    for H, W in [(1, 1), (1, 7), (5, 1), (3, 3), (17, 13), (32, 45)]:
        img = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
        gx = ndimage.sobel(img.astype(np.int32), axis=1, mode="nearest")
        gy = ndimage.sobel(img.astype(np.int32), axis=0, mode="nearest")
        want = np.minimum(255, (np.abs(gx) + np.abs(gy)) >> 3).astype(np.uint8)
        np.testing.assert_array_equal(orc.sobel_grad_u8(img), want)


def test_sobel_hand_edge(orc):
    # columns 0,0,80: |gx| = 4*80 = 320 at x=1 and x=2 (edge-clamped), >>3 = 40.
    img = np.array([[0, 0, 80]] * 3, np.uint8)
    np.testing.assert_array_equal(orc.sobel_grad_u8(img), np.array([[0, 40, 40]] * 3, np.uint8))


def test_quality_hand_counts(orc):
    # Sec. 5 indicators on a worked example: TP=2, TN=3, FP=1, FN=2.
    mask = np.array([255, 255, 0, 0, 0, 255, 0, 0], np.uint8)
    gt = np.array([255, 255, 0, 0, 0, 0, 255, 255], np.uint8)
    q = orc.quality(mask, gt)
    assert (q["TP"], q["TN"], q["FP"], q["FN"]) == (2, 3, 1, 2)
    assert q["PWC"] == pytest.approx(100 * 3 / 8)
    assert q["FNR"] == pytest.approx(2 / 4)
    assert q["FPR"] == pytest.approx(1 / 4)
    assert q["Si"] == pytest.approx(2 / 5)


# ---- depth resampled to the colour grid (Sec. 4.3; nearest, floor mapping) ----

def test_depth_resample_identity(orc):
    d = np.random.default_rng(0).integers(0, 65536, (7, 11)).astype(np.uint16)
    np.testing.assert_array_equal(orc.depth_resample(d, 11, 7), d)


def test_depth_resample_integer_factor_replicates(orc):
    d = np.random.default_rng(1).integers(0, 65536, (5, 6)).astype(np.uint16)
    up = orc.depth_resample(d, 12, 15)   # x2 across, x3 down
    np.testing.assert_array_equal(up, np.repeat(np.repeat(d, 3, axis=0), 2, axis=1))


def test_depth_resample_three_halves_by_hand(orc):
    # 2x2 depth onto a 3x3 colour grid (the 1280x720 -> 1920x1080 ratio):
    # source index = floor(dst * 2 / 3): 0 -> 0, 1 -> 0, 2 -> 1
    d = np.array([[10, 20], [30, 0]], np.uint16)
    want = np.array([[10, 10, 20], [10, 10, 20], [30, 30, 0]], np.uint16)
    np.testing.assert_array_equal(orc.depth_resample(d, 3, 3), want)


def test_depth_resample_keeps_values_and_holes(orc):
    rng = np.random.default_rng(2)
    d = rng.integers(1, 65536, (72, 128)).astype(np.uint16)
    d[rng.random(d.shape) < 0.1] = 0
    up = orc.depth_resample(d, 192, 108)
    assert set(np.unique(up)) <= set(np.unique(d))       # no new values
    assert (up == 0).mean() == pytest.approx((d == 0).mean(), abs=0.02)
    down = orc.depth_resample(d, 64, 36)                  # downscale picks even rows/cols
    np.testing.assert_array_equal(down, d[::2, ::2])
