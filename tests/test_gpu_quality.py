"""Quality indicators of Sec. 5 through the C ABI against the oracle.

Counts are integers: the GPU must match the oracle exactly, for any length
(vector body and byte tail), any alignment of the two arrays and any byte
values (non-zero is foreground).  The derived ratios are host arithmetic in
the library, checked against the oracle's on the hand-counted example.
"""
import numpy as np
import pytest

from _helpers import scene


def test_metrics_from_counts_match_oracle(orc):
    from paper_2002_00250_gb300 import fos
    mask = np.array([255, 255, 0, 0, 255, 0, 0, 0, 7, 0], np.uint8)
    gt = np.array([255, 0, 255, 0, 255, 0, 0, 9, 0, 0], np.uint8)
    want = orc.quality(mask, gt)
    got = fos.quality([want["TP"], want["TN"], want["FP"], want["FN"]])
    for k in ("PWC", "FNR", "FPR", "Si"):
        assert got[k] == pytest.approx(want[k], rel=1e-15), k


@pytest.mark.gpu
@pytest.mark.parametrize("n,off_m,off_g", [(0, 0, 0), (1, 0, 0), (15, 0, 0), (16, 0, 0), (17, 3, 3),
                                           (1000, 0, 0), (4097, 5, 11), (1 << 20, 0, 0),
                                           ((1 << 20) + 13, 0, 0), ((1 << 20) + 13, 1, 0)])
def test_counts_exact(orc, n, off_m, off_g):
    import torch
    from paper_2002_00250_gb300 import fos
    rng = np.random.default_rng(n + 7 * off_m + off_g)
    m = (rng.random(n) < 0.3).astype(np.uint8) * rng.integers(1, 256, n).astype(np.uint8)
    g = (rng.random(n) < 0.4).astype(np.uint8) * 255
    bm = torch.zeros(n + 32, dtype=torch.uint8, device="cuda")
    bg = torch.zeros(n + 32, dtype=torch.uint8, device="cuda")
    dm, dg = bm[off_m:off_m + n], bg[off_g:off_g + n]
    dm.copy_(torch.from_numpy(m))
    dg.copy_(torch.from_numpy(g))
    c = fos.quality_counts(dm, dg).cpu().numpy().tolist()
    if n == 0:
        assert c == [0, 0, 0, 0]
        return
    want = orc.quality(m, g)
    assert c == [want["TP"], want["TN"], want["FP"], want["FN"]]
    assert sum(c) == n


@pytest.mark.gpu
def test_counts_accumulate_over_frames_of_a_run(orc):
    """Masks of a real GMM+PBAS run against the synthetic ground truth, frame
    by frame into one running total."""
    import torch
    from paper_2002_00250_gb300 import fos
    W, H, n = 96, 64, 12
    rgb, depth, gt = scene(W, H, n, seed=3)
    seg = fos.Segmenter(W, H)
    mg, mp = seg.process_host(rgb, depth)
    dgt = torch.from_numpy(gt).cuda()
    for masks in (mg, mp):
        dm = torch.from_numpy(masks).cuda()
        counts = None
        for t in range(n):
            counts = fos.quality_counts(dm[t], dgt[t], counts)
        got = counts.cpu().numpy().tolist()
        want = orc.quality(masks, gt)
        assert got == [want["TP"], want["TN"], want["FP"], want["FN"]]
        q = fos.quality(got)
        assert q["Si"] == pytest.approx(want["Si"], rel=1e-15)
