"""Several frames in one persistent launch (FOS_OPT_SEQUENCE): a tile of frame
t+1 starts as soon as the 3x3 tiles around it have finished frame t.  The
launch must compute exactly the bits of one launch per frame: masks of every
frame and the whole exported model, for ragged sizes (one-pixel and
two-pixel tiles), N other than 20, spatial propagation, the forced draws that
make conflicting neighbour requests, 4-row tiles, depth of another size, the
host API's chunks, and calls that mix sequence and single-frame launches."""
import numpy as np
import pytest
import torch

from _helpers import scene

pytestmark = pytest.mark.gpu


def _run(W, H, n, splits, seq, depth_size=None, options=(), **kw):
    from paper_2002_00250_gb300 import fos
    rgb, depth, _ = scene(W, H, n, seed=W + H + n)
    if depth_size is not None:
        Wd, Hd = depth_size
        depth = np.ascontiguousarray(depth[:, ::H // Hd, ::W // Wd][:, :Hd, :Wd])
    seg = fos.Segmenter(W, H, depth_size=depth_size, **kw)
    for opt, v in options:
        seg.set_option(opt, v)
    seg.set_option(fos.OPT_SEQUENCE, 1 if seq else 0)
    dev = torch.device("cuda", 0)
    r = torch.from_numpy(rgb).to(dev)
    d = torch.from_numpy(depth).to(dev)
    mg = torch.zeros((n, H, W), dtype=torch.uint8, device=dev)
    mp = torch.zeros_like(mg)
    f = 0
    for k in splits:
        seg.process_device(r[f:f + k], d[f:f + k], mg[f:f + k], mp[f:f + k])
        f += k
    assert f == n
    torch.cuda.synchronize()
    state = seg.get_state()
    seg.close()
    return mg.cpu().numpy(), mp.cpu().numpy(), state


CASES = [
    # W, H, frames, calls, extra
    (67, 45, 12, [12], {}),                                  # odd width: 1 px per thread
    (130, 70, 12, [12], {}),                                 # 2 px x 8 rows, ragged tiles
    (130, 70, 10, [10], {"pbas_propagate": 1}),
    (96, 40, 10, [10], {"N": 8}),                            # N other than 20
    (128, 64, 10, [10], {"forced_rng": 2}),                  # conflicting requests
    (128, 64, 10, [10], {"forced_rng": 3, "pbas_propagate": 1}),
    (130, 66, 12, [1, 5, 1, 2, 3], {}),                      # sequence and single-frame calls
    (1280, 720, 16, [16], {}),                               # several waves of tiles per frame
]


@pytest.mark.parametrize("W,H,n,splits,kw", CASES)
def test_sequence_equals_per_frame(W, H, n, splits, kw):
    g0, p0, s0 = _run(W, H, n, splits, seq=False, **kw)
    g1, p1, s1 = _run(W, H, n, splits, seq=True, **kw)
    for f in range(n):
        np.testing.assert_array_equal(g1[f], g0[f], err_msg=f"gmm frame {f}")
        np.testing.assert_array_equal(p1[f], p0[f], err_msg=f"pbas frame {f}")
    assert np.array_equal(s1, s0), "exported model differs"
    assert 0 < int((p0 > 0).sum()) < p0.size


def test_sequence_with_four_row_tiles_and_depth_of_another_size():
    from paper_2002_00250_gb300 import fos
    opts = [(fos.OPT_PBAS_TY, 4)]
    g0, p0, s0 = _run(128, 72, 9, [9], seq=False, depth_size=(64, 36), options=opts)
    g1, p1, s1 = _run(128, 72, 9, [9], seq=True, depth_size=(64, 36), options=opts)
    np.testing.assert_array_equal(g1, g0)
    np.testing.assert_array_equal(p1, p0)
    assert np.array_equal(s1, s0)


def test_host_api_chunks_equal_per_frame():
    # the host API stages 16 frames per chunk: frame 0 alone, then sequence
    # launches of 15 frames and a last single frame
    from paper_2002_00250_gb300 import fos
    W, H, n = 100, 50, 17
    rgb, depth, _ = scene(W, H, n, seed=7)
    out = []
    for seq in (0, 1):
        seg = fos.Segmenter(W, H)
        seg.set_option(fos.OPT_SEQUENCE, seq)
        mg, mp = seg.process_host(rgb, depth)
        out.append((mg, mp, seg.get_state()))
        seg.close()
    np.testing.assert_array_equal(out[1][0], out[0][0])
    np.testing.assert_array_equal(out[1][1], out[0][1])
    assert np.array_equal(out[1][2], out[0][2])


def test_sequence_timing_counts_frames():
    from paper_2002_00250_gb300 import fos
    W, H, n = 128, 64, 9
    rgb, depth, _ = scene(W, H, n, seed=3)
    dev = torch.device("cuda", 0)
    seg = fos.Segmenter(W, H)
    seg.set_timing(1 << fos.KERNEL_FUSED_SEQUENCE)
    r, d = torch.from_numpy(rgb).to(dev), torch.from_numpy(depth).to(dev)
    mg = torch.empty((n, H, W), dtype=torch.uint8, device=dev)
    mp = torch.empty_like(mg)
    seg.process_device(r, d, mg, mp)
    t = seg.get_timing()["fused_sequence"]
    assert t[0] == 1 and t[2] == n - 1 and t[1] > 0
    cnt = seg.get_counters()
    assert cnt["frames"] == n
    seg.close()
