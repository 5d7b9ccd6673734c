"""The host-frame pipeline (fos_process_frames_host): frames staged in chunks
of up to 16 with padded per-frame pitches on three streams must give the same
masks and model as the same frames processed from device memory, for frame
counts that are not a multiple of the chunk, odd frame sizes (pitches padded
to 256 bytes), calls of different lengths one after another (the staging
grows), a lower-resolution depth sensor, and pinned as well as pageable
host buffers.
"""
import numpy as np
import pytest

from _helpers import scene

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("W,H", [(67, 45), (128, 40), (33, 7)])
def test_host_chunks_equal_device(W, H):
    import torch
    from paper_2002_00250_gb300 import fos
    n = 27
    rgb, depth, _ = scene(W, H, n, seed=W)
    a = fos.Segmenter(W, H, stream_id=2)
    b = fos.Segmenter(W, H, stream_id=2)
    # host: 1 frame, then 19 (chunks of 16 and 3: the staging grows), then 7
    got_g, got_p = [], []
    for lo, hi in ((0, 1), (1, 20), (20, 27)):
        mg, mp = a.process_host(rgb[lo:hi], depth[lo:hi])
        got_g.append(mg)
        got_p.append(mp)
    got_g, got_p = np.concatenate(got_g), np.concatenate(got_p)
    d_rgb, d_dep = torch.from_numpy(rgb).cuda(), torch.from_numpy(depth).cuda()
    mg = torch.empty((n, H, W), dtype=torch.uint8, device="cuda")
    mp = torch.empty_like(mg)
    b.process_device(d_rgb, d_dep, mg, mp)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got_g, mg.cpu().numpy())
    np.testing.assert_array_equal(got_p, mp.cpu().numpy())
    np.testing.assert_array_equal(a.get_state(), b.get_state())


def test_host_pinned_buffers_and_rgbd_sizes():
    import torch
    from paper_2002_00250_gb300 import fos
    W, H, Wd, Hd, n = 96, 54, 64, 36, 11
    rgb, _, _ = scene(W, H, n, seed=3)
    _, depth, _ = scene(Wd, Hd, n, seed=4)
    a = fos.Segmenter(W, H, depth_size=(Wd, Hd))
    b = fos.Segmenter(W, H, depth_size=(Wd, Hd))
    h_rgb = torch.from_numpy(rgb).pin_memory()
    h_dep = torch.from_numpy(depth).pin_memory()
    h_mg = torch.empty((n, H, W), dtype=torch.uint8).pin_memory()
    h_mp = torch.empty_like(h_mg).pin_memory()
    lib = fos.load()
    assert lib.fos_process_frames_host(a.h, n, h_rgb.data_ptr(), h_dep.data_ptr(),
                                       h_mg.data_ptr(), h_mp.data_ptr()) == 0
    rg, rp = b.process_host(rgb, depth)  # pageable buffers
    np.testing.assert_array_equal(h_mg.numpy(), rg)
    np.testing.assert_array_equal(h_mp.numpy(), rp)
    np.testing.assert_array_equal(a.get_state(), b.get_state())
