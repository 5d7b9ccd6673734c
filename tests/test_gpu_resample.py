"""Depth resampled onto the colour grid (Sec. 4.3) through the C ABI.

The resample is integer index arithmetic: bit-exact against the oracle.  A
context created for a lower depth resolution must give exactly what a
same-resolution context gives when fed the oracle's resampled depth.
"""
import numpy as np
import pytest

from _helpers import scene

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("src,dst", [((128, 72), (192, 108)), ((64, 48), (64, 48)), ((67, 45), (130, 91)),
                                     ((13, 7), (200, 3)), ((200, 150), (64, 48)), ((1, 1), (33, 17)),
                                     ((1280, 720), (1920, 1080))])
def test_resample_exact(orc, src, dst):
    import torch
    from paper_2002_00250_gb300 import fos
    (sw, sh), (dw, dh) = src, dst
    d = np.random.default_rng(sw * 7 + dh).integers(0, 65536, (sh, sw)).astype(np.uint16)
    d[::5, ::3] = 0
    got = fos.depth_resample(torch.from_numpy(d).cuda(), dw, dh).cpu().numpy()
    np.testing.assert_array_equal(got, orc.depth_resample(d, dw, dh))


@pytest.mark.parametrize("W,H,Wd,Hd", [(96, 54, 64, 36), (67, 45, 50, 30)])
@pytest.mark.parametrize("kind", ["both", "gmm", "pbas", "gmm_literal"])
def test_mixed_resolution_context_equals_resampled_input(orc, W, H, Wd, Hd, kind):
    """Every kernel path (fused, GMM alone including the all-frames launch,
    PBAS alone, the literal GMM) reads the lower-resolution depth through the
    resampling map: same bits as a same-size context fed resampled depth."""
    import torch
    from paper_2002_00250_gb300 import fos
    kw = {"both": {}, "gmm": dict(methods=fos.METHOD_GMM), "pbas": dict(methods=fos.METHOD_PBAS),
          "gmm_literal": dict(methods=fos.METHOD_GMM, gmm_literal=1)}[kind]
    n = 8
    rgb, _, _ = scene(W, H, n, seed=11)
    _, depth, _ = scene(Wd, Hd, n, seed=12)   # a lower-resolution depth sensor
    up = np.stack([orc.depth_resample(depth[t], W, H) for t in range(n)])
    a = fos.Segmenter(W, H, depth_size=(Wd, Hd), stream_id=3, **kw)
    b = fos.Segmenter(W, H, stream_id=3, **kw)
    ra = a.process_host(rgb, depth)
    rb = b.process_host(rgb, up)
    for x, y in zip(ra, rb):
        if x is not None:
            np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(a.get_state(), b.get_state())
    # device entry point (several frames per call), continuing the same models
    d_rgb = torch.from_numpy(rgb).cuda()
    d_dep = torch.from_numpy(depth).cuda()
    d_up = torch.from_numpy(up).cuda()
    m = [torch.empty((n, H, W), dtype=torch.uint8, device="cuda") for _ in range(4)]
    mg_a, mp_a = (m[0] if a.gmm else None), (m[1] if a.pbas else None)
    mg_b, mp_b = (m[2] if b.gmm else None), (m[3] if b.pbas else None)
    a.process_device(d_rgb, d_dep, mg_a, mp_a)
    b.process_device(d_rgb, d_up, mg_b, mp_b)
    torch.cuda.synchronize()
    if a.gmm:
        assert torch.equal(m[0], m[2])
    if a.pbas:
        assert torch.equal(m[1], m[3])
    np.testing.assert_array_equal(a.get_state(), b.get_state())


def test_bad_sizes_rejected():
    import torch
    from paper_2002_00250_gb300 import fos
    src = torch.zeros((4, 4), dtype=torch.uint16, device="cuda")
    with pytest.raises(fos.FosError):
        fos.depth_resample(src, 0, 4)
    with pytest.raises(fos.FosError):
        fos.Segmenter(64, 48, depth_size=(0, 48))
