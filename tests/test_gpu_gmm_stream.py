"""The bulk-copy GMM kernel (frames >= 1 of the 3+3 model staged through
shared memory in 256-pixel chunks) against the register kernels and the
FP64 oracle.

Both kernels run the same per-pixel arithmetic, so masks and every state
plane must be bit-identical; the oracle bar is the GMM one (1e-4 relative
parameters, masks equal away from the 1e-5 decision margin).
"""
import numpy as np
import pytest

from _helpers import scene
from test_gpu_gmm import step_parity

pytestmark = pytest.mark.gpu


def _run(W, H, n, stream_opt, offset=0, seed=0):
    import torch
    from paper_2002_00250_gb300 import fos
    rgb, depth, _ = scene(W, H, n, seed=seed, n_objects=3)
    dev = torch.device("cuda", 0)
    # `offset` bytes / elements in front of each frame buffer: 0 keeps the
    # 16-byte alignment the bulk copies need, 1 forces the register kernels
    r = torch.zeros(n * H * W * 3 + 16, dtype=torch.uint8, device=dev)
    d = torch.zeros(n * H * W + 8, dtype=torch.uint16, device=dev)
    m = torch.zeros(n * H * W + 16, dtype=torch.uint8, device=dev)
    r[offset:offset + r.numel() - 16].copy_(torch.from_numpy(rgb.reshape(-1)))
    d[offset:offset + d.numel() - 8].copy_(torch.from_numpy(depth.reshape(-1)))
    rv = r[offset:offset + n * H * W * 3].view(n, H, W, 3)
    dv = d[offset:offset + n * H * W].view(n, H, W)
    mv = m[offset:offset + n * H * W].view(n, H, W)
    seg = fos.Segmenter(W, H, methods=fos.METHOD_GMM, alpha=0.05)
    seg.set_option(fos.OPT_TEMPORAL, 0)  # one launch per frame
    seg.set_option(fos.OPT_GMM_STREAM, stream_opt)
    for t in range(n):
        seg.process_device(rv[t], dv[t], mv[t], None)
    torch.cuda.synchronize()
    out = mv.cpu().numpy().copy(), seg.get_state().copy()
    seg.close()
    return out


@pytest.mark.parametrize("W,H", [(1280, 720), (67, 45), (16, 16), (257, 3), (1, 1)])
def test_stream_kernel_same_bits(W, H):
    # whole chunks only, ragged tails, a frame smaller than one chunk
    m1, s1 = _run(W, H, 5, 1)
    m0, s0 = _run(W, H, 5, 0)
    assert np.array_equal(m1, m0)
    assert np.array_equal(s1, s0)


def test_unaligned_buffers_fall_back():
    m1, s1 = _run(96, 40, 4, 1, offset=1)
    m0, s0 = _run(96, 40, 4, 0)
    assert np.array_equal(m1, m0)
    assert np.array_equal(s1, s0)


def test_stream_kernel_oracle_720p(orc):
    # step parity on the full 1280x720 frame (the oracle reloads the GPU
    # state before every frame); the bulk-copy kernel is the default path
    step_parity(orc, 1280, 720, 4, alpha=0.05, seed=3)
