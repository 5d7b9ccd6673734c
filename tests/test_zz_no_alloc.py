"""fos_pbas_step_noalloc against the context API, through the C ABI.

The entry point is for callers that cannot allocate device memory while they
process frames (plug-ins whose framework owns all device memory, real-time
capture callbacks that cannot wait on cudaMalloc, code that must leave the
allocator alone).  It must give the same bits as a PBAS context: the same mask
every frame, and a model equal to the context's exported state after the same
frame.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from _helpers import scene

pytestmark = pytest.mark.gpu


def _unblock(blocked, W, H, N):
    """Model-buffer sample / D array [4][H*spr][N][128] -> [4][N][H*W]."""
    spr = (W + 127) // 128
    b = blocked.reshape(4, H, spr, N, 128).transpose(0, 3, 1, 2, 4).reshape(4, N, H, spr * 128)
    return b[..., :W].reshape(4, N, H * W)


def _planes(buf, W, H):
    spr = (W + 127) // 128
    return buf.reshape(4, H, spr * 128)[..., :W].reshape(4, H * W)


@pytest.mark.parametrize("W,H,N,forced", [(200, 48, 20, 0), (67, 45, 20, 0), (136, 40, 8, 0), (136, 40, 20, 3)])
def test_noalloc_matches_context(W, H, N, forced):
    """N = 8 runs the kernels' generic slot count, forced_rng = 3 the draws
    that make neighbour requests collide; after the first call, further calls
    leave the device's free memory unchanged."""
    import torch
    from paper_2002_00250_gb300 import fos

    n = 6
    rgb, depth, _ = scene(W, H, n, seed=21, hole_fraction=0.05)
    params = fos.default_params(methods=fos.METHOD_PBAS, N=N, forced_rng=forced)
    Sp = ((W + 127) // 128) * 128 * H
    model = torch.zeros(16 * N * Sp + 48 * Sp + 96, dtype=torch.uint8, device="cuda")
    d_rgb = torch.from_numpy(rgb).cuda()
    d_dep = torch.from_numpy(depth).cuda()
    mask = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    ref = fos.Segmenter(W, H, params=params)
    ref_mask = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    lib = fos.load()
    stream = torch.cuda.current_stream().cuda_stream
    for t in range(n):
        st = lib.fos_pbas_step_noalloc(W, H, ctypes.byref(params), t, d_rgb[t].data_ptr(),
                                       d_dep[t].data_ptr(), model.data_ptr(), mask.data_ptr(), stream)
        assert st == 0, lib.fos_last_error(None)
        ref.process_device(d_rgb[t], d_dep[t], mask_pbas=ref_mask)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(mask.cpu().numpy(), ref_mask.cpu().numpy(), err_msg=f"frame {t}")
        want = ref.decode_state().pbas
        m = model.cpu().numpy()
        o = 0
        samp = _unblock(m[o:o + 8 * N * Sp].view(np.uint16), W, H, N); o += 8 * N * Sp
        D = _unblock(m[o:o + 8 * N * Sp].view(np.uint16), W, H, N); o += 8 * N * Sp
        R = _planes(m[o:o + 16 * Sp].view(np.float32), W, H); o += 16 * Sp
        T = _planes(m[o:o + 16 * Sp].view(np.float32), W, H); o += 16 * Sp
        S = _planes(m[o:o + 16 * Sp].view(np.uint32), W, H); o += 16 * Sp
        np.testing.assert_array_equal((samp & 0xFF).astype(np.uint8).transpose(2, 0, 1), want["sv"])
        np.testing.assert_array_equal((samp >> 8).astype(np.uint8).transpose(2, 0, 1), want["sg"])
        np.testing.assert_array_equal(D.transpose(2, 0, 1), want["sD"])
        np.testing.assert_array_equal(R.T, want["R"])
        np.testing.assert_array_equal(T.T, want["T"])
        np.testing.assert_array_equal(S.T, want["S"])
    # more frames, nothing else in between: the free device memory must not move
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for t in range(n, n + 4):
        st = lib.fos_pbas_step_noalloc(W, H, ctypes.byref(params), t, d_rgb[t % n].data_ptr(),
                                       d_dep[t % n].data_ptr(), model.data_ptr(), mask.data_ptr(), stream)
        assert st == 0, lib.fos_last_error(None)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_oversized_frames():
    from paper_2002_00250_gb300 import fos
    lib = fos.load()
    params = fos.default_params(methods=fos.METHOD_PBAS)
    # 2048 x 1025 -> 2,099,200 padded pixels > 2,097,152
    st = lib.fos_pbas_step_noalloc(2048, 1025, ctypes.byref(params), 0, 16, 16, 16, 16, None)
    assert st == 1
    assert b"FOS_NOALLOC_MAX_PIXELS" in lib.fos_last_error(None)


def test_noalloc_rejects_bad_model_alignment_and_parameters():
    """Host-side checks only (no kernel is launched): a model buffer off the
    256-byte boundary, and parameters that fos_create refuses for a PBAS
    context, are refused here too."""
    from paper_2002_00250_gb300 import fos
    lib = fos.load()
    params = fos.default_params(methods=fos.METHOD_PBAS)
    st = lib.fos_pbas_step_noalloc(64, 32, ctypes.byref(params), 0, 16, 16, 16 + 1, 16, None)
    assert st == 1 and b"256-byte" in lib.fos_last_error(None)
    for bad in (dict(R_lower_rgb=0.0), dict(R_lower_d=-1.0), dict(R_incdec=1.0), dict(forced_rng=4),
                dict(pbas_propagate=2), dict(depth_full_scale_mm=65535 * 4 + 1)):
        p = fos.default_params(methods=fos.METHOD_PBAS, **bad)
        st = lib.fos_pbas_step_noalloc(64, 32, ctypes.byref(p), 0, 256, 256, 256, 256, None)
        assert st == 1, bad
