"""torch.autograd.Function over the soft-GMM kernels (argument marshalling only).

The forward and the hand-written adjoint both run in libfos.so
(fos_softgmm_forward / fos_softgmm_backward); this module only passes
pointers and turns the four gradient numbers into a tensor.
"""
from __future__ import annotations

import ctypes

import torch

from . import fos


def default_params(**overrides) -> fos.SoftParams:
    p = fos.SoftParams()
    fos.load().fos_softgmm_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


class SoftGMM:
    """Workspace for B sequences of T frames of W x H (checkpoints live here).
    fp64=1 (a params field) runs the recurrence and the adjoint in double."""

    def __init__(self, width: int, height: int, batch: int, frames: int, params=None, **overrides):
        self.lib = fos.load()
        self.params = params if params is not None else default_params(**overrides)
        h = self.lib.fos_softgmm_create(width, height, batch, frames, ctypes.byref(self.params))
        if not h:
            raise fos.FosError(1, self.lib.fos_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.fos_softgmm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            raise fos.FosError(st, self.lib.fos_softgmm_last_error(self.h).decode())

    def set_theta(self, theta) -> None:
        """theta = (alpha, lambda^2, w_depth, v_init_rgb); kept in double (the
        FP32 kernels round it to float, the FP64 ones use it as given)."""
        arr = (ctypes.c_double * 4)(*[float(v) for v in theta])
        self._check(self.lib.fos_softgmm_set_theta64(self.h, arr))

    def forward(self, rgb, depth, gt, stream=None) -> float:
        out = ctypes.c_double()
        self._check(self.lib.fos_softgmm_forward(self.h, rgb.data_ptr(), depth.data_ptr(), gt.data_ptr(),
                                                 ctypes.byref(out), fos._stream_handle(stream)))
        return out.value

    def backward(self, rgb, depth, gt, pixel_grad=None, stream=None):
        out = (ctypes.c_double * 4)()
        self._check(self.lib.fos_softgmm_backward(
            self.h, rgb.data_ptr(), depth.data_ptr(), gt.data_ptr(), out,
            pixel_grad.data_ptr() if pixel_grad is not None else None, fos._stream_handle(stream)))
        return [out[i] for i in range(4)]


class SoftGMMLoss(torch.autograd.Function):
    """loss = SoftGMMLoss.apply(theta, workspace, rgb, depth, gt).

    theta: float64 tensor (alpha, lambda^2, w_depth, v_init_rgb); the data are
    CUDA tensors of the workspace's shape.  backward() runs the adjoint kernel.
    """

    @staticmethod
    def forward(ctx, theta, ws: SoftGMM, rgb, depth, gt):
        ws.set_theta(theta.detach().cpu().tolist())
        loss = ws.forward(rgb, depth, gt)
        ctx.ws, ctx.data = ws, (rgb, depth, gt)
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gout):
        g = ctx.ws.backward(*ctx.data)
        return gout * torch.tensor(g, dtype=torch.float64), None, None, None, None
