"""Thin ctypes binding of the C ABI in include/fos.h (argument marshalling only).

Every step of the segmentation runs in the CUDA library ``libfos.so``; this
module converts numpy arrays / torch tensors to pointers and back.  There is
no CPU fallback: if the library cannot be loaded, importing the binding
raises.  Device tensors are torch CUDA tensors; streams are torch streams.
"""
from __future__ import annotations

import ctypes
import time
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfos.so")
BOUNDS_LIB_PATH = os.path.join(_PKG, "libfos_bounds.so")  # range-checked build (build.build(bounds=True))

METHOD_GMM = 1
METHOD_PBAS = 2
KERNEL_GMM, KERNEL_PBAS_CLASSIFY, KERNEL_PBAS_FLUSH, KERNEL_INIT, KERNEL_FUSED, KERNEL_FUSED_SEQUENCE = \
    0, 1, 2, 3, 4, 5
KERNEL_NAMES = ("gmm_step", "pbas_classify", "pbas_flush", "init", "fused_classify", "fused_sequence")
STATUS = {0: "FOS_OK", 1: "FOS_ERR_INVALID_ARG", 2: "FOS_ERR_CUDA", 3: "FOS_ERR_OOM",
          4: "FOS_ERR_TIMEOUT", 5: "FOS_ERR_BUDGET", 6: "FOS_ERR_STATE", 7: "FOS_ERR_UNSUPPORTED",
          8: "FOS_ERR_BUSY"}


class FosError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    """Mirror of fos_params (include/fos.h)."""
    _fields_ = [("methods", ctypes.c_uint32),
                ("K_rgb", ctypes.c_int32), ("K_d", ctypes.c_int32),
                ("alpha", ctypes.c_float), ("lambda_", ctypes.c_float),
                ("w_depth", ctypes.c_float), ("T_bg", ctypes.c_float),
                ("v_init_rgb", ctypes.c_float), ("v_init_d", ctypes.c_float),
                ("v_min_rgb", ctypes.c_float), ("v_min_d", ctypes.c_float),
                ("N", ctypes.c_int32), ("n_min", ctypes.c_int32),
                ("R_lower_rgb", ctypes.c_float), ("R_lower_d", ctypes.c_float),
                ("R_scale", ctypes.c_float), ("R_incdec", ctypes.c_float),
                ("T_lower", ctypes.c_float), ("T_upper", ctypes.c_float),
                ("T_inc", ctypes.c_float), ("T_dec", ctypes.c_float),
                ("alpha_g", ctypes.c_float), ("eps_d", ctypes.c_float),
                ("seed", ctypes.c_uint32), ("stream_id", ctypes.c_uint32),
                ("forced_rng", ctypes.c_int32), ("depth_full_scale_mm", ctypes.c_uint32),
                ("gmm_literal", ctypes.c_int32), ("density_scale", ctypes.c_float),
                ("density_threshold", ctypes.c_float), ("pbas_propagate", ctypes.c_int32),
                ("pbas_joint", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class StateHeader(ctypes.Structure):
    _fields_ = [("magic", ctypes.c_uint32), ("abi_version", ctypes.c_uint32),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("methods", ctypes.c_uint32), ("K_rgb", ctypes.c_int32),
                ("K_d", ctypes.c_int32), ("N", ctypes.c_int32),
                ("frame_index", ctypes.c_int64), ("gmm_bytes", ctypes.c_uint64),
                ("pbas_bytes", ctypes.c_uint64)]


class BatchTuning(ctypes.Structure):
    _fields_ = [("gmm_px", ctypes.c_int32), ("pbas_px", ctypes.c_int32),
                ("pbas_ty", ctypes.c_int32), ("ms_per_step", ctypes.c_float)]


class SoftParams(ctypes.Structure):
    """Mirror of fos_softgmm_params."""
    _fields_ = [("alpha", ctypes.c_float), ("lambda2", ctypes.c_float),
                ("w_depth", ctypes.c_float), ("v_init_rgb", ctypes.c_float),
                ("tau", ctypes.c_float), ("T_bg", ctypes.c_float),
                ("v_min_rgb", ctypes.c_float), ("v_min_d", ctypes.c_float),
                ("v_init_d_ratio", ctypes.c_float), ("K_rgb", ctypes.c_int32),
                ("K_d", ctypes.c_int32), ("ckpt_every", ctypes.c_int32),
                ("depth_full_scale_mm", ctypes.c_uint32), ("fp64", ctypes.c_int32)]


class ServerResult(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_int32), ("status", ctypes.c_int32), ("tag", ctypes.c_int64),
                ("latency_us", ctypes.c_double), ("queue_us", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("ticks", ctypes.c_int64), ("frames_done", ctypes.c_int64),
                ("device_bytes_used", ctypes.c_size_t), ("streams_active", ctypes.c_int32),
                ("streams_waiting", ctypes.c_int32), ("busy_us", ctypes.c_double),
                ("housekeeping_us", ctypes.c_double), ("kernel_us", ctypes.c_double)]


class KernelTiming(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("total_ms", ctypes.c_double), ("frames", ctypes.c_int64)]


# Every exported function and its ctypes signature (checked against the header
# by the tests).
_vp, _i32, _i64, _u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
_st = ctypes.c_int
SIGNATURES = {
    "fos_default_params": (None, [ctypes.POINTER(Params)]),
    "fos_abi_version": (_i32, []),
    "fos_create": (_vp, [_i32, _i32, ctypes.POINTER(Params)]),
    "fos_create_rgbd": (_vp, [_i32, _i32, _i32, _i32, ctypes.POINTER(Params)]),
    "fos_depth_resample_device": (_st, [_vp, _i32, _i32, _vp, _i32, _i32, _vp]),
    "fos_destroy": (None, [_vp]),
    "fos_last_error": (ctypes.c_char_p, [_vp]),
    "fos_last_status": (_st, [_vp]),
    "fos_reset": (_st, [_vp]),
    "fos_frame_index": (_i64, [_vp]),
    "fos_process_frame": (_st, [_vp, _vp, _vp, _vp]),
    "fos_process_frame2": (_st, [_vp, _vp, _vp, _vp, _vp]),
    "fos_process_frame_device": (_st, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "fos_process_frames_device": (_st, [_vp, _i32, _vp, _vp, _vp, _vp, _vp]),
    "fos_process_frames_host": (_st, [_vp, _i32, _vp, _vp, _vp, _vp]),
    "fos_state_size": (_st, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "fos_get_state": (_st, [_vp, _vp, ctypes.c_size_t]),
    "fos_set_state": (_st, [_vp, _vp, ctypes.c_size_t]),
    "fos_set_timing": (_st, [_vp, _u32]),
    "fos_get_timing": (_st, [_vp, ctypes.POINTER(KernelTiming)]),
    "fos_get_counters": (_st, [_vp, ctypes.POINTER(ctypes.c_uint64)]),
    "fos_set_option": (_st, [_vp, _i32, _i32]),
    "fos_get_option": (_i32, [_vp, _i32]),
    "fos_quality_counts_device": (_st, [_vp, _vp, _i64, _vp, _vp]),
    "fos_quality_metrics": (None, [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double)]),
    "fos_pbas_step_noalloc": (_st, [_i32, _i32, ctypes.POINTER(Params), _i64, _vp, _vp, _vp, _vp, _vp]),
    "fos_bounds_checked": (_i32, []),
    "fos_bounds_status": (_st, [_vp, ctypes.POINTER(_u32), ctypes.POINTER(_u32), ctypes.POINTER(_i64)]),
    "fos_bounds_selftest": (_st, [ctypes.POINTER(_u32), ctypes.POINTER(_u32), ctypes.POINTER(_i64)]),
    "fos_stream_device_bytes": (ctypes.c_size_t, [_i32, _i32, ctypes.POINTER(Params)]),
    "fos_batch_create": (_vp, [_i32, ctypes.POINTER(Params)]),
    "fos_batch_destroy": (None, [_vp]),
    "fos_batch_last_error": (ctypes.c_char_p, [_vp]),
    "fos_batch_add_stream": (_i32, [_vp, _i32, _i32, _u32]),
    "fos_batch_remove_stream": (_st, [_vp, _i32]),
    "fos_batch_stream": (_vp, [_vp, _i32]),
    "fos_batch_process_device": (_st, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "fos_batch_process_frames_device": (_st, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "fos_batch_sequence_status": (_st, [_vp]),
    "fos_batch_set_shape": (_st, [_vp, _i32, _i32, _i32]),
    "fos_batch_autotune": (_st, [_vp, _i32, _vp, _vp, _vp, _vp, ctypes.POINTER(BatchTuning)]),
    "fos_server_stream_bytes": (ctypes.c_size_t, [_i32, _i32, ctypes.POINTER(Params)]),
    "fos_server_create": (_vp, [ctypes.POINTER(Params), ctypes.c_size_t, _i32, _i32]),
    "fos_server_destroy": (None, [_vp]),
    "fos_server_last_error": (ctypes.c_char_p, [_vp]),
    "fos_server_open_stream": (_i32, [_vp, _i32, _i32, _u32]),
    "fos_server_close_stream": (_st, [_vp, _i32]),
    "fos_server_submit": (_st, [_vp, _i32, _vp, _vp, _vp, _vp, _i64]),
    "fos_server_submit_nocopy": (_st, [_vp, _i32, _vp, _vp, _vp, _vp, _i64]),
    "fos_server_poll": (_i32, [_vp, ctypes.POINTER(ServerResult), _i32]),
    "fos_server_stats": (_st, [_vp, ctypes.POINTER(ServerStats)]),
    "fos_softgmm_default_params": (None, [ctypes.POINTER(SoftParams)]),
    "fos_softgmm_create": (_vp, [_i32, _i32, _i32, _i32, ctypes.POINTER(SoftParams)]),
    "fos_softgmm_destroy": (None, [_vp]),
    "fos_softgmm_last_error": (ctypes.c_char_p, [_vp]),
    "fos_softgmm_set_theta": (_st, [_vp, ctypes.POINTER(ctypes.c_float)]),
    "fos_softgmm_set_theta64": (_st, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "fos_softgmm_forward": (_st, [_vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_double), _vp]),
    "fos_softgmm_backward": (_st, [_vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_double), _vp, _vp]),
}
OPT_GMM_PX, OPT_GMM_TPB, OPT_PBAS_PX, OPT_PBAS_TY, OPT_FUSE, OPT_TEMPORAL, OPT_SEQUENCE = 1, 2, 3, 4, 5, 6, 7
OPT_GMM_STREAM = 8

_lib = None


def load(path: str = LIB_PATH):
    """Load libfos.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def params_from_dict(d: dict) -> Params:
    """Defaults overridden by the fields present in `d` (field names of
    fos_params; "lambda" is accepted for lambda_); unknown keys raise."""
    names = {f for f, _ in Params._fields_}
    over = {}
    for k, v in d.items():
        k2 = "lambda_" if k == "lambda" else k
        if k2 not in names:
            raise KeyError(f"unknown parameter {k!r}")
        over[k2] = v
    return default_params(**over)


def params_from_json(path_or_text: str) -> Params:
    """Parameters from a JSON object (a file path or the JSON text itself)."""
    import json
    text = path_or_text
    if not path_or_text.lstrip().startswith("{"):
        with open(path_or_text) as f:
            text = f.read()
    return params_from_dict(json.loads(text))


def params_to_json(p: Params) -> str:
    import json
    return json.dumps(p.as_dict(), sort_keys=True)


def default_params(**overrides) -> Params:
    p = Params()
    load().fos_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        key = "lambda_" if k == "lambda" else k
        if not hasattr(p, key):
            raise KeyError(k)
        setattr(p, key, v)
    return p


def _ptr(x) -> int | None:
    """Raw address of a numpy array or torch tensor (None passes NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    assert x.is_contiguous()
    return x.data_ptr()


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


@dataclass
class StateView:
    """Decoded state blob (numpy views into the host copy)."""
    header: StateHeader
    gmm: dict | None
    pbas: dict | None


class Segmenter:
    """One camera stream: owns a fos_ctx (device-resident GMM and/or PBAS model)."""

    def __init__(self, width: int, height: int, params: Params | None = None, depth_size=None,
                 **overrides):
        """depth_size=(depth_width, depth_height): depth frames of another
        resolution, resampled onto the colour grid (fos_create_rgbd)."""
        self.lib = load()
        self.params = params if params is not None else default_params(**overrides)
        if params is not None and overrides:
            for k, v in overrides.items():
                setattr(self.params, "lambda_" if k == "lambda" else k, v)
        self.W, self.H, self.P = width, height, width * height
        self.Wd, self.Hd = depth_size if depth_size is not None else (width, height)
        self.Pd = self.Wd * self.Hd
        h = self.lib.fos_create_rgbd(width, height, self.Wd, self.Hd, ctypes.byref(self.params))
        if not h:
            raise FosError(self.lib.fos_last_status(None) or 1, self.lib.fos_last_error(None).decode())
        self.h = h

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            self.lib.fos_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st: int):
        if st != 0:
            raise FosError(st, self.lib.fos_last_error(self.h).decode())

    @property
    def gmm(self) -> bool:
        return bool(self.params.methods & METHOD_GMM)

    @property
    def pbas(self) -> bool:
        return bool(self.params.methods & METHOD_PBAS)

    def reset(self):
        self._check(self.lib.fos_reset(self.h))

    @property
    def frame_index(self) -> int:
        return int(self.lib.fos_frame_index(self.h))

    # -- host frames ---------------------------------------------------------
    def process_host(self, rgb: np.ndarray, depth: np.ndarray):
        """Frames from host memory ((n,H,W,3) u8 and (n,H,W) u16, or one frame).
        Returns (mask_gmm, mask_pbas) numpy arrays (None for a disabled method)."""
        single = rgb.ndim == 3
        rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
        depth = np.ascontiguousarray(depth, dtype=np.uint16)
        n = 1 if single else rgb.shape[0]
        shape = (self.H, self.W) if single else (n, self.H, self.W)
        assert rgb.size == n * self.P * 3 and depth.size == n * self.Pd
        mg = np.empty(shape, np.uint8) if self.gmm else None
        mp = np.empty(shape, np.uint8) if self.pbas else None
        self._check(self.lib.fos_process_frames_host(self.h, n, _ptr(rgb), _ptr(depth),
                                                     _ptr(mg), _ptr(mp)))
        return mg, mp

    def process_frame(self, rgb, depth, mask_out) -> None:
        """fos_process_frame: one host frame, the primary method's mask."""
        self._check(self.lib.fos_process_frame(self.h, _ptr(rgb), _ptr(depth), _ptr(mask_out)))

    # -- device frames -------------------------------------------------------
    def process_device(self, rgb, depth, mask_gmm=None, mask_pbas=None, stream=None):
        """Frames already on the device (torch CUDA tensors), asynchronous.
        rgb (n,H,W,3) or (H,W,3) u8; depth u16 (n,Hd,Wd) or (Hd,Wd); masks u8."""
        n = 1 if rgb.dim() == 3 else rgb.shape[0]
        assert rgb.numel() == n * self.P * 3 and depth.numel() == n * self.Pd
        self._check(self.lib.fos_process_frames_device(
            self.h, n, _ptr(rgb), _ptr(depth), _ptr(mask_gmm), _ptr(mask_pbas),
            _stream_handle(stream)))

    # -- state -----------------------------------------------------------------
    def state_size(self) -> int:
        n = ctypes.c_size_t()
        self._check(self.lib.fos_state_size(self.h, ctypes.byref(n)))
        return n.value

    def get_state(self) -> np.ndarray:
        buf = np.empty(self.state_size(), np.uint8)
        self._check(self.lib.fos_get_state(self.h, _ptr(buf), buf.size))
        return buf

    def set_state(self, blob: np.ndarray) -> None:
        blob = np.ascontiguousarray(blob, dtype=np.uint8)
        self._check(self.lib.fos_set_state(self.h, _ptr(blob), blob.size))

    def decode_state(self, blob: np.ndarray | None = None) -> StateView:
        return decode_state(self.get_state() if blob is None else blob)

    # -- measurement -------------------------------------------------------------
    def set_timing(self, kernel_mask: int) -> None:
        self._check(self.lib.fos_set_timing(self.h, kernel_mask))

    def get_timing(self) -> dict:
        arr = (KernelTiming * len(KERNEL_NAMES))()
        self._check(self.lib.fos_get_timing(self.h, arr))
        """{kernel: (launches, total ms, frames processed)}."""
        return {KERNEL_NAMES[k]: (arr[k].launches, arr[k].total_ms, arr[k].frames) for k in range(len(KERNEL_NAMES))}

    def set_option(self, option: int, value: int) -> None:
        self._check(self.lib.fos_set_option(self.h, option, value))

    def get_option(self, option: int) -> int:
        return int(self.lib.fos_get_option(self.h, option))

    def bounds_status(self):
        """(violations, first site code, first index) of a range-checked build;
        raises FosError in a release build."""
        n, site, idx = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_int64()
        self._check(self.lib.fos_bounds_status(self.h, ctypes.byref(n), ctypes.byref(site), ctypes.byref(idx)))
        return n.value, site.value, idx.value

    def get_counters(self) -> dict:
        arr = (ctypes.c_uint64 * 4)()
        self._check(self.lib.fos_get_counters(self.h, arr))
        return dict(own_updates=arr[0], neighbour_writes=arr[1], requests=arr[2], frames=arr[3])


def decode_state(blob: np.ndarray) -> StateView:
    """Split a fos_get_state blob into named planes (layout: include/fos.h)."""
    hdr = StateHeader.from_buffer_copy(blob[:ctypes.sizeof(StateHeader)].tobytes())
    off = ctypes.sizeof(StateHeader)
    P = hdr.width * hdr.height
    gmm = pbas = None
    if hdr.methods & METHOD_GMM and hdr.gmm_bytes == (7 * hdr.K_rgb + 3 * hdr.K_d) * P * 8:
        # the paper-literal model: doubles, one variance per colour channel
        Kr, Kd = hdr.K_rgb, hdr.K_d
        planes = blob[off:off + hdr.gmm_bytes].view(np.float64).reshape(7 * Kr + 3 * Kd, P)
        off += hdr.gmm_bytes
        gmm = dict(w_rgb=planes[0:Kr].T,
                   mu_rgb=np.stack([planes[(1 + c) * Kr:(2 + c) * Kr].T for c in range(3)], axis=2),
                   v_rgb=np.stack([planes[(4 + c) * Kr:(5 + c) * Kr].T for c in range(3)], axis=2),
                   w_d=planes[7 * Kr:7 * Kr + Kd].T, mu_d=planes[7 * Kr + Kd:7 * Kr + 2 * Kd].T,
                   v_d=planes[7 * Kr + 2 * Kd:].T)
    elif hdr.methods & METHOD_GMM:
        Kr, Kd = hdr.K_rgb, hdr.K_d
        planes = blob[off:off + hdr.gmm_bytes].view(np.float32).reshape(5 * Kr + 3 * Kd, P)
        off += hdr.gmm_bytes
        gmm = dict(w_rgb=planes[0:Kr].T, mu_rgb=np.stack([planes[Kr:2 * Kr].T, planes[2 * Kr:3 * Kr].T,
                                                           planes[3 * Kr:4 * Kr].T], axis=2),
                   v_rgb=planes[4 * Kr:5 * Kr].T, w_d=planes[5 * Kr:5 * Kr + Kd].T,
                   mu_d=planes[5 * Kr + Kd:5 * Kr + 2 * Kd].T, v_d=planes[5 * Kr + 2 * Kd:].T)
    if hdr.methods & METHOD_PBAS:
        N = hdr.N
        s = blob[off:off + 4 * N * P * 2].view(np.uint16).reshape(4, N, P)
        off += 4 * N * P * 2
        D = blob[off:off + 4 * N * P * 2].view(np.uint16).reshape(4, N, P)
        off += 4 * N * P * 2
        R = blob[off:off + 16 * P].view(np.float32).reshape(4, P)
        off += 16 * P
        T = blob[off:off + 16 * P].view(np.float32).reshape(4, P)
        off += 16 * P
        S = blob[off:off + 16 * P].view(np.uint32).reshape(4, P)
        off += 16 * P
        gsum = blob[off:off + 32].view(np.uint64).copy()
        pbas = dict(sv=(s & 0xFF).astype(np.uint8).transpose(2, 0, 1),
                    sg=(s >> 8).astype(np.uint8).transpose(2, 0, 1),
                    sD=D.transpose(2, 0, 1), R=R.T, T=T.T, S=S.T, gsum=gsum)
    return StateView(hdr, gmm, pbas)


class Batch:
    """Many camera streams processed together: one graph replay per frame step."""

    def __init__(self, max_streams: int, params: Params | None = None, **overrides):
        self.lib = load()
        self.params = params if params is not None else default_params(**overrides)
        h = self.lib.fos_batch_create(max_streams, ctypes.byref(self.params))
        if not h:
            raise FosError(1, self.lib.fos_last_error(None).decode())
        self.h = h
        self.sizes = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.fos_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != 0:
            raise FosError(st, self.lib.fos_batch_last_error(self.h).decode())

    def add(self, width: int, height: int, stream_id: int) -> int:
        slot = self.lib.fos_batch_add_stream(self.h, width, height, stream_id)
        if slot < 0:
            raise FosError(5, self.lib.fos_batch_last_error(self.h).decode())
        self.sizes[slot] = (width, height)
        return slot

    def remove(self, slot: int) -> None:
        self._check(self.lib.fos_batch_remove_stream(self.h, slot))
        self.sizes.pop(slot, None)

    def context(self, slot: int) -> int:
        return self.lib.fos_batch_stream(self.h, slot)

    @staticmethod
    def _arr(ptrs):
        return (ctypes.c_void_p * len(ptrs))(*ptrs)

    def process(self, slots, rgb, depth, mask_gmm=None, mask_pbas=None, stream=None):
        """One frame for each listed slot (lists of torch CUDA tensors)."""
        n = len(slots)
        sl = (ctypes.c_int32 * n)(*slots)
        mg = self._arr([_ptr(m) for m in mask_gmm]) if mask_gmm is not None else None
        mp = self._arr([_ptr(m) for m in mask_pbas]) if mask_pbas is not None else None
        self._check(self.lib.fos_batch_process_device(
            self.h, n, sl, self._arr([_ptr(r) for r in rgb]), self._arr([_ptr(d) for d in depth]),
            mg, mp, _stream_handle(stream)))

    def process_frames(self, slots, rgb, depth, mask_gmm=None, mask_pbas=None, stream=None):
        """Several frames for each listed slot: rgb[i] (n_i, H, W, 3), depth[i]
        (n_i, Hd, Wd), masks (n_i, H, W) torch CUDA tensors (n_i may differ)."""
        n = len(slots)
        nf = [int(r.shape[0]) for r in rgb]
        mg = self._arr([_ptr(m) for m in mask_gmm]) if mask_gmm is not None else None
        mp = self._arr([_ptr(m) for m in mask_pbas]) if mask_pbas is not None else None
        self._check(self.lib.fos_batch_process_frames_device(
            self.h, n, (ctypes.c_int32 * n)(*slots), (ctypes.c_int32 * n)(*nf),
            self._arr([_ptr(r) for r in rgb]), self._arr([_ptr(d) for d in depth]), mg, mp,
            _stream_handle(stream)))

    def sequence_status(self) -> None:
        """Raises if a bounded wait of the last multi-frame launch gave up."""
        self._check(self.lib.fos_batch_sequence_status(self.h))

    def set_shape(self, gmm_px: int, pbas_px: int, pbas_ty: int) -> None:
        self._check(self.lib.fos_batch_set_shape(self.h, gmm_px, pbas_px, pbas_ty))

    def autotune(self, slots, rgb, depth, stream=None) -> dict:
        n = len(slots)
        out = BatchTuning()
        self._check(self.lib.fos_batch_autotune(
            self.h, n, (ctypes.c_int32 * n)(*slots), self._arr([_ptr(r) for r in rgb]),
            self._arr([_ptr(d) for d in depth]), _stream_handle(stream), ctypes.byref(out)))
        return dict(gmm_px=out.gmm_px, pbas_px=out.pbas_px, pbas_ty=out.pbas_ty,
                    ms_per_step=out.ms_per_step)

    def get_state(self, slot: int) -> np.ndarray:
        c = self.context(slot)
        n = ctypes.c_size_t()
        st = self.lib.fos_state_size(c, ctypes.byref(n))
        buf = np.empty(n.value, np.uint8)
        st = st or self.lib.fos_get_state(c, _ptr(buf), buf.size)
        if st != 0:
            raise FosError(st, self.lib.fos_last_error(c).decode())
        return buf


class Server:
    """Serving loop: admission by device-memory budget, continuous batching."""

    def __init__(self, hbm_budget_bytes: int, max_streams: int, queue_depth: int = 16,
                 params: Params | None = None, **overrides):
        self.lib = load()
        self.params = params if params is not None else default_params(**overrides)
        h = self.lib.fos_server_create(ctypes.byref(self.params), hbm_budget_bytes, max_streams, queue_depth)
        if not h:
            raise FosError(1, self.lib.fos_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.fos_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def open_stream(self, width: int, height: int, stream_id: int) -> int:
        sid = self.lib.fos_server_open_stream(self.h, width, height, stream_id)
        if sid < 0:
            raise FosError(5, self.lib.fos_server_last_error(self.h).decode())
        return sid

    def close_stream(self, sid: int) -> None:
        st = self.lib.fos_server_close_stream(self.h, sid)
        if st != 0:
            raise FosError(st, "close_stream")

    def submit(self, sid: int, rgb: np.ndarray, depth: np.ndarray, mask_gmm, mask_pbas, tag: int,
               wait: float = 0.0, copy: bool = True) -> bool:
        """True if queued.  False if refused for longer than ``wait`` seconds;
        ``self.refusal`` then says why: "waiting" (stream not admitted yet) or
        "full" (its queue is full).  copy=False: zero-copy submit, the arrays
        must stay unchanged until poll() reports the tag (pinned for DMA)."""
        fn = self.lib.fos_server_submit if copy else self.lib.fos_server_submit_nocopy
        deadline = time.monotonic() + wait
        while True:
            st = fn(self.h, sid, _ptr(rgb), _ptr(depth), _ptr(mask_gmm), _ptr(mask_pbas), tag)
            if st == 0:
                self.refusal = None
                return True
            if st not in (5, 8):
                raise FosError(st, self.lib.fos_server_last_error(self.h).decode())
            self.refusal = "waiting" if st == 5 else "full"
            if time.monotonic() >= deadline:
                return False
            time.sleep(0.0002)

    def poll(self, max_results: int = 256):
        arr = (ServerResult * max_results)()
        n = self.lib.fos_server_poll(self.h, arr, max_results)
        return [(arr[i].stream, arr[i].status, arr[i].tag, arr[i].latency_us, arr[i].queue_us) for i in range(n)]

    def stats(self) -> dict:
        s = ServerStats()
        st = self.lib.fos_server_stats(self.h, ctypes.byref(s))
        d = {f: getattr(s, f) for f, _ in ServerStats._fields_}
        d["ok"] = st == 0
        return d


QUALITY_NAMES = ("TP", "TN", "FP", "FN", "PWC", "FNR", "FPR", "Si")


def quality_counts(mask, gt, counts=None, stream=None):
    """Adds TP, TN, FP, FN of device masks against device ground truth (torch
    uint8 CUDA tensors of the same number of bytes) to `counts` (an int64
    CUDA tensor of 4, created zeroed if None); returns counts (asynchronous)."""
    import torch
    lib = load()
    if counts is None:
        counts = torch.zeros(4, dtype=torch.int64, device=mask.device)  # same bits as uint64 here
    n = mask.numel()
    if gt.numel() != n:
        raise ValueError("mask and ground truth differ in size")
    st = lib.fos_quality_counts_device(_ptr(mask), _ptr(gt), n, _ptr(counts), _stream_handle(stream))
    if st != 0:
        raise FosError(st, lib.fos_last_error(None).decode())
    return counts


def quality(counts) -> dict:
    """TP, TN, FP, FN and PWC, FNR, FPR, Si from four counts (host values)."""
    lib = load()
    c = (ctypes.c_uint64 * 4)(*[int(v) for v in counts])
    out = (ctypes.c_double * 4)()
    lib.fos_quality_metrics(c, out)
    return dict(zip(QUALITY_NAMES, [int(v) for v in counts] + list(out)))


def depth_resample(src, width: int, height: int, out=None, stream=None):
    """Device depth frame (torch uint16 CUDA tensor (h, w)) resampled onto a
    (height, width) grid by fos_depth_resample_device (asynchronous)."""
    import torch
    lib = load()
    sh, sw = src.shape[-2], src.shape[-1]
    if out is None:
        out = torch.empty((height, width), dtype=src.dtype, device=src.device)
    st = lib.fos_depth_resample_device(_ptr(src), sw, sh, _ptr(out), width, height, _stream_handle(stream))
    if st != 0:
        raise FosError(st, lib.fos_last_error(None).decode())
    return out

