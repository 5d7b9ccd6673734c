"""Plain CPU oracle for the RGB-D GMM and PBAS background models.

TEST INFRASTRUCTURE ONLY.  This package checks the CUDA library; it is not a
fallback for it.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with ``paper_2002_00250_gb300`` and never imports it.

The arithmetic lives in ``fos_oracle.c`` (plain C, GMM in FP64, PBAS in IEEE
FP32 + integers, compiled with ``-ffp-contract=off``); this module builds it
with gcc and wraps it with ctypes over numpy arrays.  Citations are to the
paper (Janus, Kryjak, Gorgon): Sec. 3.1 GMM and Eq. 1, Sec. 3.2 PBAS,
Sec. 4.2 depth rescale, Sec. 5 quality indicators.

Functions whose parity pin is missing say "parity unpinned" in their
docstring (none at present).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libfos_oracle.so")
_SRC = [os.path.join(_HERE, "fos_oracle.c")]
_HDR = [os.path.join(_HERE, "fos_oracle.h")]
_lock = threading.Lock()
_lib = None


def _stale() -> bool:
    if not os.path.exists(_SO):
        return True
    t = os.path.getmtime(_SO)
    return any(os.path.getmtime(s) > t for s in _SRC + _HDR)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available). Returns the .so path."""
    if not force and not _stale():
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", "-Wall", "-o", _SO + ".tmp"] + _SRC + ["-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


class _GmmParams(ctypes.Structure):
    _fields_ = [("K_rgb", ctypes.c_int), ("K_d", ctypes.c_int),
                ("alpha", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("w_depth", ctypes.c_double), ("T_bg", ctypes.c_double),
                ("v_init_rgb", ctypes.c_double), ("v_init_d", ctypes.c_double),
                ("v_min_rgb", ctypes.c_double), ("v_min_d", ctypes.c_double),
                ("depth_full_scale_mm", ctypes.c_uint32)]


class _GmmLiteralParams(ctypes.Structure):
    _fields_ = [("base", _GmmParams), ("s", ctypes.c_double), ("theta", ctypes.c_double)]


class _PbasParams(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("n_min", ctypes.c_int),
                ("R_lower_rgb", ctypes.c_float), ("R_lower_d", ctypes.c_float),
                ("R_scale", ctypes.c_float), ("R_incdec", ctypes.c_float),
                ("T_lower", ctypes.c_float), ("T_upper", ctypes.c_float),
                ("T_inc", ctypes.c_float), ("T_dec", ctypes.c_float),
                ("alpha_g", ctypes.c_float), ("eps_d", ctypes.c_float),
                ("seed", ctypes.c_uint32), ("stream_id", ctypes.c_uint32),
                ("forced_rng", ctypes.c_int), ("depth_full_scale_mm", ctypes.c_uint32),
                ("propagate", ctypes.c_int), ("joint", ctypes.c_int)]


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            so = build()
            L = ctypes.CDLL(so)
            vp, i64, i32, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32
            L.or_philox4x32_10.argtypes = [vp, vp, vp]
            L.or_philox_many.argtypes = [i64, vp, vp, vp]
            L.or_depth_to_u8.argtypes = [i64, vp, u32, vp]
            L.or_sobel_grad_u8.argtypes = [i32, i32, vp, vp]
            L.or_depth_resample.argtypes = [i32, i32, vp, i32, i32, vp]
            L.or_gmm_frame.argtypes = [ctypes.POINTER(_GmmParams), i32, i32, i64, vp, vp,
                                       vp, vp, vp, vp, vp, vp, vp, vp, i32]
            L.or_pbas_frame.argtypes = [ctypes.POINTER(_PbasParams), i32, i32, i64, vp, vp,
                                        vp, vp, vp, vp, vp, vp, vp, vp, i32]
            L.or_quality.argtypes = [i64, vp, vp, vp]
            L.or_openmp.argtypes = []
            L.or_openmp.restype = ctypes.c_int
            L.or_threads.argtypes = [ctypes.c_int]
            L.or_threads.restype = ctypes.c_int
            L.or_gmm_literal_frame.argtypes = [ctypes.POINTER(_GmmLiteralParams), i32, i32, i64, vp, vp,
                                               vp, vp, vp, vp, vp, vp, vp, vp, i32]
            for f in ("or_philox4x32_10", "or_philox_many", "or_depth_to_u8", "or_depth_resample", "or_sobel_grad_u8",
                      "or_gmm_frame", "or_gmm_literal_frame", "or_pbas_frame", "or_quality"):
                getattr(L, f).restype = None
            _lib = L
    return _lib


# ---------------------------------------------------------------------------
# parameter sets (the method's constants; readings listed in the design notes)
# ---------------------------------------------------------------------------
GMM_DEFAULTS = dict(K_rgb=3, K_d=3, alpha=0.001, lambda_=2.5, w_depth=0.5, T_bg=0.7,
                    v_init_rgb=36.0, v_init_d=4.0, v_min_rgb=4.0, v_min_d=0.25,
                    depth_full_scale_mm=10000)
PBAS_DEFAULTS = dict(N=20, n_min=2, R_lower_rgb=18.0, R_lower_d=4.0, R_scale=5.0,
                     R_incdec=0.05, T_lower=2.0, T_upper=200.0, T_inc=1.0, T_dec=0.05,
                     alpha_g=10.0, eps_d=1.0 / 16.0, seed=0, stream_id=0, forced_rng=0,
                     depth_full_scale_mm=10000, propagate=0, joint=0)


def openmp() -> bool:
    """True when the oracle was built with OpenMP (its pixel loops use the
    host's cores); the build falls back to one thread when gcc has none."""
    return bool(lib().or_openmp())


def threads_used(nthreads: int = 0) -> int:
    """Threads the oracle's parallel loops run on for an `nthreads` argument."""
    return int(lib().or_threads(nthreads))


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 (Salmon et al., SC'11) for arrays of counters (n,4) and keys (n,2)."""
    ctr = np.ascontiguousarray(np.atleast_2d(np.asarray(ctr, dtype=np.uint32)))
    key = np.ascontiguousarray(np.atleast_2d(np.asarray(key, dtype=np.uint32)))
    key = np.ascontiguousarray(np.broadcast_to(key, (ctr.shape[0], 2)))
    out = np.empty_like(ctr)
    lib().or_philox_many(ctr.shape[0], _p(ctr), _p(key), _p(out))
    return out


def depth_to_u8(depth, full_scale_mm: int = 10000) -> np.ndarray:
    """Sec. 4.2: depth u16 mm -> u8 (0 = invalid, 1..255 over the full scale)."""
    d = np.ascontiguousarray(depth, dtype=np.uint16)
    out = np.empty(d.shape, dtype=np.uint8)
    lib().or_depth_to_u8(d.size, _p(d), full_scale_mm, _p(out))
    return out


def depth_resample(depth, width: int, height: int) -> np.ndarray:
    """Depth frame (h, w) u16 resampled onto a (height, width) colour grid,
    nearest neighbour with floor mapping (Sec. 4.3)."""
    d = np.ascontiguousarray(depth, dtype=np.uint16)
    sh, sw = d.shape
    out = np.empty((height, width), dtype=np.uint16)
    lib().or_depth_resample(sw, sh, _p(d), width, height, _p(out))
    return out


def sobel_grad_u8(img) -> np.ndarray:
    """PBAS gradient feature: min(255, (|Sobel x| + |Sobel y|) >> 3), edge-clamped."""
    a = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = a.shape
    out = np.empty_like(a)
    lib().or_sobel_grad_u8(W, H, _p(a), _p(out))
    return out


def quality(mask, gt) -> dict:
    """Sec. 5: TP, TN, FP, FN and PWC, FNR, FPR, Si."""
    m = np.ascontiguousarray(mask, dtype=np.uint8).ravel()
    g = np.ascontiguousarray(gt, dtype=np.uint8).ravel()
    out = np.zeros(8, dtype=np.float64)
    lib().or_quality(m.size, _p(m), _p(g), _p(out))
    return dict(zip(("TP", "TN", "FP", "FN", "PWC", "FNR", "FPR", "Si"), out.tolist()))


class GMM:
    """Sec. 3.1 GMM over RGB and depth (two models), FP64.

    State arrays (pixel-major, then component, ranked order):
    ``w_rgb (P,Kr)``, ``mu_rgb (P,Kr,3)``, ``v_rgb (P,Kr)``, ``w_d (P,Kd)``,
    ``mu_d (P,Kd)``, ``v_d (P,Kd)``.  ``t`` counts processed frames.
    """

    def __init__(self, width: int, height: int, nthreads: int = 0, **params):
        pr = dict(GMM_DEFAULTS)
        pr.update(params)
        self.params = pr
        self._c = _GmmParams(**pr)
        self.W, self.H = width, height
        P = width * height
        Kr, Kd = pr["K_rgb"], pr["K_d"]
        self.w_rgb = np.zeros((P, Kr))
        self.mu_rgb = np.zeros((P, Kr, 3))
        self.v_rgb = np.zeros((P, Kr))
        self.w_d = np.zeros((P, Kd))
        self.mu_d = np.zeros((P, Kd))
        self.v_d = np.zeros((P, Kd))
        self.t = 0
        self.nthreads = nthreads

    def step(self, rgb, depth, want_margin: bool = False):
        """Process one frame; returns the mask (H,W) u8, and the margins if asked."""
        rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
        depth = np.ascontiguousarray(depth, dtype=np.uint16)
        assert rgb.shape == (self.H, self.W, 3) and depth.shape == (self.H, self.W)
        mask = np.empty((self.H, self.W), dtype=np.uint8)
        margin = np.empty((self.H, self.W), dtype=np.float64) if want_margin else None
        lib().or_gmm_frame(ctypes.byref(self._c), self.W, self.H, self.t, _p(rgb), _p(depth),
                           _p(self.w_rgb), _p(self.mu_rgb), _p(self.v_rgb),
                           _p(self.w_d), _p(self.mu_d), _p(self.v_d), _p(mask),
                           _p(margin) if margin is not None else None, self.nthreads)
        self.t += 1
        return (mask, margin) if want_margin else mask


GMM_LITERAL_DEFAULTS = dict(GMM_DEFAULTS, K_rgb=7, K_d=3, s=10000.0, theta=1.0)


class GMMLiteral:
    """Sec. 3.1 as printed: K = 7 / 3, FP64, one variance per colour channel,
    decision on the product of the two models' s-scaled Eq. 1 densities
    (full definition with or_gmm_literal_frame in fos_oracle.h).

    State arrays: ``w_rgb (P,Kr)``, ``mu_rgb (P,Kr,3)``, ``v_rgb (P,Kr,3)``,
    ``w_d (P,Kd)``, ``mu_d (P,Kd)``, ``v_d (P,Kd)``.
    """

    def __init__(self, width: int, height: int, nthreads: int = 0, **params):
        pr = dict(GMM_LITERAL_DEFAULTS)
        pr.update(params)
        self.params = pr
        base = {k: v for k, v in pr.items() if k not in ("s", "theta")}
        self._c = _GmmLiteralParams(_GmmParams(**base), pr["s"], pr["theta"])
        self.W, self.H = width, height
        P = width * height
        Kr, Kd = pr["K_rgb"], pr["K_d"]
        self.w_rgb = np.zeros((P, Kr))
        self.mu_rgb = np.zeros((P, Kr, 3))
        self.v_rgb = np.zeros((P, Kr, 3))
        self.w_d = np.zeros((P, Kd))
        self.mu_d = np.zeros((P, Kd))
        self.v_d = np.zeros((P, Kd))
        self.t = 0
        self.nthreads = nthreads

    def step(self, rgb, depth, want_margin: bool = False):
        rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
        depth = np.ascontiguousarray(depth, dtype=np.uint16)
        assert rgb.shape == (self.H, self.W, 3) and depth.shape == (self.H, self.W)
        mask = np.empty((self.H, self.W), dtype=np.uint8)
        margin = np.empty((self.H, self.W), dtype=np.float64) if want_margin else None
        lib().or_gmm_literal_frame(ctypes.byref(self._c), self.W, self.H, self.t, _p(rgb), _p(depth),
                                   _p(self.w_rgb), _p(self.mu_rgb), _p(self.v_rgb),
                                   _p(self.w_d), _p(self.mu_d), _p(self.v_d), _p(mask),
                                   _p(margin) if margin is not None else None, self.nthreads)
        self.t += 1
        return (mask, margin) if want_margin else mask


class PBAS:
    """Sec. 3.2 PBAS with (R, G, B, D) samples, FP32 + integers.

    State arrays: ``sv, sg (P,4,N) u8``, ``sD (P,4,N) u16``, ``R, T (P,4) f32``,
    ``S (P,4) u32``, ``gsum (4,) u64`` (gradient sums of the last frame).
    """

    def __init__(self, width: int, height: int, nthreads: int = 0, **params):
        pr = dict(PBAS_DEFAULTS)
        pr.update(params)
        self.params = pr
        self._c = _PbasParams(**pr)
        self.W, self.H = width, height
        P, N = width * height, pr["N"]
        self.sv = np.zeros((P, 4, N), dtype=np.uint8)
        self.sg = np.zeros((P, 4, N), dtype=np.uint8)
        self.sD = np.zeros((P, 4, N), dtype=np.uint16)
        self.R = np.zeros((P, 4), dtype=np.float32)
        self.T = np.zeros((P, 4), dtype=np.float32)
        self.S = np.zeros((P, 4), dtype=np.uint32)
        self.gsum = np.zeros(4, dtype=np.uint64)
        self.t = 0
        self.nthreads = nthreads

    def step(self, rgb, depth):
        rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
        depth = np.ascontiguousarray(depth, dtype=np.uint16)
        assert rgb.shape == (self.H, self.W, 3) and depth.shape == (self.H, self.W)
        mask = np.empty((self.H, self.W), dtype=np.uint8)
        lib().or_pbas_frame(ctypes.byref(self._c), self.W, self.H, self.t, _p(rgb), _p(depth),
                            _p(self.sv), _p(self.sg), _p(self.sD), _p(self.R), _p(self.T),
                            _p(self.S), _p(self.gsum), _p(mask), self.nthreads)
        self.t += 1
        return mask
