"""Test glue: maps library parameters onto the oracle's and makes inputs.

Imports both the oracle and the library binding (tests may; the two never
import each other).
"""
import numpy as np

from paper_2002_00250_gb300 import synth

GMM_KEYS = ("K_rgb", "K_d", "alpha", "lambda_", "w_depth", "T_bg", "v_init_rgb", "v_init_d",
            "v_min_rgb", "v_min_d", "depth_full_scale_mm")
PBAS_KEYS = ("N", "n_min", "R_lower_rgb", "R_lower_d", "R_scale", "R_incdec", "T_lower",
             "T_upper", "T_inc", "T_dec", "alpha_g", "eps_d", "seed", "stream_id", "forced_rng",
             "depth_full_scale_mm")


def oracle_gmm_params(p):
    """Same constants as the library's float32 params, widened to float64."""
    d = p.as_dict()
    out = {}
    for k in GMM_KEYS:
        v = d[k]
        out[k] = int(v) if k in ("K_rgb", "K_d", "depth_full_scale_mm") else float(np.float32(v))
    return out


def oracle_pbas_params(p):
    d = p.as_dict()
    out = {k: d[k] for k in PBAS_KEYS}
    out["propagate"] = d["pbas_propagate"]
    out["joint"] = d["pbas_joint"]
    return out


def scene(W, H, n, seed=0, **kw):
    cfg = synth.SceneConfig(W, H, n, seed=seed, **kw)
    sc = synth.RGBDScene(cfg)
    rgb, depth, gt = (synth.to_numpy(a) for a in sc.sequence())
    return rgb, depth, gt


def close(g, o, rtol=1e-4, atol=1e-6):
    """|g - o| <= rtol |o| + atol, elementwise."""
    return np.abs(np.asarray(g, np.float64) - o) <= rtol * np.abs(o) + atol
