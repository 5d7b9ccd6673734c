"""The paper-literal GMM (FP64, per-channel variances, s-scaled density
product) on the GPU against the FP64 oracle.

Both sides compute in IEEE double; they differ only in operation order,
fused multiply-adds and the last bit of exp/pow, i.e. ~1e-15 relative per
step.  Step parity loads the oracle with the GPU's state of frame t-1 and
runs one frame: every parameter must agree to 1e-11 relative (+1e-13
absolute) and the masks exactly, except at pixels where one of the frame's
discrete decisions lies within 1e-9 (relative; log-ratio for the density
decision) of its threshold in the oracle.
"""
import numpy as np
import pytest

from _helpers import oracle_gmm_params, scene

pytestmark = pytest.mark.gpu


def _oracle(orc, seg, W, H):
    """The oracle with the library's float32 constants widened to double."""
    pr = oracle_gmm_params(seg.params)
    return orc.GMMLiteral(W, H, s=float(np.float32(seg.params.density_scale)),
                          theta=float(np.float32(seg.params.density_threshold)), **pr)


def _load(o, g):
    for k in ("w_rgb", "mu_rgb", "v_rgb", "w_d", "mu_d", "v_d"):
        getattr(o, k)[...] = g[k]


@pytest.mark.parametrize("Kr,Kd", [(7, 3), (3, 3)])
def test_step_parity(orc, Kr, Kd):
    from paper_2002_00250_gb300 import fos
    W, H, n = 40, 24, 12
    rgb, depth, _ = scene(W, H, n, seed=21)
    seg = fos.Segmenter(W, H, methods=fos.METHOD_GMM, gmm_literal=1, K_rgb=Kr, K_d=Kd, alpha=0.05)
    o = _oracle(orc, seg, W, H)
    prev = None
    for t in range(n):
        mg, _ = seg.process_host(rgb[t], depth[t])
        g = fos.decode_state(seg.get_state()).gmm
        if t == 0:
            o.step(rgb[0], depth[0])
        else:
            _load(o, prev)
            o.t = t
            m_o, margin = o.step(rgb[t], depth[t], want_margin=True)
            clear = margin.ravel() > 1e-9
            assert clear.mean() > 0.97
            np.testing.assert_array_equal(mg.ravel()[clear], m_o.ravel()[clear])
            for k in ("w_rgb", "mu_rgb", "v_rgb", "w_d", "mu_d", "v_d"):
                np.testing.assert_allclose(g[k][clear], getattr(o, k)[clear], rtol=1e-11, atol=1e-13,
                                           err_msg=f"{k} frame {t}")
        prev = {k: np.array(v) for k, v in g.items()}


def test_free_run_masks(orc):
    from paper_2002_00250_gb300 import fos
    W, H, n = 160, 120, 20
    rgb, depth, _ = scene(W, H, n, seed=22)
    seg = fos.Segmenter(W, H, methods=fos.METHOD_GMM, gmm_literal=1, K_rgb=7, K_d=3)
    mg, _ = seg.process_host(rgb, depth)
    o = _oracle(orc, seg, W, H)
    # a pixel whose decision was ever within 1e-9 of a threshold may have
    # taken the other branch there, and its model differs from then on
    tied = np.zeros((H, W), bool)
    for t in range(n):
        m_o, margin = o.step(rgb[t], depth[t], want_margin=True)
        tied |= margin < 1e-9
        np.testing.assert_array_equal(mg[t][~tied], m_o[~tied], err_msg=f"frame {t}")
    assert tied.mean() <= 1e-2
    g = fos.decode_state(seg.get_state()).gmm
    np.testing.assert_allclose(g["w_rgb"].sum(1), 1.0, atol=1e-12)


def test_literal_variant_is_not_batched():
    from paper_2002_00250_gb300 import fos
    with pytest.raises(fos.FosError):
        fos.Batch(2, gmm_literal=1)
