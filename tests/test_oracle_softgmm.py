"""Pins for the soft-GMM oracle (the differentiable form of the Sec. 3.1 GMM).

* As the temperature goes to 0 the soft forward equals the hard GMM oracle
  (C, FP64) on every pixel whose hard decisions are clear of their
  thresholds.
* The autograd adjoint equals central FP64 finite differences (h = 1e-6 |theta|)
  to 1e-5 relative, where the discrete decisions (ranks, background sets,
  arg-mins, v_min clamps) are the same at theta +/- h.
* Invariants of the soft state.
"""
import numpy as np
import pytest
import torch

from _helpers import scene

THETA = (0.05, 6.25, 0.5, 36.0)


def _seq(W, H, T, seed):
    rgb, depth, gt = scene(W, H, T, seed=seed, n_objects=2, hole_fraction=0.1)
    return rgb[None], depth[None], gt[None]


def test_zero_temperature_is_the_hard_gmm(orc):
    from oracle import softgmm
    W, H, T = 14, 10, 12
    rgb, depth, gt = _seq(W, H, T, 3)
    alpha = 0.05
    hard = orc.GMM(W, H, alpha=alpha)
    clear = np.ones(W * H, bool)
    for t in range(T):
        _, margin = hard.step(rgb[0, t], depth[0, t], want_margin=True)
        clear &= margin.ravel() >= 0.15
    assert clear.mean() > 0.5
    th = [torch.tensor(v, dtype=torch.float64) for v in (alpha, 6.25, 0.5, 36.0)]
    _, finals, probs = softgmm.forward(rgb, depth, gt, *th, tau=1e-3)
    mr, md = finals[0]
    np.testing.assert_allclose(mr.w.numpy()[clear], hard.w_rgb[clear], rtol=0, atol=1e-12)
    np.testing.assert_allclose(mr.mu.numpy()[clear], hard.mu_rgb[clear], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(mr.v.numpy()[clear], hard.v_rgb[clear], rtol=1e-12)
    np.testing.assert_allclose(md.w.numpy()[clear], hard.w_d[clear], rtol=0, atol=1e-12)
    np.testing.assert_allclose(md.mu.numpy()[clear][:, :, 0], hard.mu_d[clear], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(md.v.numpy()[clear], hard.v_d[clear], rtol=1e-12)
    # the last frame's soft mask is the hard mask
    hard2 = orc.GMM(W, H, alpha=alpha)
    for t in range(T):
        m = hard2.step(rgb[0, t], depth[0, t])
    p = probs[0, -1].numpy()
    np.testing.assert_array_equal((p[clear] > 0.5), m.ravel()[clear] > 0)


@pytest.mark.parametrize("seed", [1, 2])
def test_adjoint_matches_finite_differences(seed):
    from oracle import softgmm
    rgb, depth, gt = _seq(8, 6, 10, seed)
    loss, g = softgmm.loss_and_grad(rgb, depth, gt, THETA)
    assert np.isfinite(loss) and np.all(np.isfinite(g))
    fp0 = softgmm.fingerprint(rgb, depth, gt, THETA)
    checked = 0
    for i in range(4):
        h = 1e-6 * abs(THETA[i])
        tp = list(THETA); tp[i] += h
        tm = list(THETA); tm[i] -= h
        if not (softgmm.fingerprint(rgb, depth, gt, tp) == fp0 == softgmm.fingerprint(rgb, depth, gt, tm)):
            continue
        lp, _ = softgmm.loss_and_grad(rgb, depth, gt, tp)
        lm, _ = softgmm.loss_and_grad(rgb, depth, gt, tm)
        fd = (lp - lm) / (2 * h)
        scale = max(abs(g[i]), 1e-3 * np.abs(g * np.array(THETA)).max() / abs(THETA[i]))
        assert abs(fd - g[i]) <= 1e-5 * scale, (i, fd, g[i])
        checked += 1
    assert checked >= 3


def test_soft_state_invariants():
    from oracle import softgmm
    rgb, depth, gt = _seq(10, 8, 9, 4)
    th = [torch.tensor(v, dtype=torch.float64) for v in THETA]
    loss, finals, probs = softgmm.forward(rgb, depth, gt, *th)
    mr, md = finals[0]
    for m, vmin in ((mr, 4.0), (md, 0.25)):
        np.testing.assert_allclose(m.w.sum(1).numpy(), 1.0, atol=1e-12)
        assert (m.v.numpy() >= vmin).all()
        key = (m.w / torch.sqrt(m.v)).numpy()
        assert (np.diff(key, axis=1) <= 0).all()
    assert ((probs >= 0) & (probs <= 1)).all()
    assert float(loss) > 0


def test_gradient_step_lowers_the_loss():
    from oracle import softgmm
    rgb, depth, gt = _seq(8, 6, 10, 5)
    # a small step along minus the gradient in log-parameter space
    theta = np.array(THETA)
    l0, g = softgmm.loss_and_grad(rgb, depth, gt, theta)
    d = -g * theta
    theta1 = theta * np.exp(1e-4 * d / np.abs(d).max())
    l1, _ = softgmm.loss_and_grad(rgb, depth, gt, theta1)
    assert l1 < l0
    # first-order prediction of the decrease
    pred = float(np.dot(g, theta1 - theta))
    assert l1 - l0 == pytest.approx(pred, rel=0.05)
