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


def _d8_to_mm(d8, fs=10000):
    """A depth in mm whose 8-bit reading (Sec. 4.2 rescale) is d8."""
    mm = int(round(d8 * fs / 255))
    assert (mm * 255 + fs // 2) // fs == d8
    return mm


def test_finite_temperature_one_step_closed_form():
    """One soft step at tau = 0.25 on two pixels, with theta chosen so that
    every sigmoid is a simple fraction (sigma(+-ln 3) = 3/4, 1/4); the values
    below are worked by hand from the soft step's definition.

    Pixel A, colour (1,1,1) -> (2,2,3), depth invalid at frame 1:
      S0 = |x - mu_0|^2 = 6, S1 = |x - 0|^2 = 17 (components 1, 2 are the
      bootstrap's empty ones, mu = 0).  With v0 = 22 / (3 ln 3) and
      L = 23 ln 3 / 44: (L - S0/(3 v0)) / tau = ln 3 and
      (L - S1/(3 v0)) / tau = -ln 3, so m = (3/4, 1/4, 1/4),
      r = (3/4, 1/16, 3/64), q = 9/64.  Components 1 and 2 were never used
      (w = 0): rho = 1, they jump to x with v = S1/3.  The last one is
      blended toward (alpha, x, v0) with weight q.  Classification: the
      background set is component 0 alone, Q = S0/(3 v0), p = sigma(-ln 3) = 1/4.
    Pixel B, colour constant, depth reading 50 -> 51: the colour distance to
      the background set is 0, the depth one 9/v0 (v_init_d = v0 / 9), and
      w = 17/27 gives (w 9/v0 - L)/tau = ln 3, p = 3/4.
    With ground truth (1, 0) both BCE terms are ln 4, so the loss is ln 4.
    A wrong temperature scale, a wrong responsibility product, a blend of the
    wrong component (or with 1 - q), or alpha instead of 1 for the rho of a
    never-used component each changes one of the checked numbers."""
    import math
    from oracle import softgmm
    ln3 = math.log(3.0)
    tau, alpha = 0.25, 0.2
    v0 = 22.0 / (3.0 * ln3)
    L = 23.0 * ln3 / 44.0
    w = 17.0 / 27.0
    rgb = np.zeros((1, 2, 1, 2, 3), np.uint8)
    rgb[0, 0, 0, 0] = (1, 1, 1)
    rgb[0, 1, 0, 0] = (2, 2, 3)
    rgb[0, :, 0, 1] = (1, 1, 1)
    depth = np.zeros((1, 2, 1, 2), np.uint16)
    depth[0, 0, 0, 0] = _d8_to_mm(50)
    depth[0, 0, 0, 1] = _d8_to_mm(50)
    depth[0, 1, 0, 1] = _d8_to_mm(51)
    gt = np.zeros((1, 2, 1, 2), np.uint8)
    gt[0, 1, 0, 0] = 255
    th = [torch.tensor(v, dtype=torch.float64) for v in (alpha, L, w, v0)]
    loss, finals, probs = softgmm.forward(rgb, depth, gt, *th, tau=tau)
    mr, md = finals[0]
    # soft masks and loss
    np.testing.assert_allclose(probs[0, 0].numpy(), [0.25, 0.75], rtol=1e-12)
    assert float(loss) == pytest.approx(math.log(4.0), rel=1e-12)
    # pixel A, colour model, before re-ranking: (w, mu, v) per component
    rho0 = (0.75 * alpha) / ((1 - alpha) + 0.75 * alpha)
    q = 9.0 / 64.0
    w_raw = [(1 - alpha) + 0.75 * alpha, alpha / 16.0, (1 - q) * (3.0 * alpha / 64.0) + q * alpha]
    mu_raw = [[1 + rho0 * 1, 1 + rho0 * 1, 1 + rho0 * 2], [2, 2, 3], [2, 2, 3]]
    v_raw = [v0 + rho0 * (6.0 / 3.0 - v0), 17.0 / 3.0, (1 - q) * (17.0 / 3.0) + q * v0]
    s = sum(w_raw)
    w_n = [x / s for x in w_raw]
    # ranking by w / sqrt(v): component 0 first; the blended component 2
    # (weight ~0.036) overtakes component 1 (~0.0125)
    order = sorted(range(3), key=lambda k: -w_n[k] / math.sqrt(v_raw[k]))
    assert order == [0, 2, 1]
    np.testing.assert_allclose(mr.w[0].numpy(), [w_n[k] for k in order], rtol=1e-12)
    np.testing.assert_allclose(mr.mu[0].numpy(), [mu_raw[k] for k in order], rtol=1e-12)
    np.testing.assert_allclose(mr.v[0].numpy(), [v_raw[k] for k in order], rtol=1e-12)
    # pixel A's depth model is untouched (reading invalid at frame 1)
    np.testing.assert_allclose(md.w[0].numpy(), [1, 0, 0], rtol=0, atol=0)
    np.testing.assert_allclose(md.mu[0].numpy()[:, 0], [50, 0, 0], rtol=0, atol=0)
    np.testing.assert_allclose(md.v[0].numpy(), [v0 / 9.0] * 3, rtol=1e-15)
    # pixel B, depth model: component 0 softly matched with
    # m0 = sigma((L - 9/v0)/tau) = 1 / (1 + 3^(31/11)); the empty components
    # are 51^2 * 9 / v0 away (m = 0 in double precision), so q = 1 - m0 and
    # the last one becomes (q alpha, 51 q, q v0/9 + (1-q) v0/9) = (q alpha, 51 q, v0/9)
    m0 = 1.0 / (1.0 + 3.0 ** (31.0 / 11.0))
    qd = 1.0 - m0
    w1 = (1 - alpha) + alpha * m0
    rho = alpha * m0 / w1
    wd_raw = [w1, 0.0, qd * alpha]
    sd = sum(wd_raw)
    np.testing.assert_allclose(md.w[1].numpy(), [wd_raw[0] / sd, wd_raw[2] / sd, 0.0], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(md.mu[1].numpy()[:, 0], [50 + rho, 51 * qd, 0.0], rtol=1e-12, atol=1e-15)
    vd0 = max(0.25, v0 / 9.0 + rho * (1.0 - v0 / 9.0))
    np.testing.assert_allclose(md.v[1].numpy(), [vd0, v0 / 9.0, v0 / 9.0], rtol=1e-12)
