"""Pins for the FP64 GMM oracle (Sec. 3.1, Eq. 1; Stauffer-Grimson base update).

Closed forms (constant input), a library special case (K = 1 is an
exponential moving average, checked with scipy.signal.lfilter), a hand trace
of a step change, invariants on synthetic video, the depth-weight special
cases, and the threshold-margin report.
"""
import numpy as np
import pytest


def _frames(rgb_val, depth_val, n, H=3, W=4):
    rgb = np.empty((n, H, W, 3), np.uint8)
    rgb[:] = np.asarray(rgb_val, np.uint8)
    depth = np.full((n, H, W), depth_val, np.uint16)
    return rgb, depth


def test_constant_pixel_closed_form(orc):
    # Constant X: component 0 matches every frame with weight 1, so rho = alpha,
    # mu stays X and v(t) = max(v_min, v_init (1-alpha)^t); nothing is foreground.
    n = 200
    rgb, depth = _frames((100, 150, 200), 2000, n)
    g = orc.GMM(4, 3, alpha=0.01)
    for t in range(n):
        m = g.step(rgb[t], depth[t])
        assert not m.any()
    P = 12
    vt = max(4.0, 36.0 * (1 - 0.01) ** (n - 1))
    np.testing.assert_allclose(g.w_rgb[:, 0], 1.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(g.w_rgb[:, 1:], 0.0, atol=0)
    np.testing.assert_array_equal(g.mu_rgb[:, 0], np.tile([100.0, 150.0, 200.0], (P, 1)))
    np.testing.assert_allclose(g.v_rgb[:, 0], vt, rtol=1e-12)
    # depth 2000 mm -> 51 (Sec. 4.2 rescale)
    np.testing.assert_array_equal(g.mu_d[:, 0], 51.0)
    np.testing.assert_allclose(g.v_d[:, 0], max(0.25, 4.0 * 0.99 ** (n - 1)), rtol=1e-12)


def test_single_component_is_ema(orc):
    signal = pytest.importorskip("scipy.signal")
    # K = 1, threshold never exceeded: w stays 1, rho = alpha, so the mean is the
    # exponential moving average of the input and v the EMA of the squared
    # deviation from the previous mean.
    rng = np.random.default_rng(0)
    n, a = 80, 0.05
    x = rng.integers(60, 200, size=(n, 3)).astype(np.uint8)
    rgb = np.broadcast_to(x[:, None, None, :], (n, 1, 1, 3)).copy()
    depth = np.zeros((n, 1, 1), np.uint16)
    g = orc.GMM(1, 1, K_rgb=1, K_d=1, alpha=a, lambda_=1e6, v_min_rgb=1e-12)
    mus = []
    for t in range(n):
        g.step(rgb[t], depth[t])
        mus.append(g.mu_rgb[0, 0].copy())
    xf = x.astype(np.float64)
    ema = np.stack([signal.lfilter([a], [1, -(1 - a)], xf[1:, c], zi=[(1 - a) * xf[0, c]])[0]
                    for c in range(3)], axis=1)
    np.testing.assert_allclose(np.array(mus[1:]), ema, rtol=1e-12)
    prev_mu = np.vstack([xf[:1], ema[:-1]])
    e = ((xf[1:] - prev_mu) ** 2).sum(axis=1) / 3.0
    v = signal.lfilter([a], [1, -(1 - a)], e, zi=[(1 - a) * 36.0])[0]
    np.testing.assert_allclose(g.v_rgb[0, 0], v[-1], rtol=1e-10)


def test_step_change_hand_trace(orc):
    # K = 2, alpha = 0.1, T_bg = 0.7, depth invalid (colour-only decision).
    # 30 frames of X then Y far from X.  At frame t0+m the old component's
    # weight before the update is 0.9^m and it stays ranked first (its variance
    # sits at v_min), so B = {old} while 0.9^m > 0.7: foreground for m = 0..3
    # (0.9^3 = 0.729), background from m = 4 (0.9^4 = 0.6561).
    t0, n = 30, 45
    rgb = np.empty((n, 1, 1, 3), np.uint8)
    rgb[:t0] = 100
    rgb[t0:] = 200
    depth = np.zeros((n, 1, 1), np.uint16)
    g = orc.GMM(1, 1, K_rgb=2, K_d=2, alpha=0.1, T_bg=0.7)
    masks = [int(g.step(rgb[t], depth[t])[0, 0]) for t in range(n)]
    assert masks[:t0] == [0] * t0
    assert masks[t0:t0 + 4] == [255] * 4
    assert masks[t0 + 4:] == [0] * (n - t0 - 4)
    # replay to frame t0 and check the state written out by hand
    g = orc.GMM(1, 1, K_rgb=2, K_d=2, alpha=0.1, T_bg=0.7)
    for t in range(t0 + 1):
        g.step(rgb[t], depth[t])
    np.testing.assert_allclose(g.w_rgb[0], [0.9, 0.1], rtol=1e-12)
    np.testing.assert_array_equal(g.mu_rgb[0, 1], [200.0, 200.0, 200.0])
    assert g.v_rgb[0, 1] == 36.0 and g.v_rgb[0, 0] == 4.0
    # one more frame: the new component matched, w = (0.81, 0.19), v = 36 (1 - 0.1/0.19)
    g.step(rgb[t0 + 1], depth[t0 + 1])
    np.testing.assert_allclose(g.w_rgb[0], [0.81, 0.19], rtol=1e-12)
    np.testing.assert_allclose(g.v_rgb[0, 1], 36.0 * (1 - 0.1 / 0.19), rtol=1e-12)


def test_invariants_on_synthetic_video(orc):
    from paper_2002_00250_gb300 import synth
    cfg = synth.SceneConfig(64, 48, 40, seed=5, n_objects=2)
    sc = synth.RGBDScene(cfg)
    rgb, depth, _ = (synth.to_numpy(a) for a in sc.sequence())
    g = orc.GMM(64, 48, alpha=0.05)
    for t in range(cfg.n_frames):
        before = (g.w_d.copy(), g.mu_d.copy(), g.v_d.copy())
        g.step(rgb[t], depth[t])
        for w, v, vmin in ((g.w_rgb, g.v_rgb, 4.0), (g.w_d, g.v_d, 0.25)):
            np.testing.assert_allclose(w.sum(axis=1), 1.0, atol=1e-12)
            assert (w >= 0).all() and (w <= 1).all()
            assert (v >= vmin).all()
            key = w / np.sqrt(v)
            assert (np.diff(key, axis=1) <= 0).all()
        if t > 0:
            inv = (depth[t].ravel() == 0)
            for a, b in zip(before, (g.w_d, g.mu_d, g.v_d)):
                np.testing.assert_array_equal(a[inv], b[inv])


def test_depth_weight_special_cases(orc):
    # Colour camouflage: colour unchanged, the pixel moves 1000 mm closer.
    # w_depth = 0 is the colour-only Stauffer decision (background); with
    # w_depth = 0.5 the depth distance alone makes it foreground; with the
    # depth reading invalid the decision falls back to colour only.
    n = 21
    rgb, depth = _frames((100, 100, 100), 2000, n + 1, 1, 1)
    depth[n] = 1000
    for w, want in ((0.0, 0), (0.5, 255)):
        g = orc.GMM(1, 1, w_depth=w)
        for t in range(n):
            g.step(rgb[t], depth[t])
        assert int(g.step(rgb[n], depth[n])[0, 0]) == want
    g = orc.GMM(1, 1, w_depth=0.5)
    for t in range(n):
        g.step(rgb[t], depth[t])
    depth[n] = 0
    assert int(g.step(rgb[n], depth[n])[0, 0]) == 0


def test_margin_is_zero_on_an_exact_tie(orc):
    # diff = 15 on each channel with v = 36: d^2 = 675 / 108 = 6.25 = lambda^2 exactly.
    # The strict match test fails (new component), the score equals lambda^2
    # (foreground), and the reported margin is 0.
    rgb = np.array([[[[100, 100, 100]]], [[[115, 115, 115]]]], np.uint8)
    depth = np.zeros((2, 1, 1), np.uint16)
    g = orc.GMM(1, 1)
    g.step(rgb[0], depth[0])
    m, margin = g.step(rgb[1], depth[1], want_margin=True)
    assert int(m[0, 0]) == 255
    assert margin[0, 0] == 0.0
    np.testing.assert_allclose(g.w_rgb[0], [0.999, 0.001, 0.0], rtol=1e-12)
    np.testing.assert_array_equal(g.mu_rgb[0, 1], [115.0] * 3)
