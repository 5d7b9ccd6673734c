"""Pins for the paper-literal GMM variant of the oracle (Sec. 3.1 as printed:
K = 7 / 3, FP64, one variance per colour channel, decision on the product of
the two models' s-scaled Eq. 1 densities).

* On grey input (R = G = B) the three channel variances of a component stay
  equal, so the update must reproduce the default GMM oracle exactly (its
  isotropic variance), component by component, frame by frame.
* The density factor follows Eq. 1 in closed form: a constant pixel keeps one
  component (w = 1, mu = x, v = max(v_min, v_init (1 - alpha)^t)) and a
  factor s / (2 pi v) per model; one frame after the bootstrap the colour
  factor is s exp(-D / 2) / (2 pi v_init), D = sum (x1 - x0)^2 / v_init.
  The decision flips exactly where the product crosses theta.
* Channels are independent: with only R varying, the G and B means never
  move and their variances stay equal to each other.
* Invariants: weights sum to 1, every channel variance >= v_min.
"""
import numpy as np
import pytest

from _helpers import scene

ALPHA = 0.001


def _grey(rgb):
    g = rgb.mean(axis=-1).round().astype(np.uint8)
    return np.repeat(g[..., None], 3, axis=-1)


def test_grey_input_reproduces_the_default_gmm(orc):
    W, H, n = 24, 16, 30
    rgb, depth, _ = scene(W, H, n, seed=5)
    rgb = _grey(rgb)
    lit = orc.GMMLiteral(W, H, K_rgb=7, K_d=3, alpha=0.05)
    ref = orc.GMM(W, H, K_rgb=7, K_d=3, alpha=0.05)
    for t in range(n):
        lit.step(rgb[t], depth[t])
        _, margin = ref.step(rgb[t], depth[t], want_margin=True)
        if t == 0:
            continue
        ok = margin.ravel() > 1e-9
        assert ok.mean() > 0.9
        np.testing.assert_allclose(lit.w_rgb[ok], ref.w_rgb[ok], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(lit.mu_rgb[ok], ref.mu_rgb[ok], rtol=1e-12, atol=1e-12)
        for ch in range(3):
            np.testing.assert_allclose(lit.v_rgb[ok][..., ch], ref.v_rgb[ok], rtol=1e-12)
        np.testing.assert_allclose(lit.w_d[ok], ref.w_d[ok], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(lit.v_d[ok], ref.v_d[ok], rtol=1e-12)


def test_constant_pixel_density_closed_form(orc):
    x, d_mm, t_end = (90, 120, 150), 2500, 12
    v_rgb = max(4.0, 36.0 * (1 - ALPHA) ** (t_end - 1))
    v_d = max(0.25, 4.0 * (1 - ALPHA) ** (t_end - 1))
    s = 10000.0
    F = (s / (2 * np.pi * v_rgb)) * (s / (2 * np.pi * v_d))
    for theta, want in ((F * (1 - 1e-9), 0), (F * (1 + 1e-9), 255)):
        g = orc.GMMLiteral(1, 1, theta=theta)
        rgb = np.array([[x]], np.uint8)
        dep = np.array([[d_mm]], np.uint16)
        for t in range(t_end + 1):
            m = g.step(rgb, dep)
        assert m[0, 0] == want
        np.testing.assert_allclose(g.v_rgb[0, 0], v_rgb * (1 - ALPHA), rtol=1e-13)
        assert g.w_rgb[0, 0] == 1.0


def test_first_step_factor_by_hand(orc):
    x0, x1 = np.array([100, 100, 100]), np.array([104, 97, 101])
    D = float(((x1 - x0) ** 2).sum()) / 36.0
    F = 10000.0 * np.exp(-D / 2) / (2 * np.pi * 36.0)   # depth invalid: colour factor only
    for theta, want in ((F * (1 - 1e-9), 0), (F * (1 + 1e-9), 255)):
        g = orc.GMMLiteral(1, 1, theta=theta)
        g.step(x0.astype(np.uint8).reshape(1, 1, 3), np.zeros((1, 1), np.uint16))
        m = g.step(x1.astype(np.uint8).reshape(1, 1, 3), np.zeros((1, 1), np.uint16))
        assert m[0, 0] == want


def test_channels_are_independent(orc):
    rng = np.random.default_rng(3)
    g = orc.GMMLiteral(1, 1, alpha=0.05)
    for t in range(40):
        r = int(100 + rng.integers(-6, 7))
        g.step(np.array([[[r, 80, 80]]], np.uint8), np.array([[3000]], np.uint16))
    k0 = 0
    assert g.mu_rgb[0, k0, 1] == 80.0 and g.mu_rgb[0, k0, 2] == 80.0
    assert g.v_rgb[0, k0, 1] == g.v_rgb[0, k0, 2]
    assert g.v_rgb[0, k0, 0] != g.v_rgb[0, k0, 1]


def test_invariants(orc):
    W, H, n = 20, 12, 25
    rgb, depth, _ = scene(W, H, n, seed=9)
    g = orc.GMMLiteral(W, H, alpha=0.02)
    for t in range(n):
        g.step(rgb[t], depth[t])
        np.testing.assert_allclose(g.w_rgb.sum(1), 1.0, atol=1e-12)
        np.testing.assert_allclose(g.w_d.sum(1), 1.0, atol=1e-12)
        assert (g.v_rgb >= 4.0).all() and (g.v_d >= 0.25).all()


def test_diagonal_mixture_factor_recomputed(orc):
    """After the channel variances diverge, the next frame's factor equals the
    s-scaled background-set mixture density with the geometric-mean
    normalisation, recomputed here from the state."""
    rng = np.random.default_rng(11)
    frames = [np.array([[[int(100 + rng.integers(-9, 10)), int(60 + rng.integers(-2, 3)),
                          int(200 + rng.integers(-20, 21))]]], np.uint8) for _ in range(41)]
    nodepth = np.zeros((1, 1), np.uint16)
    probe = orc.GMMLiteral(1, 1, alpha=0.05)
    for t in range(40):
        probe.step(frames[t], nodepth)
    w, mu, v = probe.w_rgb[0], probe.mu_rgb[0], probe.v_rgb[0]
    assert np.ptp(v[0]) > 1.0                      # the channels did diverge
    x = frames[40][0, 0].astype(np.float64)
    num = den = cum = 0.0
    for k in range(len(w)):
        D = (((x - mu[k]) ** 2) / v[k]).sum()
        g = np.prod(v[k]) ** (1.0 / 3.0)
        num += w[k] * np.exp(-D / 2) / (2 * np.pi * g)
        den += w[k]
        cum += w[k]
        if cum > 0.7:
            break
    F = 10000.0 * num / den
    for theta, want in ((F * (1 - 1e-9), 0), (F * (1 + 1e-9), 255)):
        g2 = orc.GMMLiteral(1, 1, alpha=0.05, theta=theta)
        for t in range(41):
            m = g2.step(frames[t], nodepth)
        assert m[0, 0] == want
