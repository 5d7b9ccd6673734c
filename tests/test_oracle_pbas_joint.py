"""Pins for the joint-channel PBAS variant of the oracle (one R, T, D per
pixel; one decision on the mean distance over the active channels).

Closed forms on one-pixel frames (the mean over four channels absorbs a
single-channel change that the per-channel method flags; with the depth
reading invalid the mean is over three), the depth slot left alone where the
reading is invalid, neighbour updates and propagation writing whole samples,
the bootstrap values of the unused per-channel entries, S equal to the sum of
D, the own-value history of every slot, and one random draw per pixel (the
counter's channel word 0).
"""
import numpy as np
import pytest

from test_oracle_pbas import _channels, _two_frames

f32 = np.float32


def _px(rgb0, rgb1, d0, d1):
    rgb = np.array([rgb0, rgb1], np.uint8).reshape(2, 1, 1, 3)
    d = np.array([d0, d1], np.uint16).reshape(2, 1, 1)
    return rgb, d


@pytest.mark.parametrize("dr,depth1,joint_fg", [(60, 5000, False), (80, 5000, True), (60, 0, True),
                                                (52, 0, False), (54, 0, True)])
def test_mean_over_active_channels(orc, dr, depth1, joint_fg):
    # one pixel (gradient 0), both slots hold frame 0; R = 18.  Red moves by dr,
    # the other channels stay: mean distance dr / 4 with valid depth, dr / 3
    # (times the rounded 1/3) without; 52/3 -> 17.33 < 18 < 18 = 54/3
    rgb, d = _px([100, 50, 50], [100 + dr, 50, 50], 5000, depth1)
    pj = orc.PBAS(1, 1, N=2, forced_rng=1, joint=1)
    ps = orc.PBAS(1, 1, N=2, forced_rng=1, joint=0)
    for t in range(2):
        mj = int(pj.step(rgb[t], d[t])[0, 0])
        ms = int(ps.step(rgb[t], d[t])[0, 0])
    assert mj == (255 if joint_fg else 0)
    assert ms == 255  # the red channel alone is beyond R = 18
    nc = 4 if depth1 else 3
    dist = f32(f32(dr) * (f32(1) / f32(nc)))
    if joint_fg:
        # no update; mean D = eps = 1/16: R shrinks to its floor, T += 1 / (1/16)
        assert pj.R[0, 0] == 18 and pj.T[0, 0] == 18 and pj.S[0, 0] == 0
        assert pj.sv[0, 0].tolist() == [100, 100]
    else:
        q = int(np.rint(dist * f32(16)))
        assert pj.sv[0, 0].tolist() == [100, 100 + dr]          # own slot t mod 2 = 1
        assert pj.sD[0, 0].tolist() == [0, q] and pj.S[0, 0] == q
        dbar = f32(f32(q) / f32(32))
        assert pj.R[0, 0] == (f32(18) * f32(f32(1) + f32(0.05)) if f32(18) <= dbar * f32(5) else 18)
        assert pj.T[0, 0] == 2
        # the depth slot is written only with a valid reading
        assert pj.sv[0, 3, 1] == (orc.depth_to_u8(np.array([depth1], np.uint16))[0] if depth1 else pj.sv[0, 3, 0])
    # the per-channel entries of channels 1..3 keep their bootstrap values
    assert pj.R[0, 1:].tolist() == [18, 18, 4] and (pj.T[0, 1:] == 2).all()
    assert (pj.S[0, 1:] == 0).all() and (pj.sD[0, 1:] == 0).all()


@pytest.mark.parametrize("prop", [0, 1])
def test_neighbour_update_writes_whole_samples(orc, prop):
    """Forced draws at t = 1: every pixel asks its north-east neighbour for
    slot 0 and updates its own slot 1.  The asked pixel's slot 0 gets, in all
    four channels, its own frame-1 value (base method) or the asking pixel's
    (propagation); pixels nobody asks keep their bootstrap sample."""
    W, H, N = 5, 4, 2
    f0, f1, d = _two_frames(W, H, 4)
    p = orc.PBAS(W, H, N=N, forced_rng=1, propagate=prop, joint=1)
    p.step(f0, d)
    assert not p.step(f1, d).any()
    chs, boot = _channels(orc, f1, d), _channels(orc, f0, d)
    for yy in range(H):
        for xx in range(W):
            rx, ry = xx - 1, yy + 1
            asked = 0 <= rx < W and 0 <= ry < H
            sx, sy = ((rx, ry) if prop else (xx, yy)) if asked else (xx, yy)
            src = chs if asked else boot
            for c in range(4):
                i = yy * W + xx
                assert (p.sv[i, c, 0], p.sg[i, c, 0]) == (src[c][0][sy, sx], src[c][1][sy, sx]), (xx, yy, c)
                assert (p.sv[i, c, 1], p.sg[i, c, 1]) == (chs[c][0][yy, xx], chs[c][1][yy, xx])


def test_one_draw_per_pixel(orc):
    """Static textured scene, Philox draws, T = 2 at t = 1: exactly the
    pixels whose counter (pixel, 1, 0, 0) fires coin 1 (word 0) made an own
    update, into slot floor(word1 * N / 2^32), with D = 16 * mean distance
    (2, 2, 2, 0 over four channels: 1.5 -> 24); neighbour writes leave D."""
    W, H, N = 16, 12, 5
    f0, f1, d = _two_frames(W, H, 5)
    p = orc.PBAS(W, H, N=N, seed=7, stream_id=3, joint=1)
    p.step(f0, d)
    p.step(f1, d)
    P = W * H
    ctr = np.stack([np.arange(P), np.ones(P), np.zeros(P), np.zeros(P)], 1).astype(np.uint32)
    u = orc.philox4x32_10(ctr, np.array([7, 3], np.uint32))
    coin1 = (u[:, 0] >> 8).astype(np.float32) * f32(2.0 ** -24) < f32(0.5)
    k1 = (u[:, 1].astype(np.uint64) * N) >> 32
    want = np.zeros((P, N), np.uint16)
    want[np.arange(P)[coin1], k1[coin1].astype(np.int64)] = 24
    np.testing.assert_array_equal(p.sD[:, 0, :], want)
    assert 0.3 < coin1.mean() < 0.7


def test_invariants_and_own_value_history(orc):
    from test_oracle_pbas import _history_run
    W, H, n, N = 9, 7, 25, 6
    rgb, depth = _history_run(orc, W, H, n, seed=4)
    p = orc.PBAS(W, H, N=N, seed=12, joint=1)
    P = W * H
    hist = [[set() for _ in range(4)] for _ in range(P)]
    fg_total = 0
    for t in range(n):
        ch = np.stack([rgb[t, ..., 0], rgb[t, ..., 1], rgb[t, ..., 2], orc.depth_to_u8(depth[t])])
        gr = np.stack([orc.sobel_grad_u8(c) for c in ch])
        valid = depth[t].ravel() != 0
        for i in range(P):
            for c in range(4):
                if c < 3 or valid[i] or t == 0:
                    hist[i][c].add((int(ch[c].ravel()[i]), int(gr[c].ravel()[i])))
        fg_total += int(p.step(rgb[t], depth[t]).astype(bool).sum())
        assert (p.R[:, 0] >= 18).all() and (p.T[:, 0] >= 2).all() and (p.T[:, 0] <= 200).all()
        assert (p.R[:, 1:] == np.array([18, 18, 4], np.float32)).all() and (p.T[:, 1:] == 2).all()
        assert (p.S[:, 1:] == 0).all() and (p.sD[:, 1:] == 0).all()
        np.testing.assert_array_equal(p.S[:, 0], p.sD[:, 0].astype(np.uint64).sum(axis=1))
        for i in range(P):
            for c in range(4):
                for k in range(N):
                    assert (int(p.sv[i, c, k]), int(p.sg[i, c, k])) in hist[i][c]
    assert fg_total > 0
