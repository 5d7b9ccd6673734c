"""Pins for the PBAS oracle (Sec. 3.2; Hofmann et al. base method).

Hand traces with the test-only forced draws (every field written out), the
gradient-weight effect worked by hand, closed forms for constant input and a
step, invariants (bounds of R and T, S equal to the sum of D, the own-value
history rule, depth gating), and the rates of the Philox-driven draws.
"""
import numpy as np
import pytest

f32 = np.float32


def _seq(values_r, H=1, W=1, gb=50, depth=0):
    n = len(values_r)
    rgb = np.empty((n, H, W, 3), np.uint8)
    for t, v in enumerate(values_r):
        rgb[t, ..., 0] = v
    rgb[..., 1] = gb
    rgb[..., 2] = gb
    d = np.full((n, H, W), depth, np.uint16)
    return rgb, d


def test_hand_trace_single_pixel(orc):
    # N = 2, #min = 2, forced draws (own slot t mod 2), depth invalid, 1x1 frame
    # (gradient 0 everywhere, mean clamped to 1, weight 10).  Red: 100 100 130 110 110.
    rgb, d = _seq([100, 100, 130, 110, 110])
    p = orc.PBAS(1, 1, N=2, forced_rng=1)
    masks = [int(p.step(rgb[t], d[t])[0, 0]) for t in range(5)]
    assert masks == [0, 0, 255, 0, 0]
    # frame 3: d_min 10 -> D[1] = 160, S = 160, mean D = 160 / 32 = 5;
    # frame 4: slot 0 takes 110 with d_min 0.
    assert p.sv[0, 0].tolist() == [110, 110]
    assert p.sg[0, 0].tolist() == [0, 0]
    assert p.sD[0, 0].tolist() == [0, 160]
    assert int(p.S[0, 0]) == 160
    # R: 18 (floored) through frame 2, then grows twice (R < 5 * 5).
    up = f32(1) + f32(0.05)
    assert p.R[0, 0] == f32(f32(18) * up) * up
    # T: 2 (clamped) -> 2 + 1/0.0625 = 18 at frame 2, then -0.05/5 twice.
    step = f32(0.05) / f32(5)
    assert p.T[0, 0] == f32(f32(18) - step) - step
    # green/blue constant: R stays at its floor, T at its floor
    assert p.R[0, 1] == 18 and p.T[0, 1] == 2 and p.S[0, 1] == 0


def test_hand_trace_neighbour_update_3x3(orc):
    # Forced draws at frame 1: own slot 1, neighbour direction 1 (north-east),
    # neighbour slot 0.  Red goes 50 -> 60 everywhere (background, gradient 0).
    # Sources whose NE neighbour is inside: (x,y) in {0,1}x{1,2}; their targets
    # (1,0),(2,0),(1,1),(2,1) take their own value 60 into slot 0.
    rgb, d = _seq([50, 60], H=3, W=3)
    p = orc.PBAS(3, 3, N=2, forced_rng=1)
    for t in range(2):
        assert not p.step(rgb[t], d[t]).any()
    sv = p.sv[:, 0, :].reshape(3, 3, 2)
    assert (sv[..., 1] == 60).all()
    want0 = np.full((3, 3), 50)
    for (x, y) in [(1, 0), (2, 0), (1, 1), (2, 1)]:
        want0[y, x] = 60
    np.testing.assert_array_equal(sv[..., 0], want0)


def test_gradient_weight_uses_previous_mean(orc):
    # Frame 0 columns 0,0,100,100: gradient row 0,50,50,0, mean 25, weight 10/25.
    # Frame 1 columns 0,0,120,120: gradient 0,60,60,0.  Distances to the frame-0
    # samples: 0, 0.4*10 = 4, 4 + 20 = 24, 20, against R = 18:
    # only the last two columns are foreground (weight 10 would flag column 1).
    rgb = np.zeros((2, 4, 4, 3), np.uint8)
    rgb[0, :, 2:, :] = 100
    rgb[1, :, 2:, :] = 120
    d = np.zeros((2, 4, 4), np.uint16)
    p = orc.PBAS(4, 4, N=3)
    p.step(rgb[0], d[0])
    assert p.gsum.tolist() == [400, 400, 400, 0]
    m = p.step(rgb[1], d[1])
    np.testing.assert_array_equal(m, np.tile([0, 0, 255, 255], (4, 1)).astype(np.uint8))


def test_constant_input_closed_form(orc):
    # Every distance is 0: background, d_min = 0, so S = 0, mean D = eps = 1/16,
    # R stays at its floor (R > 5/16 shrinks it, the floor restores it) and T
    # drops to T_lower after one frame; samples never change.
    rgb, d = _seq([77] * 12, H=5, W=6, depth=3000)
    p = orc.PBAS(6, 5)
    for t in range(12):
        assert not p.step(rgb[t], d[t]).any()
    assert (p.R[:, :3] == 18).all() and (p.R[:, 3] == 4).all()
    assert (p.T == 2).all() and (p.S == 0).all() and (p.sD == 0).all()
    assert (p.sv[:, 0] == 77).all() and (p.sv[:, 3] == 77).all()  # 3000 mm -> 77


def test_step_change_raises_T(orc):
    # After a jump of 60 the pixel is foreground; no own update, so S stays 0
    # and mean D = 1/16: T rises by T_inc / (1/16) = 16 per frame up to 200.
    rgb, d = _seq([50] * 5 + [110] * 16, H=2, W=2)
    p = orc.PBAS(2, 2)
    Ts = []
    for t in range(21):
        m = p.step(rgb[t], d[t])
        assert m.all() == (t >= 5)
        Ts.append(float(p.T[0, 0]))
    assert Ts[4] == 2.0
    assert Ts[5:16] == [2.0 + 16 * k for k in range(1, 12)]
    assert Ts[17:] == [200.0] * 4


def _history_run(orc, W=9, H=7, n=25, seed=3):
    from paper_2002_00250_gb300 import synth
    cfg = synth.SceneConfig(W, H, n, seed=seed, n_objects=1, hole_fraction=0.2)
    sc = synth.RGBDScene(cfg)
    rgb, depth, _ = (synth.to_numpy(a) for a in sc.sequence())
    return rgb, depth


def test_invariants_and_own_value_history(orc):
    W, H, n = 9, 7, 25
    rgb, depth = _history_run(orc, W, H, n)
    p = orc.PBAS(W, H, N=6, seed=11)
    P = W * H
    hist = [[set() for _ in range(4)] for _ in range(P)]
    for t in range(n):
        ch = np.stack([rgb[t, ..., 0], rgb[t, ..., 1], rgb[t, ..., 2], orc.depth_to_u8(depth[t])])
        gr = np.stack([orc.sobel_grad_u8(c) for c in ch])
        valid = depth[t].ravel() != 0
        for i in range(P):
            for c in range(4):
                if c < 3 or valid[i] or t == 0:
                    hist[i][c].add((int(ch[c].ravel()[i]), int(gr[c].ravel()[i])))
        before_d = (p.sv[:, 3].copy(), p.sg[:, 3].copy(), p.R[:, 3].copy(), p.T[:, 3].copy())
        p.step(rgb[t], depth[t])
        assert (p.R[:, :3] >= 18).all() and (p.R[:, 3] >= 4).all()
        assert (p.T >= 2).all() and (p.T <= 200).all()
        np.testing.assert_array_equal(p.S, p.sD.astype(np.uint64).sum(axis=2))
        for i in range(P):
            for c in range(4):
                for k in range(6):
                    assert (int(p.sv[i, c, k]), int(p.sg[i, c, k])) in hist[i][c]
        if t > 0:  # depth channel untouched where the reading is invalid
            inv = ~valid
            for a, b in zip(before_d, (p.sv[:, 3], p.sg[:, 3], p.R[:, 3], p.T[:, 3])):
                np.testing.assert_array_equal(a[inv], b[inv])


def test_draw_rates(orc):
    # Background everywhere, T = 2 -> update probability 1/2.  Red 50 -> 52 with
    # gradient 0: an own update writes D = 2*16 = 32 into a uniform slot; a
    # neighbour write sets the value 52 but leaves D = 0.
    W = H = 64
    rgb, d = _seq([50, 52], H=H, W=W)
    p = orc.PBAS(W, H, seed=123)
    p.step(rgb[0], d[0])
    p.step(rgb[1], d[1])
    own = p.sD[:, 0, :] == 32
    n_own = own.sum(axis=1)
    assert set(np.unique(n_own).tolist()) <= {0, 1}
    frac = n_own.mean()
    assert abs(frac - 0.5) < 4 * np.sqrt(0.25 / (W * H))
    counts = own.sum(axis=0)
    expect = own.sum() / 20
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < 45.3  # chi-square, 19 dof, p = 0.001
    assert (counts > 0).all()
    # neighbour writes: interior pixels receive on average 8 * 1/2 * 1/8 = 0.5
    nb = ((p.sv[:, 0, :] == 52) & (p.sD[:, 0, :] == 0)).sum(axis=1).reshape(H, W)
    inner = nb[1:-1, 1:-1].mean()
    assert 0.4 < inner < 0.55


def test_seed_and_stream_change_draws(orc):
    rgb, d = _seq([50, 52], H=16, W=16)
    outs = []
    for seed, sid in [(1, 0), (1, 0), (2, 0), (1, 1)]:
        p = orc.PBAS(16, 16, seed=seed, stream_id=sid)
        p.step(rgb[0], d[0])
        p.step(rgb[1], d[1])
        outs.append(p.sD.copy())
    assert (outs[0] == outs[1]).all()
    assert (outs[0] != outs[2]).any() and (outs[0] != outs[3]).any()


# ---- spatial propagation (neighbour takes the updating pixel's value) ----

def _two_frames(W, H, seed):
    """A textured frame and the same frame 2 levels brighter: gradients are
    unchanged, so every pixel stays background and takes its draws, while
    neighbouring pixels hold different values."""
    y, x = np.mgrid[0:H, 0:W]
    f0 = np.stack([60 + (37 * x + 53 * y + 29 * c + 7 * seed) % 120 for c in range(3)], axis=-1).astype(np.uint8)
    f1 = (f0 + 2).astype(np.uint8)
    d = (1000 + 113 * x + 271 * y).astype(np.uint16)
    return f0, f1, d


def _channels(orc, rgb, depth):
    d8 = orc.depth_to_u8(depth)
    ch = [rgb[..., c] for c in range(3)] + [d8]
    return [(c_.astype(np.uint8), orc.sobel_grad_u8(c_.astype(np.uint8))) for c_ in ch]


def test_propagation_takes_the_requesters_value(orc):
    """Forced draws at t = 1: every pixel asks its north-east neighbour (slot
    (t+1) mod N = 0); with propagation that slot gets the asking pixel's
    frame-1 value and gradient; pixels nobody asks keep their bootstrap value."""
    W, H, N = 5, 4, 2
    f0, f1, d = _two_frames(W, H, 1)
    p = orc.PBAS(W, H, N=N, forced_rng=1, propagate=1)
    p.step(f0, d)
    p.step(f1, d)
    chs = _channels(orc, f1, d)
    boot = _channels(orc, f0, d)
    for yy in range(H):
        for xx in range(W):
            rx, ry = xx - 1, yy + 1          # the pixel whose NE neighbour this is
            i = yy * W + xx
            for c in range(4):
                if 0 <= rx < W and 0 <= ry < H:
                    want = (chs[c][0][ry, rx], chs[c][1][ry, rx])
                else:
                    want = (boot[c][0][yy, xx], boot[c][1][yy, xx])
                assert (p.sv[i, c, 0], p.sg[i, c, 0]) == want, (xx, yy, c)
                # own update (slot t mod N = 1) with its own frame-1 value
                assert (p.sv[i, c, 1], p.sg[i, c, 1]) == (chs[c][0][yy, xx], chs[c][1][yy, xx])


def test_propagation_conflict_east_neighbour_wins(orc):
    """Forced mode 2: columns 0,1 (mod 4) ask east, 2,3 ask west, so columns
    1 and 2 (mod 4) are asked by both sides for the same slot; seen from the
    asked pixel the right neighbour lies east (direction 2) and the left one
    west (6), so the right one wins.  Without propagation every asked pixel
    takes its own value."""
    W, H, N = 9, 3, 2
    f0, f1, d = _two_frames(W, H, 2)
    chs = _channels(orc, f1, d)
    boot = _channels(orc, f0, d)
    east = lambda x: ((x >> 1) & 1) == 0
    for prop in (1, 0):
        p = orc.PBAS(W, H, N=N, forced_rng=2, propagate=prop)
        p.step(f0, d)
        p.step(f1, d)
        for yy in range(H):
            for u in range(W):
                from_left = u - 1 >= 0 and east(u - 1)
                from_right = u + 1 < W and not east(u + 1)
                if not (from_left or from_right):
                    src = None
                elif not prop:
                    src = u
                else:
                    src = u + 1 if from_right else u - 1
                for c in range(4):
                    got = (p.sv[yy * W + u, c, 0], p.sg[yy * W + u, c, 0])
                    if src is None:
                        want = (boot[c][0][yy, u], boot[c][1][yy, u])
                    else:
                        want = (chs[c][0][yy, src], chs[c][1][yy, src])
                    assert got == want, (prop, u, yy, c)


@pytest.mark.parametrize("joint", [0, 1])
def test_propagation_own_update_and_lowest_direction_win(orc, joint):
    """Forced mode 3 at t = 1 (N = 2, own slot 1): even columns ask north,
    odd ones south-east, so every pixel of an even column is asked from below
    (direction 4 seen from it) and from the north-west (7).  Requesters on
    even rows ask for slot 1, the slot of the asked pixel's own update, which
    keeps the pixel's own value; requesters on odd rows ask for slot 0, which
    takes the value of the neighbour below where there is one, else of the
    north-west one.  Without propagation an asked slot 0 takes the pixel's
    own value.  The joint-channel variant (one draw per pixel, whole-sample
    requests) gives the same slots in every channel."""
    W, H, N = 8, 6, 2
    f0, f1, d = _two_frames(W, H, 3)
    chs = _channels(orc, f1, d)
    boot = _channels(orc, f0, d)
    for prop in (1, 0):
        p = orc.PBAS(W, H, N=N, forced_rng=3, propagate=prop, joint=joint)
        p.step(f0, d)
        p.step(f1, d)
        for v in range(H):
            for u in range(W):
                below = u % 2 == 0 and v + 1 < H
                northwest = u % 2 == 0 and u >= 1 and v >= 1
                if v % 2 == 1 or not (below or northwest):
                    src = None                        # slot 0 not asked for
                elif not prop:
                    src = (u, v)
                else:
                    src = (u, v + 1) if below else (u - 1, v - 1)
                for c in range(4):
                    i = v * W + u
                    want = (boot[c][0][v, u], boot[c][1][v, u]) if src is None else \
                        (chs[c][0][src[1], src[0]], chs[c][1][src[1], src[0]])
                    assert (p.sv[i, c, 0], p.sg[i, c, 0]) == want, (prop, u, v, c)
                    # slot 1: the own update, never overwritten by a neighbour
                    assert (p.sv[i, c, 1], p.sg[i, c, 1]) == (chs[c][0][v, u], chs[c][1][v, u]), (prop, u, v, c)
