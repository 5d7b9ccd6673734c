"""A second, independent PBAS path (Sec. 3.2) against the oracle on tiny frames.

The oracle resolves neighbour updates by gathering: each asked pixel looks at
its eight neighbours in direction order.  This path is written the other way
round, pixel by pixel in raster order as a sequential CPU PBAS would be, but
with the two-phase semantics of the definition: every pixel is classified
against the model of the previous frame (a snapshot), then the own updates
and the neighbour requests are scattered into the model.  Conflicts follow the
stated rule: a slot that the asked pixel's own update of this frame wrote
keeps that value, and among requesters asking for the same slot the one at
the lowest direction index seen from the asked pixel wins.  In the base method
every writer of a slot writes the asked pixel's own value, so the result may
not depend on the order at all.  Arithmetic is numpy float32 (one rounding per
operation), the gradient feature is scipy's Sobel, the draws the Philox
generator the oracle's known-answer tests pin.  Every 5x4 frame of random
sequences, Philox and forced draws (including the conflict-making modes), with
and without spatial propagation: the masks and the whole model must be equal
after every frame.
"""
import numpy as np
import pytest
from scipy import ndimage

DX = (0, 1, 1, 1, 0, -1, -1, -1)   # N, NE, E, SE, S, SW, W, NW
DY = (-1, -1, 0, 1, 1, 1, 0, -1)
F = np.float32


def _depth_u8(d, fs):
    d = int(d)
    if d == 0:
        return 0
    return min(255, max(1, (d * 255 + fs // 2) // fs))


def _grad(img):
    a = img.astype(np.int32)
    gx = ndimage.sobel(a, axis=1, mode="nearest")
    gy = ndimage.sobel(a, axis=0, mode="nearest")
    return np.minimum(255, (np.abs(gx) + np.abs(gy)) >> 3).astype(np.int64)


class ScatterPBAS:
    """Per-channel PBAS, model arrays shaped like the oracle's."""

    def __init__(self, W, H, p):
        self.W, self.H, self.p = W, H, p
        P, N = W * H, p["N"]
        self.sv = np.zeros((P, 4, N), np.uint8)
        self.sg = np.zeros((P, 4, N), np.uint8)
        self.sD = np.zeros((P, 4, N), np.uint16)
        self.R = np.zeros((P, 4), np.float32)
        self.T = np.zeros((P, 4), np.float32)
        self.S = np.zeros((P, 4), np.uint32)
        self.gsum = np.zeros(4, np.uint64)
        self.t = 0

    def _draws(self, orc, i, c, prob):
        p, t, N = self.p, self.t, self.p["N"]
        if p["forced_rng"]:
            col, row = i % self.W, i // self.W
            k1, k2 = t % N, (t + 1) % N
            if p["forced_rng"] == 1:
                j = t % 8
            elif p["forced_rng"] == 2:
                j = 2 if ((col >> 1) & 1) == 0 else 6
            else:
                j = 0 if (col & 1) == 0 else 3
                if (row & 1) == 0:
                    k2 = k1
            return True, k1, True, j, k2
        u = orc.philox4x32_10([i, t, c, 0], [p["seed"], p["stream_id"]])[0]
        u = [int(x) for x in u]
        two24 = F(1.0 / 16777216.0)
        coin1 = F(u[0] >> 8) * two24 < prob
        coin2 = F(u[2] >> 8) * two24 < prob
        k1 = (u[1] * N) >> 32
        j = u[3] >> 29
        k2 = ((u[3] & 0x1FFFFFFF) * N) >> 29
        return bool(coin1), k1, bool(coin2), j, k2

    def step(self, orc, rgb, depth):
        W, H, p = self.W, self.H, self.p
        P, N = W * H, p["N"]
        ch = np.stack([rgb[..., 0], rgb[..., 1], rgb[..., 2],
                       np.vectorize(lambda d: _depth_u8(d, p["depth_full_scale_mm"]))(depth)]).astype(np.int64)
        gr = np.stack([_grad(ch[c]) for c in range(4)])
        ch, gr = ch.reshape(4, P), gr.reshape(4, P)
        valid = depth.reshape(P) != 0
        mask = np.zeros(P, np.uint8)
        if self.t == 0:
            for i in range(P):
                for c in range(4):
                    self.sv[i, c, :] = ch[c, i]
                    self.sg[i, c, :] = gr[c, i]
                    self.sD[i, c, :] = 0
                    self.R[i, c] = F(p["R_lower_rgb"] if c < 3 else p["R_lower_d"])
                    self.T[i, c] = F(p["T_lower"])
                    self.S[i, c] = 0
        else:
            wg = []
            for c in range(4):
                mean = F(int(self.gsum[c])) / F(P)
                wg.append(F(p["alpha_g"]) / max(mean, F(1.0)))
            snap_v, snap_g = self.sv.copy(), self.sg.copy()   # phase 1 reads the old model
            own = {}          # (i, c) -> slot of this frame's own update
            requests = []     # (requester i, channel c, direction j, slot k), raster order
            n16 = F(16 * N)
            for i in range(P):
                anyfg = False
                for c in range(4):
                    if c == 3 and not valid[i]:
                        continue
                    v, g = int(ch[c, i]), int(gr[c, i])
                    Rx, count, dmin = self.R[i, c], 0, F(np.inf)
                    for k in range(N):
                        dist = F(wg[c] * F(abs(g - int(snap_g[i, c, k])))) + F(abs(v - int(snap_v[i, c, k])))
                        count += int(dist < Rx)
                        dmin = min(dmin, dist)
                    fg = count < p["n_min"]
                    anyfg |= fg
                    Tx = self.T[i, c]
                    coin1, k1, coin2, j, k2 = self._draws(orc, i, c, F(1.0) / Tx)
                    if not fg and coin1:
                        self.sv[i, c, k1], self.sg[i, c, k1] = v, g
                        own[(i, c)] = k1
                        q16 = F(dmin * F(16.0))
                        q = 65535 if q16 >= F(65535.0) else int(np.rint(q16))
                        self.S[i, c] = np.uint32(int(self.S[i, c]) + q - int(self.sD[i, c, k1]))
                        self.sD[i, c, k1] = q
                    dbar = max(F(int(self.S[i, c])) / n16, F(p["eps_d"]))
                    Rs = F(dbar * F(p["R_scale"]))
                    Rx = F(Rx * F(1 - F(p["R_incdec"]))) if Rx > Rs else F(Rx * F(1 + F(p["R_incdec"])))
                    self.R[i, c] = max(Rx, F(p["R_lower_rgb"] if c < 3 else p["R_lower_d"]))
                    Tx = F(Tx + F(F(p["T_inc"]) / dbar)) if fg else F(Tx - F(F(p["T_dec"]) / dbar))
                    self.T[i, c] = min(max(Tx, F(p["T_lower"])), F(p["T_upper"]))
                    if not fg and coin2:
                        requests.append((i, c, j, k2))
                mask[i] = 255 if anyfg else 0
            # phase 2: scatter the requests in raster order; a later request only
            # replaces an earlier one for the same slot if it comes from a lower
            # direction index seen from the asked pixel
            best = {}  # (asked n, c, slot) -> (direction from n to the requester, value, gradient)
            for (i, c, j, k) in requests:
                x, y = i % W, i // W
                nx, ny = x + DX[j], y + DY[j]
                if not (0 <= nx < W and 0 <= ny < H):
                    continue
                n = ny * W + nx
                if p["propagate"]:
                    if own.get((n, c)) == k:
                        continue
                    jy = j ^ 4
                    if (n, c, k) not in best or jy < best[(n, c, k)][0]:
                        best[(n, c, k)] = (jy, int(ch[c, i]), int(gr[c, i]))
                else:
                    if c == 3 and not valid[n]:
                        continue
                    self.sv[n, c, k], self.sg[n, c, k] = ch[c, n], gr[c, n]
            for (n, c, k), (_, v, g) in best.items():
                self.sv[n, c, k], self.sg[n, c, k] = v, g
        for c in range(4):
            self.gsum[c] = int(gr[c].sum())
        self.t += 1
        return mask.reshape(H, W)


def _sequence(seed, W, H, n):
    """Random frames that stay close to a background, so that both
    foreground and background decisions (and hence updates) occur."""
    rng = np.random.default_rng(seed)
    bg = rng.integers(40, 215, size=(H, W, 3))
    dbg = rng.integers(500, 4000, size=(H, W))
    rgb, depth = [], []
    for t in range(n):
        f = bg + rng.integers(-4, 5, size=(H, W, 3))
        jump = rng.random((H, W)) < 0.25
        f[jump] += rng.integers(-80, 81, size=(int(jump.sum()), 3))
        d = dbg + rng.integers(-30, 31, size=(H, W))
        d[rng.random((H, W)) < 0.15] = 0
        rgb.append(np.clip(f, 0, 255).astype(np.uint8))
        depth.append(np.clip(d, 0, 65535).astype(np.uint16))
    return rgb, depth


@pytest.mark.parametrize("propagate", [0, 1])
@pytest.mark.parametrize("forced", [0, 1, 2, 3])
@pytest.mark.parametrize("seed", [0, 1])
def test_scatter_path_equals_oracle(orc, propagate, forced, seed):
    W, H, n = 5, 4, 8
    p = dict(orc.PBAS_DEFAULTS)
    p.update(N=5, propagate=propagate, forced_rng=forced, seed=11 + seed, stream_id=3)
    ref = orc.PBAS(W, H, **p)
    alt = ScatterPBAS(W, H, p)
    rgb, depth = _sequence(100 * forced + 10 * propagate + seed, W, H, n)
    fg = 0
    for t in range(n):
        m_ref = ref.step(rgb[t], depth[t])
        m_alt = alt.step(orc, rgb[t], depth[t])
        np.testing.assert_array_equal(m_alt, m_ref, err_msg=f"mask frame {t}")
        for name in ("sv", "sg", "sD", "R", "T", "S", "gsum"):
            np.testing.assert_array_equal(getattr(alt, name), getattr(ref, name), err_msg=f"{name} frame {t}")
        fg += int(m_ref.astype(bool).sum())
    assert fg > 0 and fg < W * H * (n - 1)
