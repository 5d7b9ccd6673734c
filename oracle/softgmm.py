"""Soft (differentiable) GMM over RGB-D video: FP64 forward, adjoint by autograd.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The paper (Sec. 3.1, Eq. 1)
defines the hard per-pixel GMM; this soft form replaces its hard match test
by a sigmoid so the mask loss has gradients with respect to the learning
rate alpha, the squared match threshold L = lambda^2, the depth weight w and
the initial variance v0 (colour; the depth model uses v0 * 4/36).  Written
in plain PyTorch FP64 on the CPU, vectorised over pixels; the adjoint is
torch.autograd over that forward (a library primitive as a step).

Per model (colour C = 3, depth C = 1; depth skipped where the reading is
invalid), per pixel, frame t >= 1, temperature tau:
  d_k  = ||x - mu_k||^2 / (C v_k)
  m_k  = sigmoid((L - d_k) / tau)                 soft match
  r_k  = m_k * prod_{j<k} (1 - m_j),  q = prod_k (1 - m_k)
  w1_k = (1 - alpha) w_k + alpha r_k
  rho_k = alpha r_k / w1_k   (a never-used component, w_k = 0: rho_k = [r_k > 0])
  mu1_k = mu_k + rho_k (x - mu_k)
  v1_k = max(v_min, v_k + rho_k (||x - mu_k||^2 / C - v_k))
  last-ranked component blended toward the replacement with weight q:
  w2 = (1-q) w1 + q alpha, mu2 = (1-q) mu1 + q x, v2 = (1-q) v1 + q v_init
  w3 = w2 / sum(w2); re-rank by w3 / sqrt(v2) (stable)
Classification with the model before the update: B = shortest ranked prefix
with weight > T_bg, delta = d at the first arg-min over B; Q = (1-w) delta_rgb
+ w delta_d (depth valid) else delta_rgb; p = sigmoid((Q - L) / tau).
Loss = mean over pixels and frames 1..T-1 of BCE(p, gt).
The ranking permutation, B and the arg-min are taken from the forward values
and held constant for the gradient; v_min acts as a hard max.  Frame 0
initialises the model (component 0 = (1, x, v_init), the rest (0, 0, v_init)).
As tau -> 0 the forward equals the hard GMM (pinned in tests).
"""
from __future__ import annotations

import numpy as np
import torch

DEFAULTS = dict(K_rgb=3, K_d=3, tau=0.25, T_bg=0.7, v_min_rgb=4.0, v_min_d=0.25,
                depth_full_scale_mm=10000, v_init_d_ratio=4.0 / 36.0)


def depth_to_u8(depth: np.ndarray, fs: int = 10000) -> np.ndarray:
    """Sec. 4.2 rescale (same definition as the C oracle)."""
    d = depth.astype(np.int64)
    q = np.clip((d * 255 + fs // 2) // fs, 1, 255)
    return np.where(d == 0, 0, q).astype(np.uint8)


class _Model:
    """State of one mixture over P pixels: w (P,K), mu (P,K,C), v (P,K)."""

    def __init__(self, w, mu, v):
        self.w, self.mu, self.v = w, mu, v


def _init(x, K, v_init):
    P, C = x.shape
    w = torch.zeros(P, K, dtype=torch.float64)
    w[:, 0] = 1.0
    mu = torch.zeros(P, K, C, dtype=torch.float64)
    mu[:, 0, :] = x
    v = v_init * torch.ones(P, K, dtype=torch.float64)
    return _Model(w, mu, v)


def _classify(m: _Model, x, T_bg):
    """Distance of x to the background set of the model (pre-update)."""
    C = x.shape[1]
    s = ((x[:, None, :] - m.mu) ** 2).sum(-1)
    d = s / (C * m.v)
    with torch.no_grad():
        cum_before = torch.cumsum(m.w, dim=1) - m.w
        inB = cum_before <= T_bg
        dd = torch.where(inB, d, torch.full_like(d, float("inf")))
        kstar = torch.argmin(dd, dim=1)
    return d.gather(1, kstar[:, None])[:, 0], d, s


def _rho(w, w1, r, alpha):
    """rho = alpha r / w1.  A never-used component (w = 0) has w1 = alpha r, so
    rho is 1 whenever r > 0 (0 otherwise) and does not depend on theta; taking
    that branch explicitly keeps the quotient rule away from w1 -> 0."""
    unused = w == 0
    safe = torch.where(unused, torch.ones_like(w1), w1)
    return torch.where(unused, (r > 0).to(w1.dtype), alpha * r / safe)


def _step(m: _Model, x, d, s, alpha, L, tau, v_init, v_min):
    C = x.shape[1]
    K = m.w.shape[1]
    mk = torch.sigmoid((L - d) / tau)
    r = []
    P_run = torch.ones_like(mk[:, 0])
    for k in range(K):
        r.append(mk[:, k] * P_run)
        P_run = P_run * (1.0 - mk[:, k])
    r = torch.stack(r, dim=1)
    q = P_run
    w1 = (1.0 - alpha) * m.w + alpha * r
    rho = _rho(m.w, w1, r, alpha)
    e = x[:, None, :] - m.mu
    mu1 = m.mu + rho[:, :, None] * e
    u = m.v + rho * (s / C - m.v)
    v1 = torch.clamp_min(u, v_min)
    last = torch.zeros(K, dtype=torch.float64)
    last[K - 1] = 1.0
    qq = q[:, None] * last[None, :]
    w2 = (1.0 - qq) * w1 + qq * alpha
    mu2 = (1.0 - qq[:, :, None]) * mu1 + qq[:, :, None] * x[:, None, :]
    v2 = (1.0 - qq) * v1 + qq * v_init
    w3 = w2 / w2.sum(dim=1, keepdim=True)
    with torch.no_grad():
        key = w3 / torch.sqrt(v2)
        perm = torch.sort(key, dim=1, descending=True, stable=True).indices
    return _Model(w3.gather(1, perm), mu2.gather(1, perm[:, :, None].expand(-1, -1, C)),
                  v2.gather(1, perm))


def _where(valid, new: _Model, old: _Model):
    vv = valid[:, None]
    return _Model(torch.where(vv, new.w, old.w), torch.where(vv[:, :, None], new.mu, old.mu),
                  torch.where(vv, new.v, old.v))


def forward(rgb, depth, gt, alpha, L, w, v0, **kw):
    """Loss of one or more sequences.

    rgb (B,T,H,W,3) u8, depth (B,T,H,W) u16, gt (B,T,H,W) u8 (nonzero = fg);
    alpha, L, w, v0: FP64 scalar tensors (may require grad).
    Returns (loss, final models, per-frame soft masks (B,T-1,H*W)).
    """
    o = dict(DEFAULTS)
    o.update(kw)
    Bn, T = rgb.shape[:2]
    P = rgb.shape[2] * rgb.shape[3]
    tau, T_bg = o["tau"], o["T_bg"]
    v_init_d = v0 * o["v_init_d_ratio"]
    total = torch.zeros((), dtype=torch.float64)
    probs = []
    finals = []
    for b in range(Bn):
        xs = torch.from_numpy(rgb[b].reshape(T, P, 3).astype(np.float64))
        d8 = depth_to_u8(depth[b], o["depth_full_scale_mm"]).reshape(T, P)
        xd = torch.from_numpy(d8.astype(np.float64))[:, :, None]
        valid = torch.from_numpy(d8 != 0)
        y = torch.from_numpy((gt[b].reshape(T, P) != 0).astype(np.float64))
        mr = _init(xs[0], o["K_rgb"], v0)
        md = _init(xd[0], o["K_d"], v_init_d)
        pb = []
        for t in range(1, T):
            dB_r, d_r, s_r = _classify(mr, xs[t], T_bg)
            dB_d, d_d, s_d = _classify(md, xd[t], T_bg)
            Q = torch.where(valid[t], (1.0 - w) * dB_r + w * dB_d, dB_r)
            a = (Q - L) / tau
            total = total + (torch.nn.functional.softplus(a) - y[t] * a).sum()
            pb.append(torch.sigmoid(a))
            mr = _step(mr, xs[t], d_r, s_r, alpha, L, tau, v0, o["v_min_rgb"])
            md = _where(valid[t], _step(md, xd[t], d_d, s_d, alpha, L, tau, v_init_d, o["v_min_d"]), md)
        probs.append(torch.stack(pb) if pb else torch.zeros(0, P, dtype=torch.float64))
        finals.append((mr, md))
    loss = total / (Bn * (T - 1) * P)
    return loss, finals, torch.stack(probs)


def loss_and_grad(rgb, depth, gt, theta, **kw):
    """theta = (alpha, L, w, v0) floats -> (loss, dloss/dtheta as a float64 array)."""
    th = [torch.tensor(float(v), dtype=torch.float64, requires_grad=True) for v in theta]
    loss, _, _ = forward(rgb, depth, gt, *th, **kw)
    g = torch.autograd.grad(loss, th)
    return float(loss.detach()), np.array([float(x) for x in g])


def fingerprint(rgb, depth, gt, theta, **kw):
    """Every hard decision of a forward run (ranks, background sets, arg-mins,
    v_min clamps), to check that finite-difference points share them."""
    o = dict(DEFAULTS)
    o.update(kw)
    Bn, T = rgb.shape[:2]
    P = rgb.shape[2] * rgb.shape[3]
    alpha, L, w, v0 = (torch.tensor(float(v), dtype=torch.float64) for v in theta)
    out = []
    for b in range(Bn):
        xs = torch.from_numpy(rgb[b].reshape(T, P, 3).astype(np.float64))
        d8 = depth_to_u8(depth[b], o["depth_full_scale_mm"]).reshape(T, P)
        xd = torch.from_numpy(d8.astype(np.float64))[:, :, None]
        valid = torch.from_numpy(d8 != 0)
        mr = _init(xs[0], o["K_rgb"], v0)
        md = _init(xd[0], o["K_d"], v0 * o["v_init_d_ratio"])
        for t in range(1, T):
            for m, x, vmin, vi, isd in ((mr, xs[t], o["v_min_rgb"], v0, False),
                                        (md, xd[t], o["v_min_d"], v0 * o["v_init_d_ratio"], True)):
                cum_before = torch.cumsum(m.w, 1) - m.w
                inB = cum_before <= o["T_bg"]
                s = ((x[:, None, :] - m.mu) ** 2).sum(-1)
                d = s / (x.shape[1] * m.v)
                dd = torch.where(inB, d, torch.full_like(d, float("inf")))
                out += [inB.numpy().tobytes(), torch.argmin(dd, 1).numpy().tobytes()]
                mk = torch.sigmoid((L - d) / o["tau"])
                rr, Pr = [], torch.ones(P, dtype=torch.float64)
                for k in range(m.w.shape[1]):
                    rr.append(mk[:, k] * Pr)
                    Pr = Pr * (1 - mk[:, k])
                r = torch.stack(rr, 1)
                w1 = (1 - alpha) * m.w + alpha * r
                rho = _rho(m.w, w1, r, alpha)
                u = m.v + rho * (s / x.shape[1] - m.v)
                if isd:
                    out.append((valid[t][:, None] & (u > vmin)).numpy().tobytes())
                else:
                    out.append((u > vmin).numpy().tobytes())
            dB_r, d_r, s_r = _classify(mr, xs[t], o["T_bg"])
            dB_d, d_d, s_d = _classify(md, xd[t], o["T_bg"])
            mr2 = _step(mr, xs[t], d_r, s_r, alpha, L, o["tau"], v0, o["v_min_rgb"])
            md2 = _step(md, xd[t], d_d, s_d, alpha, L, o["tau"], v0 * o["v_init_d_ratio"], o["v_min_d"])
            key = mr2.w / torch.sqrt(mr2.v)
            out.append(torch.sort(key, dim=1, descending=True, stable=True).indices.numpy().tobytes())
            mr, md = mr2, _where(valid[t], md2, md)
    return hash(tuple(out))


def decision_margins(rgb, depth, gt, theta, w_sig=1e-6, **kw):
    """Per pixel (B, P): the smallest relative distance of any consequential
    hard decision of the forward run from its threshold (background-set prefix
    sums vs T_bg, arg-min over the background set, ranking comparisons and
    v_min floors of components with weight >= w_sig), for excluding near-tie
    pixels when comparing with a lower-precision implementation.  Decisions
    among components of negligible weight (soft-match ghosts) change the loss
    only in proportion to that weight and are not counted."""
    o = dict(DEFAULTS)
    o.update(kw)
    Bn, T = rgb.shape[:2]
    P = rgb.shape[2] * rgb.shape[3]
    alpha, L, w, v0 = (torch.tensor(float(v), dtype=torch.float64) for v in theta)
    out = np.full((Bn, P), np.inf)

    def rel(a, b):
        # exact ties (identical untouched components) resolve the same way in
        # any precision: not a near-tie
        den = torch.maximum(torch.maximum(a.abs(), b.abs()), torch.full_like(a, 1e-300))
        r = ((a - b).abs() / den).numpy()
        return np.where((a == b).numpy(), np.inf, r)

    def upd(b, mask, r_):
        out[b] = np.where(mask, np.minimum(out[b], r_), out[b])

    for b in range(Bn):
        xs = torch.from_numpy(rgb[b].reshape(T, P, 3).astype(np.float64))
        d8 = depth_to_u8(depth[b], o["depth_full_scale_mm"]).reshape(T, P)
        xd = torch.from_numpy(d8.astype(np.float64))[:, :, None]
        valid = torch.from_numpy(d8 != 0)
        mr = _init(xs[0], o["K_rgb"], v0)
        md = _init(xd[0], o["K_d"], v0 * o["v_init_d_ratio"])
        for t in range(1, T):
            for m, x, vmin, vi, msk in ((mr, xs[t], o["v_min_rgb"], v0, torch.ones(P, dtype=torch.bool)),
                                        (md, xd[t], o["v_min_d"], v0 * o["v_init_d_ratio"], valid[t])):
                K = m.w.shape[1]
                mk_np = msk.numpy()
                sig = (m.w >= w_sig).numpy()
                cum = torch.cumsum(m.w, 1)
                for k in range(K - 1):
                    upd(b, mk_np, rel(cum[:, k], torch.full_like(cum[:, k], o["T_bg"])))
                s = ((x[:, None, :] - m.mu) ** 2).sum(-1)
                d = s / (x.shape[1] * m.v)
                inB = ((cum - m.w) <= o["T_bg"]).numpy()
                for i in range(K):
                    for j in range(i + 1, K):
                        upd(b, mk_np & inB[:, i] & inB[:, j], rel(d[:, i], d[:, j]))
                mkk = torch.sigmoid((L - d) / o["tau"])
                rr, Pr = [], torch.ones(P, dtype=torch.float64)
                for k in range(K):
                    rr.append(mkk[:, k] * Pr)
                    Pr = Pr * (1 - mkk[:, k])
                r = torch.stack(rr, 1)
                w1 = (1 - alpha) * m.w + alpha * r
                rho = _rho(m.w, w1, r, alpha)
                u = m.v + rho * (s / x.shape[1] - m.v)
                for k in range(K):
                    # a component already at the floor moves by rho * (...) only;
                    # either branch changes the loss by terms proportional to rho
                    at_floor = (m.v[:, k] == vmin).numpy()
                    upd(b, mk_np & sig[:, k] & ~at_floor, rel(u[:, k], torch.full_like(u[:, k], vmin)))
                nm = _step(m, x, d, s, alpha, L, o["tau"], vi, vmin)
                key = nm.w / torch.sqrt(nm.v)
                nsig = (nm.w >= w_sig).numpy()
                for i in range(K):
                    for j in range(i + 1, K):
                        upd(b, mk_np & (nsig[:, i] | nsig[:, j]), rel(key[:, i], key[:, j]))
            dB_r, d_r, s_r = _classify(mr, xs[t], o["T_bg"])
            dB_d, d_d, s_d = _classify(md, xd[t], o["T_bg"])
            mr2 = _step(mr, xs[t], d_r, s_r, alpha, L, o["tau"], v0, o["v_min_rgb"])
            md2 = _step(md, xd[t], d_d, s_d, alpha, L, o["tau"], v0 * o["v_init_d_ratio"], o["v_min_d"])
            mr, md = mr2, _where(valid[t], md2, md)
    return out


def pixel_grads(rgb, depth, gt, theta, pixels, **kw):
    """d loss / d theta restricted to the listed (sequence, pixel) pairs, each
    pixel run alone (pixels are independent), normalised as in the full loss."""
    Bn, T, H, W = rgb.shape[:4]
    P = H * W
    out = []
    for b, p in pixels:
        y, x = divmod(int(p), W)
        _, g = loss_and_grad(rgb[b:b + 1, :, y:y + 1, x:x + 1], depth[b:b + 1, :, y:y + 1, x:x + 1],
                             gt[b:b + 1, :, y:y + 1, x:x + 1], theta, **kw)
        out.append(g / (Bn * P))
    return np.array(out)
