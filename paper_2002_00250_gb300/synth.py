"""Seeded synthetic RGB-D video (inputs only; none of the method's arithmetic).

Stands in for the paper's RealSense recordings and the SBM-RGBD sequences
(Sec. 5), which are not available here.  The scenes take the paper's
resolutions (Sec. 4.3: 480p, 720p, 1080p) and its difficulty categories
(Sec. 5: illumination changes, colour camouflage, shadows, invalid depth):

* background colour: smooth texture (three low-frequency sinusoids per
  channel) plus an 8x8 checker of +/-20, clipped to 40..215;
* per-frame per-pixel Gaussian colour noise, sigma 3, rounded and clamped;
* background depth: per-pixel uniform 500..4000 mm, fixed over time, with
  per-frame noise of 1 % of the depth and 2 % of pixels set to 0 (invalid);
* moving ellipses (semi-axes 30..80 px at 640 wide, scaled with the width),
  2..6 px/frame with wall bounce, colour +40 or -40, depth 300 mm in front
  of the background;
* optional colour-camouflage ellipses (colour within +/-5 of the
  background, depth 400 mm in front), a global illumination gain of 0.6
  ramping to 1.2 over frames 100..200, and cast shadows (each object's
  ellipse shifted by (+25, +15) px, colour x0.5, depth unchanged, not in the
  ground truth).

The generator runs on any torch device.  CPU and CUDA torch random streams
differ, so a test that compares two implementations generates its frames
once and gives the same arrays to both.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch


@dataclass
class SceneConfig:
    width: int
    height: int
    n_frames: int
    seed: int = 0
    stream_id: int = 0
    n_objects: int = 3
    n_camouflage: int = 0
    illumination_ramp: bool = False
    shadows: bool = False
    hole_fraction: float = 0.02
    name: str = field(default="scene")


def config_480p(seed: int = 0) -> SceneConfig:
    """640x480, 50 frames, three moving ellipses (static background)."""
    return SceneConfig(640, 480, 50, seed=seed, name="640x480x50")


def config_720p(seed: int = 0) -> SceneConfig:
    """1280x720, 300 frames, plus camouflage, illumination ramp and shadows."""
    return SceneConfig(1280, 720, 300, seed=seed, n_camouflage=2, illumination_ramp=True,
                       shadows=True, name="1280x720x300")


def config_stream(width: int, height: int, n_frames: int, seed: int, stream_id: int) -> SceneConfig:
    """One camera stream of a multi-stream batch: 480p-style content at any size."""
    return SceneConfig(width, height, n_frames, seed=seed, stream_id=stream_id,
                       name=f"{width}x{height}x{n_frames}/s{stream_id}")


BATCH16_SIZES = ([(424, 240)] * 4 + [(640, 480)] * 4 + [(848, 480)] * 4 +
                 [(1280, 720)] * 3 + [(1920, 1080)])


class RGBDScene:
    """Deterministic synthetic RGB-D sequence for one SceneConfig."""

    def __init__(self, cfg: SceneConfig, device="cpu"):
        self.cfg = cfg
        self.device = torch.device(device)
        W, H = cfg.width, cfg.height
        rs = np.random.default_rng([cfg.seed, cfg.stream_id, 0x5CE7E])
        scale = W / 640.0

        # background colour texture
        ys = torch.arange(H, device=self.device, dtype=torch.float32).view(H, 1)
        xs = torch.arange(W, device=self.device, dtype=torch.float32).view(1, W)
        bg = torch.empty((H, W, 3), device=self.device, dtype=torch.float32)
        for c in range(3):
            acc = torch.full((H, W), 127.5, device=self.device)
            for _ in range(3):
                fx, fy = rs.uniform(0.3, 2.5, size=2)
                ph = rs.uniform(0, 2 * math.pi)
                amp = rs.uniform(10, 22)
                acc = acc + amp * torch.sin(2 * math.pi * (fx * xs / W + fy * ys / H) + ph)
            bg[..., c] = acc
        checker = (((xs // 8) + (ys // 8)) % 2) * 40.0 - 20.0
        self.bg_rgb = (bg + checker.unsqueeze(-1)).clamp(40.0, 215.0)

        # background depth, fixed per pixel
        g0 = torch.Generator(device=self.device)
        g0.manual_seed(self._seed_for(-1))
        self.bg_depth = 500.0 + 3500.0 * torch.rand((H, W), generator=g0, device=self.device)

        # moving objects: centre, velocity, semi-axes, colour offset, depth offset
        objs = []
        for i in range(cfg.n_objects + cfg.n_camouflage):
            camo = i >= cfg.n_objects
            a, b = rs.uniform(30, 80, size=2) * scale
            cx, cy = rs.uniform(0.15, 0.85) * W, rs.uniform(0.15, 0.85) * H
            speed = rs.uniform(2, 6) * scale
            ang = rs.uniform(0, 2 * math.pi)
            if camo:
                dc = rs.uniform(-5, 5, size=3)
                dz = -400.0
            else:
                dc = np.full(3, 40.0 if rs.uniform() < 0.5 else -40.0)
                dz = -300.0
            objs.append(dict(a=a, b=b, cx=cx, cy=cy, vx=speed * math.cos(ang),
                             vy=speed * math.sin(ang), dc=dc, dz=dz))
        self.objects = objs
        self._ys, self._xs = ys, xs

    def _seed_for(self, t: int) -> int:
        c = self.cfg
        return (c.seed * 1_000_003 + c.stream_id * 7_919 + (t + 1) * 104_729) & 0x7FFFFFFFFFFF

    def _centre(self, o, t: int):
        """Position at frame t with reflection at the frame borders."""
        W, H = self.cfg.width, self.cfg.height

        def bounce(p0, v, L):
            x = p0 + v * t
            period = 2.0 * L
            x = math.fmod(x, period)
            if x < 0:
                x += period
            return x if x < L else period - x

        return bounce(o["cx"], o["vx"], W), bounce(o["cy"], o["vy"], H)

    def gain(self, t: int) -> float:
        if not self.cfg.illumination_ramp:
            return 1.0
        if t < 100:
            return 0.6
        if t < 200:
            return 0.6 + 0.6 * (t - 100) / 100.0
        return 1.2

    def frame(self, t: int):
        """Frame t: (rgb u8 (H,W,3), depth u16 (H,W), gt u8 (H,W) 0/255)."""
        cfg = self.cfg
        H, W = cfg.height, cfg.width
        dev = self.device
        g = torch.Generator(device=dev)
        g.manual_seed(self._seed_for(t))
        rgb = self.bg_rgb.clone()
        depth = self.bg_depth.clone()
        gt = torch.zeros((H, W), dtype=torch.bool, device=dev)
        scale = W / 640.0
        if cfg.shadows:
            for o in self.objects:
                cx, cy = self._centre(o, t)
                sh = (((self._xs - cx - 25 * scale) / o["a"]) ** 2 +
                      ((self._ys - cy - 15 * scale) / o["b"]) ** 2) <= 1.0
                rgb = torch.where(sh.unsqueeze(-1), rgb * 0.5, rgb)
        for o in self.objects:
            cx, cy = self._centre(o, t)
            inside = (((self._xs - cx) / o["a"]) ** 2 + ((self._ys - cy) / o["b"]) ** 2) <= 1.0
            dc = torch.tensor(o["dc"], dtype=torch.float32, device=dev)
            rgb = torch.where(inside.unsqueeze(-1), self.bg_rgb + dc, rgb)
            depth = torch.where(inside, self.bg_depth + o["dz"], depth)
            gt |= inside
        rgb = rgb * self.gain(t)
        rgb = rgb + 3.0 * torch.randn((H, W, 3), generator=g, device=dev)
        rgb = torch.round(rgb).clamp(0, 255).to(torch.uint8)
        depth = depth + 0.01 * depth * torch.randn((H, W), generator=g, device=dev)
        depth = torch.round(depth).clamp(1, 65535)
        holes = torch.rand((H, W), generator=g, device=dev) < cfg.hole_fraction
        depth = torch.where(holes, torch.zeros_like(depth), depth)
        depth = depth.to(torch.int32).to(torch.uint16) if hasattr(torch, "uint16") else depth
        return rgb, depth, (gt.to(torch.uint8) * 255)

    def sequence(self, t0: int = 0, n: int | None = None):
        """Frames t0..t0+n-1 stacked: rgb (n,H,W,3) u8, depth (n,H,W) u16, gt (n,H,W) u8."""
        n = self.cfg.n_frames - t0 if n is None else n
        H, W = self.cfg.height, self.cfg.width
        rgb = torch.empty((n, H, W, 3), dtype=torch.uint8, device=self.device)
        depth = torch.empty((n, H, W), dtype=torch.uint16, device=self.device)
        gt = torch.empty((n, H, W), dtype=torch.uint8, device=self.device)
        for i in range(n):
            r, d, g = self.frame(t0 + i)
            rgb[i], depth[i], gt[i] = r, d, g
        return rgb, depth, gt


def to_numpy(x: torch.Tensor) -> np.ndarray:
    """Host copy as numpy (uint16 tensors go through int32 where torch lacks the cast)."""
    x = x.detach().cpu()
    if x.dtype == torch.uint16:
        return x.to(torch.int32).numpy().astype(np.uint16)
    return x.numpy()
