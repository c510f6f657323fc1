"""Seeded synthetic exposure stacks.

This module makes INPUTS only: a smooth random scene, exposures of it at several
gains, and integer displacements.  It holds none of the alignment arithmetic
(no gray conversion, pyramid, median, bitmap or search), so the CUDA path and
the oracle can both be fed from it without sharing any of the method.

Scene recipe (per pixel, float, then clipped to [0, 255]):
  80 + 40 Gaussian blobs (centres uniform over the frame, sigma uniform in
  [0.01, 0.15] * min(W, H), amplitude U(-60, 60), per-channel tint U(0.7, 1.3))
  + 3 sinusoids (amplitude 10, period U(8, 64) px, random orientation and phase)
  + N(0, 2) noise.
The base level 80 keeps the median of a 2x brighter linear exposure below
saturation (with 128 more than half of such an exposure clips to 255, and its
median threshold bitmap is empty).  The blobs and sinusoids are separable, so the smooth part is one rank-46
product per channel.  Parameters come from numpy's PCG64 seeded with ``seed``;
the per-pixel noise comes from a torch generator on the target device seeded
with ``seed``, so a given (seed, device) always gives the same bytes.

An exposure at gain g is clip(round(255 * (g * (s / 255) ** gamma) ** (1 / gamma)
+ N(0, sensor_sigma))), or clip(round(g * s)) when gamma is None.  A displacement
(dx, dy) moves the content right by dx and down by dy with edge pixels replicated,
so the shift that re-aligns that exposure to an undisplaced one is (-dx, -dy).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch


@dataclass(frozen=True)
class StackSpec:
    """One exposure stack: geometry, exposures, planted shifts and search settings."""

    name: str
    seed: int
    w: int
    h: int
    n: int
    gains: Tuple[float, ...]
    gamma: Optional[float]
    sensor_sigma: float
    shift_range: int
    levels: int
    noise_tol: int
    ref: int
    fixed_shifts: Optional[Tuple[Tuple[int, int], ...]] = None

    @property
    def pairs(self) -> int:
        return self.n - 1

    @property
    def aligned_pixels(self) -> int:
        """Full-resolution pixels over all aligned pairs (the MPix/s numerator)."""
        return self.pairs * self.w * self.h

    @property
    def input_bytes(self) -> int:
        return self.n * self.w * self.h * 3


# 640x480 pair: exposure 1 = 2x brighter, content displaced by (+7, -3).
PAIR_640 = StackSpec("pair640x480", 0, 640, 480, 2, (1.0, 2.0), None, 0.0, 0, 6, 4, 0,
                     fixed_shifts=((0, 0), (7, -3)))
# 4000x3000 stack of 3, gains {0.5, 1, 2}, gamma 2.2, shifts U[-60, 60], 7 levels, ref = middle.
STACK_12MP = StackSpec("stack4000x3000x3", 1, 4000, 3000, 3, (0.5, 1.0, 2.0), 2.2, 0.0, 60, 7, 4, 1)
# 6000x4000 stack of 7, gains 2^-3..2^3, gamma 2.2, N(0,3) sensor noise, shifts U[-120, 120], 8 levels, ref = 3.
STACK_24MP = StackSpec("stack6000x4000x7", 2, 6000, 4000, 7, tuple(2.0 ** k for k in range(-3, 4)), 2.2, 3.0,
                       120, 8, 4, 3)

PLAIN_CONFIGS = (PAIR_640, STACK_12MP, STACK_24MP)


def planted_shifts(spec: StackSpec) -> np.ndarray:
    """[n, 2] int displacement (dx, dy) of each exposure's content; the ref row is 0."""
    if spec.fixed_shifts is not None:
        return np.asarray(spec.fixed_shifts, dtype=np.int64)
    rng = np.random.default_rng([spec.seed, 7])
    d = rng.integers(-spec.shift_range, spec.shift_range + 1, size=(spec.n, 2))
    d[spec.ref] = 0
    return d.astype(np.int64)


def expected_shifts(spec: StackSpec) -> np.ndarray:
    """Shift that re-aligns each exposure to the reference: minus its displacement."""
    d = planted_shifts(spec)
    return -(d - d[spec.ref])


def scene(seed: int, w: int, h: int, device="cpu", n_blobs: int = 40, noise_sigma: float = 2.0,
          base: float = 80.0, n_rects: int = 150) -> torch.Tensor:
    """[h, w, 3] float32 scene in [0, 255]."""
    rng = np.random.default_rng(seed)
    m = float(min(w, h))
    cx = rng.uniform(0, w, n_blobs)
    cy = rng.uniform(0, h, n_blobs)
    sig = rng.uniform(0.01, 0.15, n_blobs) * m
    amp = rng.uniform(-60.0, 60.0, n_blobs)
    tint = rng.uniform(0.7, 1.3, (n_blobs, 3))
    period = rng.uniform(8.0, 64.0, 3)
    theta = rng.uniform(0.0, math.pi, 3)
    phase = rng.uniform(0.0, 2 * math.pi, 3)

    dev = torch.device(device)
    xs = torch.arange(w, dtype=torch.float64, device=dev)
    ys = torch.arange(h, dtype=torch.float64, device=dev)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)
    gx = torch.exp(-((xs[:, None] - t(cx)[None, :]) ** 2) / (2 * t(sig)[None, :] ** 2))
    gy = torch.exp(-((ys[:, None] - t(cy)[None, :]) ** 2) / (2 * t(sig)[None, :] ** 2))
    # sin(a x + b y + p) = sin(a x + p) cos(b y) + cos(a x + p) sin(b y)
    a = t(2 * math.pi * np.cos(theta) / period)
    b = t(2 * math.pi * np.sin(theta) / period)
    sx = torch.sin(xs[:, None] * a[None, :] + t(phase)[None, :])
    cxs = torch.cos(xs[:, None] * a[None, :] + t(phase)[None, :])
    cyb = torch.cos(ys[:, None] * b[None, :])
    syb = torch.sin(ys[:, None] * b[None, :])
    # hard-edged rectangles: indicator(x0 <= x < x1) * indicator(y0 <= y < y1)
    rw = np.exp(rng.uniform(np.log(0.01), np.log(0.25), n_rects)) * m
    rh = np.exp(rng.uniform(np.log(0.01), np.log(0.25), n_rects)) * m
    rx = rng.uniform(-0.1 * w, w, n_rects)
    ry = rng.uniform(-0.1 * h, h, n_rects)
    ramp = rng.uniform(-40.0, 40.0, n_rects)
    rtint = rng.uniform(0.8, 1.2, (n_rects, 3))
    ix = ((xs[:, None] >= t(rx)[None, :]) & (xs[:, None] < t(rx + rw)[None, :])).double()
    iy = ((ys[:, None] >= t(ry)[None, :]) & (ys[:, None] < t(ry + rh)[None, :])).double()
    fx = torch.cat([gx, sx, cxs, ix], dim=1).float()  # [w, 46 + n_rects]
    fy = torch.cat([gy, cyb, syb, iy], dim=1).float()  # [h, 46 + n_rects]
    chans = []
    for c in range(3):
        coef = torch.cat([t(amp * tint[:, c]), t(np.full(6, 10.0)), t(ramp * rtint[:, c])]).float()
        chans.append(base + (fy * coef[None, :]) @ fx.T)
    s = torch.stack(chans, dim=-1)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    if noise_sigma > 0:
        s += noise_sigma * torch.randn(s.shape, generator=gen, device=dev, dtype=torch.float32)
    return s.clamp_(0.0, 255.0)


def displace(img: torch.Tensor, dx: int, dy: int) -> torch.Tensor:
    """Move content right by dx and down by dy; edge pixels replicated."""
    h, w = img.shape[:2]
    dev = img.device
    xi = (torch.arange(w, device=dev) - int(dx)).clamp_(0, w - 1)
    yi = (torch.arange(h, device=dev) - int(dy)).clamp_(0, h - 1)
    return img.index_select(0, yi).index_select(1, xi)


def expose(s: torch.Tensor, gain: float, gamma: Optional[float], sensor_sigma: float = 0.0,
           gen: Optional[torch.Generator] = None) -> torch.Tensor:
    """uint8 exposure of a [0, 255] float scene at the given gain."""
    if gamma is None:
        v = s * float(gain)
    else:
        v = 255.0 * (float(gain) * (s / 255.0) ** gamma) ** (1.0 / gamma)
    if sensor_sigma > 0:
        v = v + sensor_sigma * torch.randn(v.shape, generator=gen, device=v.device, dtype=v.dtype)
    return v.round_().clamp_(0.0, 255.0).to(torch.uint8)


def make_stack(spec: StackSpec, device="cpu") -> torch.Tensor:
    """[n, h, w, 3] uint8 exposure stack of ``spec`` on ``device``."""
    dev = torch.device(device)
    s = scene(spec.seed, spec.w, spec.h, dev)
    d = planted_shifts(spec)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(spec.seed) + 1)
    out = torch.empty((spec.n, spec.h, spec.w, 3), dtype=torch.uint8, device=dev)
    for e in range(spec.n):
        moved = displace(s, int(d[e, 0]), int(d[e, 1])) if (d[e, 0] or d[e, 1]) else s
        out[e] = expose(moved, spec.gains[e], spec.gamma, spec.sensor_sigma, gen)
        del moved
    return out


def batch_specs(count: int = 256, seed: int = 3) -> List[StackSpec]:
    """Uneven stacks for the batched form: pixel count log-uniform in
    [640*480, 6000*4000], aspect from {4:3, 3:2, 16:9}, 3..9 exposures at gains
    2^(k - n//2) with gamma 2.2, ref = n//2, levels = ceil(log2(max_shift)) with
    max_shift = max(8, floor(0.03 * min(W, H))), shifts within +-(2^levels - 1)."""
    rng = np.random.default_rng(seed)
    aspects = (4.0 / 3.0, 3.0 / 2.0, 16.0 / 9.0)
    out = []
    for j in range(count):
        p = math.exp(rng.uniform(math.log(640 * 480), math.log(6000 * 4000)))
        a = aspects[int(rng.integers(0, 3))]
        w = int(round(math.sqrt(p * a)))
        h = int(round(w / a))
        n = int(rng.integers(3, 10))
        max_shift = max(8, int(0.03 * min(w, h)))
        levels = int(math.ceil(math.log2(max_shift)))
        gains = tuple(2.0 ** (k - n // 2) for k in range(n))
        out.append(StackSpec(f"batch{j}", 1000 + j, w, h, n, gains, 2.2, 0.0, (1 << levels) - 1,
                             levels, 4, n // 2))
    return out


def serve_specs(count: int = 32) -> List[StackSpec]:
    """Serving jobs: the 6000x4000x7 stack's shape and exposures with fresh seeds."""
    base = STACK_24MP
    return [StackSpec(f"job{k}", 5000 + k, base.w, base.h, base.n, base.gains, base.gamma,
                      base.sensor_sigma, base.shift_range, base.levels, base.noise_tol, base.ref)
            for k in range(count)]


def paper_specs() -> List[StackSpec]:
    """The paper's measurement shape (Sec. IV): 2560x1440 (3.7 MP) exposures,
    stacks of 2 to 7, 6 pyramid levels; gains 2^(k - n//2) with gamma 2.2 and
    N(0, 1) sensor noise, handheld-size displacements within +-24 px, ref the
    middle exposure."""
    out = []
    for n in range(2, 8):
        gains = tuple(2.0 ** (k - n // 2) for k in range(n))
        out.append(StackSpec(f"paper2560x1440x{n}", 7000 + n, 2560, 1440, n, gains, 2.2, 1.0, 24, 6, 4, n // 2))
    return out


def small_spec(seed: int, w: int, h: int, n: int = 2, levels: int = 3, shift_range: int = 5,
               noise_tol: int = 4, ref: int = 0, gamma: Optional[float] = 2.2) -> StackSpec:
    """Small stacks for tests: gains 2^(k - ref)."""
    gains = tuple(2.0 ** ((k - ref) * 0.5) for k in range(n))
    return StackSpec(f"small{seed}_{w}x{h}x{n}", seed, w, h, n, gains, gamma, 0.0, shift_range, levels,
                     noise_tol, ref)
