"""Seeded synthetic images shaped like the paper's workloads.

The paper measures on one AI-generated n x n photograph that is not available; these images
stand in for it. This module holds no arithmetic of the seam-carving method: it only makes
uint8 H x W x 3 inputs, and it is the one module that both the CUDA path's tests/benchmark and
the oracle take their inputs from.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): the k-th output (k = 1, 2, ...) of a stream seeded with s is
mix(s + k * 0x9E3779B97F4A7C15 mod 2^64), so a run of outputs is computed as one vector.
u01 = (x >> 11) * 2^-53; randint(a, b) = a + floor(u01 * (b - a + 1)); Gaussian noise by the
Box-Muller transform in float64 with u1 = 1 - u01 so that log(u1) is finite.

Generator G(W, H, R, smin, smax, seed), in draw order:
  1. a linear colour gradient: colours A, B (three randint(0,255) each) and an angle
     theta = 2*pi*u01; t = projection of (x, y) on theta, scaled to [0, 1] over the image
     corners; base = A + (B - A) t;
  2. R axis-aligned solid rectangles drawn in order (later on top): w, h = randint(smin, smax),
     x0 = randint(0, W-1), y0 = randint(0, H-1), colour = three randint(0, 255); clipped;
  3. noise N(0, 8^2) per channel, rounded half-to-even and clamped to 0..255.
The libm behind log/cos/sin may differ in the last place between machines, so the same seed can
give a rare different byte on another machine; parity never depends on that, because the oracle
and the CUDA path take the same bytes in the same process.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class SplitMix64:
    """Counter form of splitmix64: outputs are drawn in blocks, in stream order."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & _MASK)
        self.count = 0

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(self.count + 1, self.count + 1 + n, dtype=np.uint64)
        self.count += n
        with np.errstate(over="ignore"):
            return _mix(self.seed + k * _GAMMA)

    def u01(self, n: int) -> np.ndarray:
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def randint(self, a: int, b: int, n: int) -> np.ndarray:
        return a + np.floor(self.u01(n) * (b - a + 1)).astype(np.int64)

    def one_randint(self, a: int, b: int) -> int:
        return int(self.randint(a, b, 1)[0])

    def one_u01(self) -> float:
        return float(self.u01(1)[0])


def uniform_image(W: int, H: int, seed: int) -> np.ndarray:
    """Every byte i.i.d. randint(0, 255), drawn in H x W x 3 row-major order."""
    rng = SplitMix64(seed)
    return rng.randint(0, 255, H * W * 3).astype(np.uint8).reshape(H, W, 3)


def gen_image(W: int, H: int, R: int, smin: int, smax: int, seed: int, sigma: float = 8.0) -> np.ndarray:
    """Generator G (module docstring): gradient + R rectangles + Gaussian noise, uint8 H x W x 3."""
    rng = SplitMix64(seed)
    A = rng.randint(0, 255, 3).astype(np.float64)
    B = rng.randint(0, 255, 3).astype(np.float64)
    theta = 2.0 * math.pi * rng.one_u01()
    c, s = math.cos(theta), math.sin(theta)
    corners = [0.0, (W - 1) * c, (H - 1) * s, (W - 1) * c + (H - 1) * s]
    pmin, pmax = min(corners), max(corners)
    xs = np.arange(W, dtype=np.float64) * c
    ys = np.arange(H, dtype=np.float64) * s
    p = ys[:, None] + xs[None, :]
    t = (p - pmin) / (pmax - pmin) if pmax > pmin else np.zeros_like(p)
    img = A[None, None, :] + (B - A)[None, None, :] * t[:, :, None]
    for _ in range(R):
        w = rng.one_randint(smin, smax)
        h = rng.one_randint(smin, smax)
        x0 = rng.one_randint(0, W - 1)
        y0 = rng.one_randint(0, H - 1)
        col = rng.randint(0, 255, 3).astype(np.float64)
        img[y0:min(H, y0 + h), x0:min(W, x0 + w), :] = col
    n = H * W * 3
    npairs = (n + 1) // 2
    u = rng.u01(2 * npairs)
    u1 = 1.0 - u[0::2]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * npairs, dtype=np.float64)
    z[0::2] = rad * np.cos(2.0 * math.pi * u2)
    z[1::2] = rad * np.sin(2.0 * math.pi * u2)
    img = img + sigma * z[:n].reshape(H, W, 3)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def _round_half_up(x: float) -> int:
    return int(math.floor(x + 0.5))


def scaled_rects(W: int, H: int) -> tuple[int, int, int]:
    """(R, smin, smax) for an image of W x H made with the 1920x1080 settings, scaled by area."""
    R = max(1, _round_half_up(40.0 * W * H / (1920.0 * 1080.0)))
    return R, 20, max(20, min(300, W, H))


@dataclass
class CarveJob:
    """One image and its targets. ``make()`` builds the pixels (uint8 H x W x 3)."""
    name: str
    W: int
    H: int
    target_w: int
    target_h: int
    make: Callable[[], np.ndarray] = field(repr=False)
    arrival_s: float = 0.0

    @property
    def seams(self) -> int:
        return (self.W - self.target_w) + (self.H - self.target_h)

    def mpix_seams(self) -> float:
        """Sum over removed seams of the pixel count of the image the seam was found in, / 1e6."""
        tot = 0
        for t in range(self.W - self.target_w):
            tot += self.H * (self.W - t)
        for t in range(self.H - self.target_h):
            tot += self.target_w * (self.H - t)
        return tot / 1e6


def config1() -> CarveJob:
    """64x48, bytes i.i.d. uniform from seed 1; 16 vertical seams."""
    return CarveJob("64x48 uniform, 16 vertical seams", 64, 48, 48, 48, lambda: uniform_image(64, 48, 1))


def config2() -> CarveJob:
    """1920x1080, G(40 rectangles, side 20..300, seed 2); 1920 -> 1440 (480 vertical seams)."""
    return CarveJob("1920x1080 -> 1440x1080 (480 vertical seams)", 1920, 1080, 1440, 1080,
                    lambda: gen_image(1920, 1080, 40, 20, 300, 2))


def config3() -> CarveJob:
    """3840x2160, G(120 rectangles, side 40..600, seed 3); 960 vertical then 540 horizontal."""
    return CarveJob("3840x2160 -> 2880x1620 (960 vertical + 540 horizontal seams)", 3840, 2160, 2880, 1620,
                    lambda: gen_image(3840, 2160, 120, 40, 600, 3))


def config4(n: int = 256, seed: int = 4) -> List[CarveJob]:
    """n images, W ~ randint(240,1280), H ~ randint(180,960), width reduced by r ~ U[0.10, 0.40]."""
    rng = SplitMix64(seed)
    jobs = []
    for k in range(n):
        W = rng.one_randint(240, 1280)
        H = rng.one_randint(180, 960)
        r = 0.10 + 0.30 * rng.one_u01()
        img_seed = int(rng.u64(1)[0])
        tw = W - int(math.floor(r * W))
        R, smin, smax = scaled_rects(W, H)
        jobs.append(CarveJob(f"batch[{k}] {W}x{H}->{tw}", W, H, tw, H,
                             (lambda W=W, H=H, R=R, smin=smin, smax=smax, s=img_seed:
                              gen_image(W, H, R, smin, smax, s))))
    return jobs


def config5(n: int = 10000, seed: int = 5, rate_hz: float = 200.0) -> List[CarveJob]:
    """n requests: Poisson arrivals at rate_hz, W, H log-uniform in [128, 4096] x [128, 2160],
    target width U[0.5, 0.9] W and height U[0.8, 1.0] H (floored, at least 1)."""
    rng = SplitMix64(seed)
    jobs = []
    t = 0.0
    lw0, lw1 = math.log(128.0), math.log(4096.0)
    lh0, lh1 = math.log(128.0), math.log(2160.0)
    for k in range(n):
        t += -math.log(1.0 - rng.one_u01()) / rate_hz
        W = _round_half_up(math.exp(lw0 + rng.one_u01() * (lw1 - lw0)))
        H = _round_half_up(math.exp(lh0 + rng.one_u01() * (lh1 - lh0)))
        tw = max(1, int(math.floor((0.5 + 0.4 * rng.one_u01()) * W)))
        th = max(1, int(math.floor((0.8 + 0.2 * rng.one_u01()) * H)))
        img_seed = int(rng.u64(1)[0])
        R, smin, smax = scaled_rects(W, H)
        jobs.append(CarveJob(f"request[{k}] {W}x{H}->{tw}x{th}", W, H, tw, th,
                             (lambda W=W, H=H, R=R, smin=smin, smax=smax, s=img_seed:
                              gen_image(W, H, R, smin, smax, s)), arrival_s=t))
    return jobs


def paper_square(n: int, seed: int = 6) -> CarveJob:
    """The paper's own workload shape: an n x n image carved to half its width (s = 0.5)."""
    R, smin, smax = scaled_rects(n, n)
    return CarveJob(f"{n}x{n} -> {n // 2}x{n}", n, n, n // 2, n, lambda: gen_image(n, n, R, smin, smax, seed + n))
