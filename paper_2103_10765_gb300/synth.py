"""Seeded synthetic test images for G-BM3D (shared by the CUDA path's tests,
the benchmark and the CPU oracle's tests).

This module holds no arithmetic of the denoising method itself: it only draws
random numbers and paints piecewise-constant scenes plus noise.

The paper measures on natural photographs (Sec. 5, Table "PSNR"), which are
not available here.  These scenes stand in for them: piecewise-constant
rectangles and disks (edges and flat regions, where block matching finds many
similar blocks), a linear gradient and band-limited sinusoidal texture, clamped
to [0, 1], plus additive white Gaussian noise of standard deviation sigma
(Sec. 5: i.i.d. zero-mean Gaussian noise).

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): doubles in [0, 1) from the top
53 bits, normals by the Box-Muller transform.  Everything is vectorised in
numpy; ``splitmix64_scalar`` is an independent scalar restatement used by the
tests.
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1

N_RECTS = 24
N_DISKS = 16
N_SINES = 3
SINE_AMPLITUDE = 0.04


def splitmix64_scalar(seed: int, count: int) -> list[int]:
    """Plain-Python SplitMix64: the first ``count`` outputs for ``seed``."""
    state = seed & _MASK
    out = []
    for _ in range(count):
        state = (state + _GAMMA) & _MASK
        z = state
        z = ((z ^ (z >> 30)) * _M1) & _MASK
        z = ((z ^ (z >> 27)) * _M2) & _MASK
        out.append(z ^ (z >> 31))
    return out


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Vectorised SplitMix64 outputs ``start .. start+count-1`` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK) + i * np.uint64(_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        return z ^ (z >> np.uint64(31))


def uniforms(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normals(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on consecutive uniform pairs."""
    npairs = (count + 1) // 2
    u = uniforms(seed, 2 * npairs)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))  # log(1 - u1), u1 < 1 so finite
    t = 2.0 * math.pi * u2
    out = np.empty(2 * npairs, dtype=np.float64)
    out[0::2] = r * np.cos(t)
    out[1::2] = r * np.sin(t)
    return out[:count]


class _Stream:
    """Sequential uniform draws from one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = seed
        self.pos = 0

    def u(self, lo: float = 0.0, hi: float = 1.0) -> float:
        v = float(uniforms(self.seed, 1, self.pos)[0])
        self.pos += 1
        return lo + (hi - lo) * v


def clean_scene(H: int, W: int, seed: int) -> np.ndarray:
    """Piecewise-constant scene with gradient and sinusoidal texture, float32 in [0,1]."""
    if H <= 0 or W <= 0:
        return np.zeros((max(H, 0), max(W, 0)), dtype=np.float32)
    rs = _Stream(seed)
    m = float(min(H, W))
    y = np.arange(H, dtype=np.float64)[:, None]
    x = np.arange(W, dtype=np.float64)[None, :]
    img = np.full((H, W), rs.u(), dtype=np.float64)
    for _ in range(N_RECTS):
        cy, cx = rs.u(0, H), rs.u(0, W)
        hh, ww = rs.u(0.03, 0.30) * m, rs.u(0.03, 0.30) * m
        val = rs.u()
        mask = (np.abs(y - cy) <= 0.5 * hh) & (np.abs(x - cx) <= 0.5 * ww)
        img = np.where(mask, val, img)
    for _ in range(N_DISKS):
        cy, cx = rs.u(0, H), rs.u(0, W)
        rad = rs.u(0.02, 0.15) * m
        val = rs.u()
        mask = (y - cy) ** 2 + (x - cx) ** 2 <= rad * rad
        img = np.where(mask, val, img)
    gy, gx = rs.u(-0.2, 0.2), rs.u(-0.2, 0.2)
    img = img + gy * (y / H - 0.5) + gx * (x / W - 0.5)
    for _ in range(N_SINES):
        f = rs.u(0.02, 0.12)
        th = rs.u(0.0, math.pi)
        ph = rs.u(0.0, 2.0 * math.pi)
        img = img + SINE_AMPLITUDE * np.sin(2.0 * math.pi * f * (x * math.cos(th) + y * math.sin(th)) + ph)
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def add_noise(clean: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """clean + sigma * N(0,1), rounded to float32, not clipped."""
    n = normals(seed, clean.size).reshape(clean.shape)
    return (clean.astype(np.float64) + sigma * n).astype(np.float32)


def make_pair(H: int, W: int, sigma: float, scene_seed: int = 1):
    """(clean, noisy) float32 images; the noise seed is 1000 + scene_seed."""
    clean = clean_scene(H, W, scene_seed)
    return clean, add_noise(clean, sigma, 1000 + scene_seed)


def make_color_pair(H: int, W: int, sigma: float, scene_seed: int = 1):
    """(clean, noisy) float32 RGB images of shape (3, H, W): two independent
    scenes A (seed s) and B (seed s + 50) give R = A, G = (A + B) / 2, B = B,
    so the channels are correlated as in natural images; noise is i.i.d. per
    channel with seeds 1000 + s, 2000 + s, 3000 + s."""
    a = clean_scene(H, W, scene_seed).astype(np.float64)
    b = clean_scene(H, W, scene_seed + 50).astype(np.float64)
    clean = np.stack([a, 0.5 * (a + b), b]).astype(np.float32)
    noisy = np.stack([add_noise(clean[c], sigma, 1000 * (c + 1) + scene_seed) for c in range(3)])
    return clean, noisy


def constant_image(H: int, W: int, value: float = 0.5) -> np.ndarray:
    return np.full((H, W), value, dtype=np.float32)


def degrade_blur(clean: np.ndarray, psf: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """Deconvolution input: the clean image circularly convolved with the
    point-spread function psf (odd side, centred), plus white Gaussian noise of
    deviation sigma from the noise seed; float32, not clipped.  This is the
    degradation that produces test inputs, not a step of the restoration."""
    x = clean.astype(np.float64)
    r = psf.shape[0] // 2
    y = np.zeros_like(x)
    for a in range(-r, r + 1):
        for b in range(-r, r + 1):
            y += psf[a + r, b + r] * np.roll(x, (a, b), axis=(0, 1))
    return (y + sigma * normals(seed, x.size).reshape(x.shape)).astype(np.float32)


def gaussian_psf(size: int = 9, std: float = 1.6) -> np.ndarray:
    """The k x k normalised Gaussian blur of the deconvolution workload (outer
    product of a sampled 1-D Gaussian, summing to 1)."""
    t = np.arange(size, dtype=np.float64) - size // 2
    g = np.exp(-0.5 * (t / std) ** 2)
    g /= g.sum()
    return np.outer(g, g)


def pnp_batch_specs(n: int = 64, seed: int = 7, lo: int = 128, hi: int = 1024):
    """Sizes and noise levels of a batch of deconvolution problems: per image
    H and W uniform over the multiples of 8 in [lo, hi] and sigma uniform in
    [5, 50] / 255, all drawn from one SplitMix64 stream.  Returns a list of
    (H, W, sigma, scene_seed)."""
    u = uniforms(seed, 3 * n)
    steps = (hi - lo) // 8 + 1
    out = []
    for i in range(n):
        H = lo + 8 * min(int(u[3 * i] * steps), steps - 1)
        W = lo + 8 * min(int(u[3 * i + 1] * steps), steps - 1)
        sigma = (5.0 + 45.0 * float(u[3 * i + 2])) / 255.0
        out.append((H, W, sigma, 100 + i))
    return out


def make_blur_pair(H: int, W: int, sigma: float, scene_seed: int = 1, psf_size: int = 9, psf_std: float = 1.6):
    """(clean, blurred + noisy) float32 images for deconvolution; the noise
    seed is 5000 + scene_seed."""
    clean = clean_scene(H, W, scene_seed)
    return clean, degrade_blur(clean, gaussian_psf(psf_size, psf_std), sigma, 5000 + scene_seed)


def he_normal_params(seed: int, shapes) -> np.ndarray:
    """Starting parameters of a network: for each (fan_in, fan_out) in shapes,
    fan_in * fan_out weights N(0, 2 / fan_in) followed by fan_out zero biases,
    concatenated; the normals come from one SplitMix64 stream."""
    n = sum(fi * fo + fo for fi, fo in shapes)
    z = normals(seed, n)
    out = np.zeros(n)
    o = 0
    for fi, fo in shapes:
        out[o:o + fi * fo] = z[o:o + fi * fo] * math.sqrt(2.0 / fi)
        o += fi * fo + fo
    return out


def pilot_training_specs(n: int = 125, seed: int = 21, size: int = 1024):
    """(H, W, sigma, scene_seed) of the learned pilot's training scenes:
    n scenes of size x size (the scale of the images it serves; training cuts
    them into crops), sigma uniform in [5, 50] / 255."""
    u = uniforms(seed, n)
    return [(size, size, (5.0 + 45.0 * float(u[i])) / 255.0, 10000 + i) for i in range(n)]
