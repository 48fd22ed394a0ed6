"""Plug-and-play ADMM deconvolution with G-BM3D as the denoiser -- FP64 oracle.

TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
benchmark's CPU legs, never by the CUDA library or its binding.  It shares
no code with the CUDA path.

The paper motivates its speed-up with plug-and-play priors (Sec. 1: coupling
a denoiser with inverse problems such as deconvolution, one denoiser call per
iteration; Sec. 6: real-time plug-and-play use).  It does not state the
iteration, so this file restates the standard plug-and-play ADMM from the
works Sec. 1 cites, with these readings:

  P1  degradation y = h * x + n: circular 2-D convolution with a normalised
      k x k Gaussian point-spread function h (std s; 9 x 9, s = 1.6 here),
      white Gaussian noise of deviation sigma_n.
  P2  splitting of 1/2 ||H x - y||^2 + lambda R(x) with x = v, scaled dual u,
      fixed penalty rho:
          x <- argmin_x 1/2 ||H x - y||^2 + rho/2 ||x - (v - u)||^2
             = (H^T H + rho I)^-1 (H^T y + rho (v - u))
          v <- D(x + u; sigma_d)
          u <- u + x - v
  P3  lambda = sigma_n^2 (the MAP weight of the data term), so the denoiser
      runs at sigma_d = sqrt(lambda / rho) = sigma_n / sqrt(rho).
  P4  start v = y, u = 0; the result is v after the last iteration.
  P5  the x-update is solved exactly: H^T H + rho I is circulant, hence
      diagonal in the 2-D DFT (numpy's FFT is used as that library step).
  P6  D is the two-stage G-BM3D of this oracle (orc_denoise) with the given
      parameters.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class PnpParams:
    """Iteration count and penalty of the ADMM loop (readings P2, P3)."""
    iters: int = 50
    rho: float = 0.1
    psf_size: int = 9
    psf_std: float = 1.6


def gaussian_psf(size: int = 9, std: float = 1.6) -> np.ndarray:
    """Normalised size x size Gaussian point-spread function (reading P1):
    h[a, b] = g(a) g(b) / (sum g)^2, g(t) = exp(-t^2 / (2 std^2)), t = -r..r."""
    r = size // 2
    t = np.arange(-r, r + 1, dtype=np.float64)
    g = np.exp(-t ** 2 / (2.0 * std ** 2))
    return np.outer(g, g) / g.sum() ** 2


def blur(x, h) -> np.ndarray:
    """Circular convolution (reading P1): out[i, j] = sum_{a,b} h[a+r, b+r]
    x[(i - a) mod H, (j - b) mod W], written as the definition."""
    x = np.asarray(x, dtype=np.float64)
    r = h.shape[0] // 2
    out = np.zeros_like(x)
    for a in range(-r, r + 1):
        for b in range(-r, r + 1):
            out += h[a + r, b + r] * np.roll(x, (a, b), axis=(0, 1))
    return out


def blur_adjoint(x, h) -> np.ndarray:
    """H^T: circular correlation with h (equal to blur for a symmetric h)."""
    return blur(x, h[::-1, ::-1])


def _otf(h, H, W) -> np.ndarray:
    """DFT of h placed circularly with its centre at (0, 0)."""
    r = h.shape[0] // 2
    pad = np.zeros((H, W))
    for a in range(-r, r + 1):
        for b in range(-r, r + 1):
            pad[a % H, b % W] += h[a + r, b + r]
    return np.fft.fft2(pad)


def x_update(b, h, rho: float) -> np.ndarray:
    """Solve (H^T H + rho I) x = b exactly (reading P5): the circulant
    operator is diagonal in the 2-D DFT with eigenvalues |DFT(h)|^2 + rho."""
    b = np.asarray(b, dtype=np.float64)
    F = _otf(h, *b.shape)
    return np.real(np.fft.ifft2(np.fft.fft2(b) / (np.abs(F) ** 2 + rho)))


def pnp_admm(y, sigma_n: float, q: PnpParams | None = None, params=None, nthreads: int = 1, denoiser=None):
    """Plug-and-play ADMM deconvolution of y (readings P1-P6).  denoiser(img,
    sigma) defaults to the oracle's two-stage G-BM3D with `params`."""
    import oracle as orc
    q = q or PnpParams()
    h = gaussian_psf(q.psf_size, q.psf_std)
    y = np.asarray(y, dtype=np.float64)
    if denoiser is None:
        def denoiser(img, s):
            return orc.denoise(img, s, params=params, nthreads=nthreads)
    sigma_d = sigma_n / np.sqrt(q.rho)
    hty = blur_adjoint(y, h)
    v, u = y.copy(), np.zeros_like(y)
    for _ in range(q.iters):
        x = x_update(hty + q.rho * (v - u), h, q.rho)
        v = denoiser(x + u, sigma_d)
        u = u + x - v
    return v
