"""Colour G-BM3D on the GPU (gbm3d_denoise_color) against the colour oracle
(readings C1-C4): end-to-end PSNR within 0.01 dB per channel, the
achromatic case bit-equal to the grayscale path, sigma = 0, pitched planes,
and the 2048 x 2048 x 3 configuration end to end."""
import math

import numpy as np
import pytest

from paper_2103_10765_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2103_10765_gb300 import gbm3d  # noqa: E402

DEV = torch.device("cuda:0")


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def psnr(x, ref):
    return 10 * math.log10(1.0 / float(np.mean((np.asarray(x, np.float64) - np.asarray(ref, np.float64)) ** 2)))


@pytest.mark.parametrize("H,W,sigma,seed", [(64, 72, 25, 1), (96, 80, 15, 2), (80, 64, 50, 3)])
def test_color_psnr_parity(orc, H, W, sigma, seed):
    clean, noisy = synth.make_color_pair(H, W, sigma / 255, seed)
    out = gbm3d.denoise_color(gpu(noisy), sigma / 255).cpu().numpy()
    ref = orc.denoise_color(noisy, sigma / 255, orc.Params(), nthreads=8)
    for c in range(3):
        assert abs(psnr(out[c], clean[c]) - psnr(ref[c], clean[c])) < 0.01, c
        assert psnr(out[c], clean[c]) > psnr(noisy[c], clean[c]) + 3


def test_color_achromatic_equals_gray_path():
    # R = G = B: the chroma planes are exactly zero and stay zero, so every
    # output channel equals the grayscale path on the same luma plane
    _, z = synth.make_pair(96, 104, 25 / 255, 4)
    Z = np.repeat(z[None], 3, axis=0)
    out = gbm3d.denoise_color(gpu(Z), 25 / 255).cpu().numpy()
    y = ((Z[0] + Z[1]) + Z[2]) * np.float32(1.0 / 3.0)  # the kernel's luma, same FP32 operations
    s_y = float(np.float32(float(np.float32(25 / 255)) * math.sqrt(1.0 / 3.0)))
    ref = gbm3d.denoise(gpu(y), s_y).cpu().numpy()
    for c in range(3):
        np.testing.assert_array_equal(out[c], ref)


def test_color_sigma_zero():
    clean, _ = synth.make_color_pair(56, 64, 0.0, 5)
    out = gbm3d.denoise_color(gpu(clean), 0.0).cpu().numpy()
    np.testing.assert_allclose(out, clean, atol=2e-6)


def test_color_pitched_planes():
    clean, noisy = synth.make_color_pair(64, 80, 25 / 255, 6)
    big = torch.zeros((3, 70, 96), device=DEV)
    big[:, 3:67, 5:85] = gpu(noisy)
    view = big[:, 3:67, 5:85]  # row pitch 96, plane stride 70 x 96
    a = gbm3d.denoise_color(view, 25 / 255).cpu().numpy()
    b = gbm3d.denoise_color(gpu(noisy), 25 / 255).cpu().numpy()
    np.testing.assert_array_equal(a, b)


def test_color_2048_runs():
    # the 2048 x 2048 x 3 configuration end to end
    clean, noisy = synth.make_color_pair(2048, 2048, 25 / 255, 7)
    out = gbm3d.denoise_color(gpu(noisy), 25 / 255).cpu().numpy()
    assert np.isfinite(out).all()
    for c in range(3):
        assert psnr(out[c], clean[c]) > psnr(noisy[c], clean[c]) + 8
