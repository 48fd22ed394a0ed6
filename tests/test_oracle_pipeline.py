"""Pins for the oracle's two-stage pipeline (Sec. 1.1 BM3D1/BM3D2, Sec. 3.1
eq. firstEst, Sec. 4; Table "PSNR": the second stage improves the first on
every test image)."""
import numpy as np
import pytest

from paper_2103_10765_gb300 import synth


def test_sigma_zero_is_identity(orc):
    _, Z = synth.make_pair(40, 48, 0.0, 1)
    out, y1 = orc.denoise(Z, 0.0, nthreads=4, return_y1=True)
    np.testing.assert_allclose(y1, Z, atol=1e-12)
    np.testing.assert_allclose(out, Z, atol=1e-12)


def test_constant_image_closed_form(orc):
    """A constant image c: stage 1 keeps it (only the coarsest approximation is
    nonzero); stage 2 keeps only the group DC coefficient P = c N sqrt(K), shrunk
    by omega = P^2 / (P^2 + sigma^2), so Y2 = c omega everywhere."""
    c, sigma = 0.6, 25 / 255
    Z = synth.constant_image(32, 40, c)
    out, y1 = orc.denoise(Z, sigma, nthreads=4, return_y1=True)
    np.testing.assert_allclose(y1, c, atol=1e-12)
    P = c * 8 * np.sqrt(32)
    np.testing.assert_allclose(out, c * P ** 2 / (P ** 2 + sigma ** 2), atol=1e-12)


@pytest.mark.parametrize("sigma", [15, 25, 50])
def test_psnr_monotone(orc, sigma):
    for seed in (1, 2):
        clean, Z = synth.make_pair(96, 96, sigma / 255, seed)
        out, y1 = orc.denoise(Z, sigma / 255, nthreads=8, return_y1=True)
        p0, p1, p2 = orc.psnr(Z, clean), orc.psnr(y1, clean), orc.psnr(out, clean)
        assert p0 < p1 < p2, (sigma, seed, p0, p1, p2)


def test_stage1_only(orc):
    clean, Z = synth.make_pair(48, 48, 0.1, 1)
    p = orc.Params(stages=1)
    out, y1 = orc.denoise(Z, 0.1, params=p, nthreads=4, return_y1=True)
    np.testing.assert_array_equal(out, y1)


def test_translations_average_shifted_runs(orc):
    """eq. firstEst with T = 2: the mean of phi(Z) and S_{-2} phi(S_2 Z)."""
    _, Z = synth.make_pair(40, 40, 0.1, 2)
    p1 = orc.Params(stages=1, translations=1)
    p2 = orc.Params(stages=1, translations=2)
    y_a = orc.denoise(Z, 0.1, params=p1, nthreads=4)
    y_b = np.roll(orc.denoise(np.roll(Z, (2, 2), (0, 1)), 0.1, params=p1, nthreads=4), (-2, -2), (0, 1))
    np.testing.assert_allclose(orc.denoise(Z, 0.1, params=p2, nthreads=4), 0.5 * (y_a + y_b), atol=1e-13)


def test_paper_preset_sigma_zero_and_constant(orc):
    """Sec. 5 parameters (N = 16 tiling blocks in stage 1, N = 8 in stage 2,
    K = 16, T = 2): sigma = 0 returns Z; a constant image c comes back from
    stage 1 unchanged and from stage 2 as c P^2 / (P^2 + sigma^2) with the
    group DC coefficient P = c N2 sqrt(K2) = c 8 sqrt(16)."""
    p = orc.Params.paper()
    _, Z = synth.make_pair(48, 64, 0.0, 1)
    out, y1 = orc.denoise(Z, 0.0, params=p, nthreads=4, return_y1=True)
    np.testing.assert_allclose(y1, Z, atol=1e-12)
    np.testing.assert_allclose(out, Z, atol=1e-12)
    c, sigma = 0.45, 25 / 255
    out, y1 = orc.denoise(synth.constant_image(48, 40, c), sigma, params=p, nthreads=4, return_y1=True)
    np.testing.assert_allclose(y1, c, atol=1e-12)
    P = c * 8 * np.sqrt(16)
    np.testing.assert_allclose(out, c * P ** 2 / (P ** 2 + sigma ** 2), atol=1e-12)


def test_paper_preset_translations_use_each_stage_block_side(orc):
    """eq. firstEst with T = 2 under the Sec. 5 parameters: stage 1 averages
    phi(Z) and S_{-4} phi(S_4 Z) (h = N1/4 = 4); stage 2, built here from the
    oracle's match / Wiener / aggregation steps, averages the runs at h = 0
    and h = N2/4 = 2 on the shifted noisy image and stage-1 estimate."""
    p = orc.Params.paper()
    sigma = 25 / 255
    _, Z = synth.make_pair(48, 56, sigma, 3)
    out, y1 = orc.denoise(Z, sigma, params=p, nthreads=8, return_y1=True)
    p1 = orc.Params.paper()
    p1.stages, p1.translations = 1, 1
    ya = orc.denoise(Z, sigma, params=p1, nthreads=8)
    yb = np.roll(orc.denoise(np.roll(Z, (4, 4), (0, 1)), sigma, params=p1, nthreads=8), (-4, -4), (0, 1))
    np.testing.assert_allclose(y1, 0.5 * (ya + yb), atol=1e-13)
    H, W = Z.shape
    y2 = np.zeros((H, W))
    for h in (0, 2):
        zs, ys = np.roll(Z.astype(np.float64), (h, h), (0, 1)), np.roll(y1, (h, h), (0, 1))
        idx, _ = orc.match(ys, N=8, s=8, R=16, K=16, nthreads=8)
        groups, w = orc.filter_wiener(zs, ys, idx, sigma, N=8, K=16, nthreads=8)
        y2 += 0.5 * np.roll(orc.aggregate(groups, w, idx, H, W, N=8, beta=2.0), (-h, -h), (0, 1))
    np.testing.assert_allclose(out, y2, atol=1e-13)


def test_paper_preset_psnr_monotone(orc):
    """Table PSNR: stage 2 improves stage 1, which improves the noisy input."""
    p = orc.Params.paper()
    for sigma in (15, 50):
        clean, Z = synth.make_pair(128, 128, sigma / 255, 2)
        out, y1 = orc.denoise(Z, sigma / 255, params=p, nthreads=8, return_y1=True)
        p0, p1, p2 = orc.psnr(Z, clean), orc.psnr(y1, clean), orc.psnr(out, clean)
        assert p0 < p1 < p2, (sigma, p0, p1, p2)
