"""The colour oracle (opponent transform, readings C1-C4) against what the
mathematics fixes: properties of the transform, the noise scale of each
channel measured on samples, the sigma = 0 identity, and the achromatic case,
which must reduce exactly to the (separately pinned) grayscale oracle."""
import numpy as np

from paper_2103_10765_gb300 import synth


def test_opp_properties(orc):
    rng = np.random.default_rng(3)
    x = rng.random((3, 17, 19))
    y = orc.opp(x)
    # invertible: the inverse transform restores the input
    np.testing.assert_allclose(orc.opp(y, inverse=True), x, atol=1e-14)
    # luma is the mean of R, G, B
    np.testing.assert_allclose(y[0], x.mean(axis=0), atol=1e-15)
    # achromatic pixels (R = G = B) have no chroma
    g = np.repeat(rng.random((1, 9, 9)), 3, axis=0)
    yg = orc.opp(g)
    assert np.abs(yg[1:]).max() == 0.0
    np.testing.assert_allclose(yg[0], g[0], atol=1e-15)
    # rows are orthogonal: transforming the basis gives F with F F^T diagonal
    F = np.stack([orc.opp(np.eye(3)[:, k].reshape(3, 1, 1))[:, 0, 0] for k in range(3)], axis=1)
    FFt = F @ F.T
    np.testing.assert_allclose(FFt - np.diag(np.diag(FFt)), 0, atol=1e-15)
    for c in range(3):
        assert abs(orc.opp_sigma_scale(c) - np.sqrt(FFt[c, c])) < 1e-15


def test_opp_noise_scale_measured(orc):
    # i.i.d. N(0, 1) in R, G, B -> channel deviations equal the scales (C2)
    n = synth.normals(77, 3 * 1_000_000).reshape(3, 1000, 1000)
    y = orc.opp(n)
    for c in range(3):
        assert abs(y[c].std() / orc.opp_sigma_scale(c) - 1) < 0.005
    # and the channels are uncorrelated
    assert abs(np.corrcoef(y.reshape(3, -1))[0, 1]) < 0.005


def test_color_sigma_zero_identity(orc):
    clean, _ = synth.make_color_pair(40, 48, 0.0, 4)
    out = orc.denoise_color(clean, 0.0, orc.Params(), nthreads=4)
    np.testing.assert_allclose(out, clean.astype(np.float64), atol=1e-12)


def test_color_achromatic_reduces_to_gray(orc):
    # R = G = B = z (one noisy gray image): U = V = 0 stay 0, and Y = z is
    # denoised exactly as the grayscale method with sigma / sqrt(3)
    _, z = synth.make_pair(48, 56, 25 / 255, 5)
    Z = np.repeat(z[None].astype(np.float64), 3, axis=0)
    out = orc.denoise_color(Z, 25 / 255, orc.Params(), nthreads=4)
    y = orc.opp(Z)[0]
    ref = orc.denoise(y, 25 / 255 * orc.opp_sigma_scale(0), orc.Params(), nthreads=4)
    for c in range(3):
        np.testing.assert_allclose(out[c], ref, atol=1e-12)


def test_color_denoises_every_channel(orc):
    clean, noisy = synth.make_color_pair(64, 64, 25 / 255, 2)
    out = orc.denoise_color(noisy, 25 / 255, orc.Params(), nthreads=4)
    for c in range(3):
        assert orc.psnr(out[c], clean[c]) > orc.psnr(noisy[c], clean[c]) + 5
