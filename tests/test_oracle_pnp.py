"""Pins for the plug-and-play ADMM deconvolution oracle (oracle/pnp.py;
readings P1-P6 in its header), each against something other than itself."""
import numpy as np
import pytest

from paper_2103_10765_gb300 import synth

scipy_ndimage = pytest.importorskip("scipy.ndimage")


@pytest.fixture(scope="module")
def pnp():
    from oracle import pnp as m
    return m


def test_psf_definition(pnp):
    h = pnp.gaussian_psf(9, 1.6)
    assert h.shape == (9, 9) and abs(h.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(h, h.T, atol=0)
    np.testing.assert_allclose(h, h[::-1, ::-1], atol=0)
    # separable: rank one, centre / edge ratio of a Gaussian of std 1.6
    assert np.linalg.matrix_rank(h, tol=1e-14) == 1
    np.testing.assert_allclose(h[4, 4] / h[4, 0], np.exp(16 / (2 * 1.6 ** 2)), rtol=1e-12)
    # the input generator's own definition of the same blur
    np.testing.assert_allclose(synth.gaussian_psf(9, 1.6), h, rtol=1e-13, atol=1e-17)


def test_blur_is_circular_convolution(pnp, rng):
    x = rng.random((23, 31))
    h = pnp.gaussian_psf(9, 1.6)
    np.testing.assert_allclose(pnp.blur(x, h), scipy_ndimage.convolve(x, h, mode="wrap"), atol=1e-14)
    # the generator's degradation is the same operator (sigma = 0)
    np.testing.assert_allclose(synth.degrade_blur(x.astype(np.float32), h, 0.0, 1),
                               pnp.blur(x.astype(np.float32), h), atol=1e-6)


def test_blur_adjoint_identity(pnp, rng):
    """<H x, z> = <x, H^T z> for a non-symmetric kernel."""
    x, z = rng.random((17, 20)), rng.random((17, 20))
    h = rng.random((5, 5))
    assert abs(np.vdot(pnp.blur(x, h), z) - np.vdot(x, pnp.blur_adjoint(z, h))) < 1e-11


@pytest.mark.parametrize("rho", [0.01, 0.1, 1.0])
def test_x_update_solves_normal_equations(pnp, rng, rho):
    """(H^T H + rho I) x = b checked with the spatial-domain operator, not the DFT."""
    b = rng.random((40, 36))
    h = pnp.gaussian_psf(9, 1.6)
    x = pnp.x_update(b, h, rho)
    r = pnp.blur_adjoint(pnp.blur(x, h), h) + rho * x - b
    assert np.abs(r).max() < 1e-11


def test_x_update_delta_psf(pnp, rng):
    b = rng.random((16, 24))
    delta = np.zeros((9, 9))
    delta[4, 4] = 1.0
    np.testing.assert_allclose(pnp.x_update(b, delta, 0.3), b / 1.3, atol=1e-14)


def test_admm_with_identity_denoiser_matches_dense_solve(pnp, rng):
    """With D = identity the loop is x_{k+1} = (H^T H + rho I)^-1 (H^T y + rho x_k)
    (u stays 0, v = x): checked against a dense circulant matrix solve."""
    Hh, Ww, rho, iters = 10, 12, 0.2, 4
    y = rng.random((Hh, Ww))
    h = pnp.gaussian_psf(5, 1.1)
    n = Hh * Ww
    M = np.zeros((n, n))
    for i in range(Hh):
        for j in range(Ww):
            for a in range(-2, 3):
                for b in range(-2, 3):
                    M[i * Ww + j, ((i - a) % Hh) * Ww + (j - b) % Ww] += h[a + 2, b + 2]
    A = M.T @ M + rho * np.eye(n)
    x = y.ravel().copy()
    for _ in range(iters):
        x = np.linalg.solve(A, M.T @ y.ravel() + rho * x)
    q = pnp.PnpParams(iters=iters, rho=rho, psf_size=5, psf_std=1.1)
    v = pnp.pnp_admm(y, 0.1, q, denoiser=lambda img, s: img)
    np.testing.assert_allclose(v.ravel(), x, atol=1e-12)


def test_denoiser_strength_and_call_count(pnp, rng):
    """Reading P3: one denoiser call per iteration at sigma_n / sqrt(rho)."""
    seen = []
    y = rng.random((16, 16))
    pnp.pnp_admm(y, 0.08, pnp.PnpParams(iters=3, rho=0.25), denoiser=lambda img, s: (seen.append(s), img)[1])
    assert seen == pytest.approx([0.16] * 3, rel=1e-15)


def test_admm_improves_on_the_blurred_input(pnp, orc):
    sigma = 25 / 255
    clean, y = synth.make_blur_pair(64, 64, sigma, 3)
    v = pnp.pnp_admm(y, sigma, pnp.PnpParams(iters=4), nthreads=8)
    assert orc.psnr(v, clean) > orc.psnr(y, clean) + 2.0


def test_batch_specs():
    s = synth.pnp_batch_specs()
    assert len(s) == 64 and s == synth.pnp_batch_specs()
    for H, W, sigma, seed in s:
        assert H % 8 == 0 and W % 8 == 0 and 128 <= H <= 1024 and 128 <= W <= 1024
        assert 5 / 255 <= sigma <= 50 / 255
    assert len({(H, W) for H, W, _, _ in s}) > 50


def test_batch_specs_small_end():
    # the small-image batch of the benchmark (sides 128..256): same noise levels
    # and scene seeds as the full batch, sides drawn from the narrower range
    s = synth.pnp_batch_specs(hi=256)
    full = synth.pnp_batch_specs()
    assert len(s) == 64
    for (H, W, sigma, seed), (_, _, sigma_f, seed_f) in zip(s, full):
        assert H % 8 == 0 and W % 8 == 0 and 128 <= H <= 256 and 128 <= W <= 256
        assert sigma == sigma_f and seed == seed_f
    assert len({H for H, _, _, _ in s}) > 10
