"""Pins for the learned-pilot oracle (oracle/pilot.py, readings L1-L5): the
convolution against scipy's correlation, the backward pass against central
finite differences of the forward pass, adjoint identities, and special
cases with closed forms."""
import numpy as np
import pytest

scipy_signal = pytest.importorskip("scipy.signal")


@pytest.fixture(scope="module")
def pl():
    from oracle import pilot
    return pilot


def test_param_count(pl):
    assert pl.param_count() == (9 * 2 * 32 + 32) + 14 * (9 * 32 * 32 + 32) + (9 * 32 + 1) == 130369


def test_conv_is_zero_padded_correlation(pl, rng):
    x = rng.standard_normal((2, 7, 9, 3))
    w = rng.standard_normal((9, 3, 4))
    b = rng.standard_normal(4)
    out = pl.conv(x, w, b)
    for n in range(2):
        for co in range(4):
            ref = np.full((7, 9), b[co])
            for ci in range(3):
                k = w[:, ci, co].reshape(3, 3)  # k[dy+1][dx+1]
                ref += scipy_signal.correlate2d(x[n, :, :, ci], k, mode="same", boundary="fill")
            np.testing.assert_allclose(out[n, :, :, co], ref, atol=1e-12)


def test_input_grad_is_adjoint(pl, rng):
    x = rng.standard_normal((1, 6, 5, 3))
    g = rng.standard_normal((1, 6, 5, 4))
    w = rng.standard_normal((9, 3, 4))
    lhs = np.vdot(pl.conv(x, w, np.zeros(4)), g)
    assert abs(lhs - np.vdot(x, pl.conv_input_grad(g, w, x.shape))) < 1e-10


def test_gradient_matches_finite_differences(pl, rng):
    theta = pl.init_params(5) + 0.01 * rng.standard_normal(pl.param_count())
    Z = rng.random((2, 6, 7))
    sig = np.array([0.1, 0.3])
    Y1 = Z + 0.05 * rng.standard_normal(Z.shape)
    L, grad = pl.loss_and_grad(theta, Z, sig, Y1)
    assert abs(L - pl.loss(theta, Z, sig, Y1)) < 1e-15
    # a sample of parameters from every layer, weights and biases
    offs, o = [], 0
    for ci, co, _ in pl.LAYERS:
        offs += [o, o + 9 * ci * co // 2, o + 9 * ci * co - 1, o + 9 * ci * co, o + 9 * ci * co + co - 1]
        o += 9 * ci * co + co
    h = 1e-6
    for i in offs:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (pl.loss(tp, Z, sig, Y1) - pl.loss(tm, Z, sig, Y1)) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_zero_last_layer_returns_the_noisy_image(pl, rng):
    theta = pl.init_params(3)
    n8 = 9 * 32 + 1
    theta[-n8:] = 0.0
    Z = rng.random((1, 5, 8))
    np.testing.assert_array_equal(pl.forward(theta, Z, [0.2]), Z)


def test_init_is_he_normal(pl):
    theta = pl.init_params(11)
    (w2, b2) = pl.unpack(theta)[1]
    assert np.all(b2 == 0)
    assert abs(w2.std() - np.sqrt(2.0 / 288)) < 0.02 * np.sqrt(2.0 / 288)
