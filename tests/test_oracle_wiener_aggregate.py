"""Pins for the oracle's stage-2 Wiener filter (Sec. 4), Kaiser window and
aggregation (Sec. 3.1 weighted average)."""
import numpy as np
import pytest
import scipy.fft
import scipy.special

from paper_2103_10765_gb300 import synth


@pytest.mark.parametrize("N", [4, 8, 16])
def test_dct2_is_scipy_orthonormal_dct2(orc, rng, N):
    x = rng.standard_normal((N, N))
    np.testing.assert_allclose(orc.dct2(x), scipy.fft.dctn(x, type=2, norm="ortho"), atol=1e-13)
    np.testing.assert_allclose(orc.dct2(orc.dct2(x), inverse=True), x, atol=1e-13)


def _haar_matrix(n):
    """Full-depth orthonormal Haar analysis matrix by recursion."""
    if n == 1:
        return np.ones((1, 1))
    s = 1 / np.sqrt(2)
    A = np.zeros((n, n))
    for m in range(n // 2):
        A[m, 2 * m] = A[m, 2 * m + 1] = s
        A[n // 2 + m, 2 * m] = s
        A[n // 2 + m, 2 * m + 1] = -s
    top = np.eye(n)
    top[:n // 2, :n // 2] = _haar_matrix(n // 2)
    return top @ A


@pytest.mark.parametrize("n", [1, 2, 8, 32])
def test_haar_full_depth(orc, rng, n):
    x = rng.standard_normal(n)
    y = orc.haar(x)
    np.testing.assert_allclose(y, _haar_matrix(n) @ x, atol=1e-13)
    assert abs(np.sum(y ** 2) - np.sum(x ** 2)) < 1e-12
    np.testing.assert_allclose(orc.haar(y, inverse=True), x, atol=1e-13)


def _gather(img, idx_row, W, N):
    return np.stack([img[v // W:v // W + N, v % W:v % W + N] for v in idx_row])


def test_wiener_matches_dense_transform(orc):
    _, Z = synth.make_pair(40, 40, 0.1, 2)
    clean = synth.clean_scene(40, 40, 2).astype(np.float64)
    K, N, sigma = 32, 8, 0.1
    idx, _ = orc.match(clean, K=K)
    groups, w = orc.filter_wiener(Z, clean, idx, sigma, N=N, K=K)
    D = scipy.fft.dct(np.eye(N), type=2, norm="ortho", axis=0)
    Hm = _haar_matrix(K)
    for g in (0, 5, len(idx) - 1):
        gz = _gather(Z.astype(np.float64), idx[g], 40, N)
        gy = _gather(clean, idx[g], 40, N)
        T = lambda x: np.einsum("rs,ua,vb,sab->ruv", Hm, D, D, x)
        Ti = lambda x: np.einsum("sr,ua,vb,suv->rab", Hm, D, D, x)
        P = T(gy)
        om = P ** 2 / (P ** 2 + sigma ** 2)
        np.testing.assert_allclose(groups[g], Ti(om * T(gz)), atol=1e-12)
        assert abs(w[g] - 1.0 / (sigma ** 2 * np.sum(om ** 2))) <= 1e-10 * w[g]


def test_wiener_special_cases(orc):
    _, Z = synth.make_pair(32, 32, 0.1, 1)
    idx, _ = orc.match(Z, K=16)
    # sigma = 0: every nonzero coefficient passes -> the noisy group itself
    g0, w0 = orc.filter_wiener(Z, Z, idx, 0.0, K=16, eps_w=1e-8)
    for g in (0, 7):
        np.testing.assert_allclose(g0[g], _gather(Z.astype(np.float64), idx[g], 32, 8), atol=1e-12)
    assert np.all(w0 == 1e8)
    # a zero pilot shrinks everything to zero
    gz, _ = orc.filter_wiener(Z, np.zeros_like(Z), idx, 0.1, K=16)
    assert np.all(gz == 0.0)


def test_wiener_with_clean_pilot_reduces_error(orc):
    clean, Z = synth.make_pair(48, 48, 30 / 255, 3)
    idx, _ = orc.match(clean, K=32)
    groups, _ = orc.filter_wiener(Z, clean, idx, 30 / 255, K=32)
    err_f = err_n = 0.0
    for g in range(len(idx)):
        gc = _gather(clean.astype(np.float64), idx[g], 48, 8)
        gn = _gather(Z.astype(np.float64), idx[g], 48, 8)
        err_f += np.sum((groups[g] - gc) ** 2)
        err_n += np.sum((gn - gc) ** 2)
    assert err_f < 0.5 * err_n


def test_kaiser_window(orc):
    for N, beta in ((8, 2.0), (16, 2.0), (8, 5.0)):
        np.testing.assert_allclose(orc.kaiser(N, beta), np.kaiser(N, beta), atol=1e-14)
    np.testing.assert_array_equal(orc.kaiser(8, 0.0), np.ones(8))
    for x in (0.0, 0.5, 2.0, 7.5):
        assert abs(orc.bessel_i0(x) - scipy.special.i0(x)) <= 1e-14 * scipy.special.i0(x)


def _brute_aggregate(groups, w, idx, H, W, N, kap):
    num = np.zeros((H, W))
    den = np.zeros((H, W))
    for g in range(len(w)):
        for r in range(idx.shape[1]):
            i, j = divmod(int(idx[g, r]), W)
            win = np.outer(kap, kap)
            num[i:i + N, j:j + N] += w[g] * win * groups[g, r]
            den[i:i + N, j:j + N] += w[g] * win
    return num / den


@pytest.mark.parametrize("beta,N,s", [(0.0, 8, 3), (2.0, 8, 3), (0.0, 16, 16), (2.0, 16, 5)])
def test_aggregate_brute_force(orc, rng, beta, N, s):
    _, Z = synth.make_pair(30 + N, 27 + N, 0.1, 1)
    H, W = Z.shape
    idx, _ = orc.match(Z, N=N, s=s, R=7, K=16)
    G = len(idx)
    groups = rng.standard_normal((G, 16, N, N))
    w = rng.random(G) + 0.1
    out = orc.aggregate(groups, w, idx, H, W, N=N, beta=beta)
    kap = np.kaiser(N, beta) if beta > 0 else np.ones(N)
    np.testing.assert_allclose(out, _brute_aggregate(groups, w, idx, H, W, N, kap), atol=1e-12)


def test_aggregate_invariants(orc, rng):
    _, Z = synth.make_pair(40, 33, 0.1, 2)
    idx, _ = orc.match(Z, K=16)
    G = len(idx)
    w = rng.random(G) + 0.01
    # constant blocks -> constant image, for any positive weights
    out = orc.aggregate(np.full((G, 16, 8, 8), 0.37), w, idx, 40, 33, beta=2.0)
    np.testing.assert_allclose(out, 0.37, atol=1e-14)
    # exact copies of the image blocks -> the image itself
    groups = np.stack([_gather(Z.astype(np.float64), idx[g], 33, 8) for g in range(G)])
    np.testing.assert_allclose(orc.aggregate(groups, w, idx, 40, 33), Z, atol=1e-14)
