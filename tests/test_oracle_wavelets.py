"""Pins for the oracle's wavelet transforms and the stage-1 global hard
thresholding (Sec. 3.1 eq. BM3DHT, cycle spinning, TV weights; Sec. 5
parameters)."""
import numpy as np
import pytest

from conftest import read_golden


def test_bior15_taps_match_published_table(orc):
    g = read_golden("bior15_filters.txt")
    dec_lo = np.array([float(v) for v in g["dec_lo"][0]])
    rec_hi = np.array([float(v) for v in g["rec_hi"][0]])
    h0, g1 = orc.bior15_filters()
    np.testing.assert_allclose(h0, dec_lo, atol=1e-15)
    # the tabulated high-pass uses the opposite sign for the detail coefficient
    np.testing.assert_allclose(g1, -rec_hi, atol=1e-15)


def test_bior15_moments(orc):
    h0, _ = orc.bior15_filters()
    t = np.arange(10.0)
    assert abs(h0.sum() - np.sqrt(2)) < 1e-15
    for m in range(5):  # five vanishing moments of the alternating sequence
        assert abs(np.sum((-1.0) ** t * t ** m * h0)) < 1e-9


@pytest.mark.parametrize("n", [2, 4, 6, 10, 16, 34, 128])
@pytest.mark.parametrize("kind", [0, 1])
def test_perfect_reconstruction_1d(orc, rng, n, kind):
    x = rng.standard_normal(n)
    lo, hi = orc.dwt1(x, kind)
    np.testing.assert_allclose(orc.idwt1(lo, hi, kind), x, atol=1e-13)


def test_haar_parseval_and_constant(orc, rng):
    x = rng.standard_normal(64)
    lo, hi = orc.dwt1(x, orc.HAAR)
    assert abs(np.sum(lo ** 2) + np.sum(hi ** 2) - np.sum(x ** 2)) < 1e-12
    lo, hi = orc.dwt1(np.full(16, 3.0), orc.BIOR15)
    np.testing.assert_allclose(hi, 0, atol=1e-15)
    np.testing.assert_allclose(lo, 3.0 * np.sqrt(2), atol=1e-13)


def test_detail_impulse_synthesis_response(orc):
    """Inverting a single detail coefficient gives the 10-tap synthesis high-pass."""
    n = 32
    lo, hi = np.zeros(n // 2), np.zeros(n // 2)
    hi[6] = 1.0
    x = orc.idwt1(lo, hi, orc.BIOR15)
    _, g1 = orc.bior15_filters()
    want = np.zeros(n)
    want[2 * 6 - 4: 2 * 6 + 6] = g1
    np.testing.assert_allclose(x, want, atol=1e-15)


@pytest.mark.parametrize("shape", [(8, 8, 8), (16, 24, 16), (32, 8, 16), (24, 40, 8)])
def test_dwt3_round_trip(orc, rng, shape):
    v = rng.standard_normal(shape)
    np.testing.assert_allclose(orc.idwt3(orc.dwt3(v)), v, atol=1e-12)


def test_dwt3_constant_volume_is_pure_approximation(orc):
    v = np.full((16, 16, 16), 0.7)
    c = orc.dwt3(v)
    approx = c[:2, :2, :2]
    rest = c.copy()
    rest[:2, :2, :2] = 0
    np.testing.assert_allclose(rest, 0, atol=1e-13)
    np.testing.assert_allclose(approx, 0.7 * (2 ** 1.5) ** 3, atol=1e-12)


def test_upsilon_keeps_exact_threshold(orc):
    lam = 0.3
    assert orc.upsilon(lam, lam) == lam
    assert orc.upsilon(-lam, lam) == -lam
    assert orc.upsilon(np.nextafter(lam, 0), lam) == 0.0
    assert orc.upsilon(0.0, 0.0) == 0.0


def test_dwt3_thresholds_per_level(orc, rng):
    """Level l (1 = finest) details thresholded at tau[l-1]; the coarsest cube untouched."""
    v = rng.standard_normal((16, 16, 16))
    c0 = orc.dwt3(v)
    tau = np.array([1.0, 2.0, 3.0])
    c1 = orc.dwt3(v, tau=tau)
    lev = np.zeros(c0.shape, dtype=int)
    for l in (1, 2, 3):
        h = 16 >> (l - 1)
        lev[:h, :h, :h] = l
    lev[:2, :2, :2] = 0
    for l in (1, 2, 3):
        m = lev == l
        want = np.where(np.abs(c0[m]) >= tau[l - 1], c0[m], 0.0)
        np.testing.assert_array_equal(c1[m], want)
    np.testing.assert_array_equal(c1[lev == 0], c0[lev == 0])


# --- independent dense-matrix evaluation of the whole stage-1 filter -------

def _ana_matrix(n, kind):
    """Single-level analysis as a dense n x n matrix, built from the filter
    definitions (not from the oracle's code)."""
    A = np.zeros((n, n))
    s = 1 / np.sqrt(2)
    h0 = np.array([3, -3, -22, 22, 128, 128, 22, -22, -3, 3]) / (128 * np.sqrt(2))
    for m in range(n // 2):
        A[n // 2 + m, 2 * m] += s
        A[n // 2 + m, 2 * m + 1] -= s
        if kind == 0:
            A[m, 2 * m] += s
            A[m, 2 * m + 1] += s
        else:
            for t in range(10):
                A[m, (2 * m - 4 + t) % n] += h0[t]
    return A


def _dense_ht(V, sigma, L, C, tau_a, tau_b):
    Y, X, Z = V.shape
    U = np.zeros_like(V)
    for h in range(C):
        S = np.roll(V, shift=(h, h, h), axis=(0, 1, 2))  # (S_h V)[y] = V[y - h]
        hh, ww, kk = Y, X, Z
        for l in range(1, L + 1):
            Ay, Ax, Az = _ana_matrix(hh, 1), _ana_matrix(ww, 1), _ana_matrix(kk, 0)
            S[:hh, :ww, :kk] = np.einsum("ay,bx,cz,yxz->abc", Ay, Ax, Az, S[:hh, :ww, :kk])
            tau = sigma * (tau_a - tau_b * l)
            blk = S[:hh, :ww, :kk]
            mask = np.ones(blk.shape, bool)
            mask[:hh // 2, :ww // 2, :kk // 2] = False
            blk[mask & (np.abs(blk) < tau)] = 0.0
            hh, ww, kk = hh // 2, ww // 2, kk // 2
        for l in range(L, 0, -1):
            hh, ww, kk = Y >> (l - 1), X >> (l - 1), Z >> (l - 1)
            iy = np.linalg.inv(_ana_matrix(hh, 1))
            ix = np.linalg.inv(_ana_matrix(ww, 1))
            iz = np.linalg.inv(_ana_matrix(kk, 0))
            S[:hh, :ww, :kk] = np.einsum("ay,bx,cz,yxz->abc", iy, ix, iz, S[:hh, :ww, :kk])
        U += np.roll(S, shift=(-h, -h, -h), axis=(0, 1, 2)) / C
    return U


@pytest.mark.parametrize("C,N,s,R,H,W", [(1, 8, 3, 19, 16, 22), (2, 8, 3, 19, 16, 22),
                                          (2, 16, 16, 16, 32, 40)])
def test_filter_ht_matches_dense_evaluation(orc, C, N, s, R, H, W):
    """Sec. 3.1 eq. BM3DHT with cycle spinning, evaluated with dense per-axis
    matrices; the last case is the Sec. 5 stage-1 geometry (16 x 16 blocks
    tiling the image)."""
    from paper_2103_10765_gb300 import synth
    clean, Zimg = synth.make_pair(H, W, 25 / 255, 3)
    K, sigma = 16, 25 / 255
    idx, _ = orc.match(Zimg, N=N, s=s, R=R, K=K)
    gy, gx = orc.grid(H, N, s), orc.grid(W, N, s)
    By, Bx = len(gy), len(gx)
    groups, w = orc.filter_ht(Zimg, idx, sigma, By, Bx, N=N, K=K, L=3, C=C)
    # volume V[pN+a, qN+b, r] = Z[k_r + a, l_r + b]
    Zd = Zimg.astype(np.float64)
    V = np.zeros((By * N, Bx * N, K))
    for p in range(By):
        for q in range(Bx):
            for r in range(K):
                v = idx[p * Bx + q, r]
                i, j = divmod(int(v), W)
                V[p * N:(p + 1) * N, q * N:(q + 1) * N, r] = Zd[i:i + N, j:j + N]
    U = _dense_ht(V, sigma, 3, C, 3.6, 0.3)
    for p in range(By):
        for q in range(Bx):
            u = U[p * N:(p + 1) * N, q * N:(q + 1) * N, :].transpose(2, 0, 1)
            np.testing.assert_allclose(groups[p * Bx + q], u, atol=1e-12)
            tv = (np.abs(np.diff(u, axis=0)).sum() + np.abs(np.diff(u, axis=1)).sum()
                  + np.abs(np.diff(u, axis=2)).sum())
            assert abs(w[p * Bx + q] - 1.0 / tv) <= 1e-12 * (1.0 / tv)


def test_filter_ht_zero_threshold_is_identity(orc):
    from paper_2103_10765_gb300 import synth
    _, Zimg = synth.make_pair(24, 24, 0.1, 1)
    idx, _ = orc.match(Zimg, K=16)
    By = Bx = len(orc.grid(24, 8, 3))
    groups, _ = orc.filter_ht(Zimg, idx, 0.0, By, Bx)
    for g in range(By * Bx):
        for r in range(16):
            i, j = divmod(int(idx[g, r]), 24)
            np.testing.assert_allclose(groups[g, r], Zimg[i:i + 8, j:j + 8], atol=1e-12)


def test_tv_weights_closed_form(orc):
    """w = 1 / TV with TV the anisotropic L1 forward-difference sum inside the
    group: an interior unit impulse has six unit differences (TV = 6), an
    impulse of 2 in a corner three differences of 2 (TV = 6); a constant
    group has TV = 0 and takes the eps guard."""
    g = np.zeros((3, 16, 8, 8))
    g[0, 5, 3, 4] = 1.0
    g[1, 0, 0, 0] = 2.0
    g[2] = 0.7
    w = orc.tv_weights(g, eps_w=1e-8)
    np.testing.assert_allclose(w, [1 / 6, 1 / 6, 1e8], rtol=1e-12)
