"""Pins for the oracle's reference grid and block matching (Sec. 2, Sec. 3.1)."""
import numpy as np
import pytest

from paper_2103_10765_gb300 import synth


def brute_match(X, N, R, K, i, j):
    """Plain enumeration: every candidate, sorted by (d, row, col)."""
    H, W = X.shape
    c = []
    for k in range(max(0, i - R), min(H - N, i + R) + 1):
        for l in range(max(0, j - R), min(W - N, j + R) + 1):
            if (k, l) == (i, j):
                continue
            d = float(np.sum((X[i:i + N, j:j + N] - X[k:k + N, l:l + N]) ** 2))
            c.append((d, k, l))
    c.sort()
    return [i * W + j] + [k * W + l for _, k, l in c[:K - 1]], [0.0] + [d for d, _, _ in c[:K - 1]]


def test_grid_closed_form(orc):
    assert [len(orc.grid(M, 8, 3)) for M in (256, 512, 1024)] == [84, 169, 340]
    for M in range(8, 120):
        for N, s in ((8, 3), (8, 8), (4, 3), (16, 16)):
            g = orc.grid(M, N, s)
            if M < N:
                assert len(g) == 0
                continue
            want = (M - N) // s + 1 + (1 if (M - N) % s else 0)
            assert len(g) == want
            assert g[0] == 0 and g[-1] == M - N
            assert np.all(np.diff(g) > 0) and np.all(np.diff(g)[:-1] == s)


@pytest.mark.parametrize("H,W,N,R,K", [(16, 16, 4, 3, 5), (20, 13, 4, 3, 8), (24, 24, 8, 19, 16), (17, 30, 8, 5, 32),
                                       (37, 29, 16, 6, 16)])
def test_match_brute_force(orc, rng, H, W, N, R, K):
    X = rng.random((H, W))
    idx, dist = orc.match(X, N=N, s=3, R=R, K=K)
    gy, gx = orc.grid(H, N, 3), orc.grid(W, N, 3)
    t = 0
    for i in gy:
        for j in gx:
            bi, bd = brute_match(X, N, R, K, int(i), int(j))
            assert list(idx[t]) == bi
            np.testing.assert_allclose(dist[t], bd, rtol=0, atol=1e-12)
            t += 1


def test_theorem1_distance_identity_via_fft(orc, rng):
    """Theorem 1: ||z^ij - z^kl||^2 = (I_N * Z^2)[i,j] + (I_N * Z^2)[k,l] - 2 (Z^ij * Z)[k,l],
    with the cross-correlations evaluated in the Fourier domain (eq. CCF)."""
    H, W, N = 32, 40, 8
    Z = rng.random((H, W))
    F = np.fft.fft2
    IN = np.zeros((H, W))
    IN[:N, :N] = 1.0

    def xcorr(Y, Zi):  # (Y * Z)[i,j] = sum_ab Y[a,b] Z[i+a, j+b], periodic
        return np.real(np.fft.ifft2(np.conj(F(Y)) * F(Zi)))

    norms = xcorr(IN, Z * Z)
    for (i, j) in [(0, 0), (5, 7), (24, 32), (13, 2)]:
        Zij = np.zeros((H, W))
        Zij[:N, :N] = Z[i:i + N, j:j + N]
        D = norms[i, j] + norms - 2.0 * xcorr(Zij, Z)
        for k in range(0, H - N + 1, 3):
            for l in range(0, W - N + 1, 2):
                assert abs(orc.patch_dist(Z, N, i, j, k, l) - D[k, l]) < 1e-10


def test_planted_copy_found_at_zero(orc, rng):
    X = rng.random((48, 48))
    X[25:33, 20:28] = X[9:17, 12:20]  # exact copy of the reference block at (9,12)
    idx, dist = orc.match_refs(X, [9], [12], N=8, R=19, K=16)
    assert idx[0, 0] == 9 * 48 + 12 and dist[0, 0] == 0.0
    assert idx[0, 1] == 25 * 48 + 20 and dist[0, 1] == 0.0


def test_match_invariants_synthetic(orc):
    _, X = synth.make_pair(64, 72, 25 / 255, 2)
    N, R, K = 8, 19, 32
    H, W = X.shape
    idx, dist = orc.match(X, N=N, s=3, R=R, K=K)
    gy, gx = orc.grid(H, N, 3), orc.grid(W, N, 3)
    refs = [(int(i), int(j)) for i in gy for j in gx]
    for t, (i, j) in enumerate(refs):
        row = idx[t]
        assert row[0] == i * W + j
        assert len(set(row.tolist())) == K
        k, l = row // W, row % W
        assert np.all(np.abs(k - i) <= R) and np.all(np.abs(l - j) <= R)
        assert np.all((k >= 0) & (k <= H - N) & (l >= 0) & (l <= W - N))
        d = dist[t, 1:]
        key = list(zip(d, k[1:], l[1:]))
        assert key == sorted(key)


def test_tie_break_on_flat_image(orc):
    X = np.full((40, 40), 0.25)
    idx, dist = orc.match_refs(X, [16], [16], N=8, R=19, K=8)
    # every candidate ties at d = 0: the earliest rows/cols win, reference excluded
    assert np.all(dist[0] == 0)
    assert list(idx[0]) == [16 * 40 + 16] + [0 * 40 + l for l in range(7)]


def test_too_few_candidates_rejected(orc):
    X = np.zeros((9, 9))
    with pytest.raises(orc.OracleError):
        orc.match(X, N=8, s=3, R=19, K=16)  # only 2 x 2 = 4 block positions
