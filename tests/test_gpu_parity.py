"""GPU parity: every C-ABI call against the FP64 oracle on the same seeded
inputs.

Tolerances (FP32 path vs FP64 oracle):
  * match lists: where the oracle's gap between the K-th and (K+1)-th
    distance exceeds 1e-5 the selected set is bit-exact; slot order is
    bit-exact wherever adjacent oracle distances differ by more than 1e-5;
    every selected block's oracle distance is within 1e-5 of the K-th best;
  * filtered groups, weights (relative) and aggregated images: max-abs 1e-4,
    with the oracle driven by the GPU's own match lists;
  * end to end (oracle with its own matching): PSNR within 0.01 dB.
"""
import os

import numpy as np
import pytest

from paper_2103_10765_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2103_10765_gb300 import gbm3d  # noqa: E402

NT = os.cpu_count() or 4
DEV = torch.device("cuda:0")
TIE = 1e-5
ATOL = 1e-4


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def block_d(X, i, j, idx, W, N=8):
    """FP64 squared distances between block (i,j) and blocks at linear positions idx."""
    ref = X[i:i + N, j:j + N]
    return np.array([np.sum((ref - X[v // W:v // W + N, v % W:v % W + N]) ** 2) for v in idx])


def check_match(X, gidx, gdist, oidx, odist, W, K, refs, N=8):
    """Compare GPU lists (K) with oracle lists computed with K+1 slots."""
    X = X.astype(np.float64)
    exact = 0
    for t, (i, j) in enumerate(refs):
        g = gidx[t]
        assert g[0] == i * W + j
        assert len(set(g.tolist())) == K
        od = odist[t]
        gd = block_d(X, i, j, g[1:], W, N)
        # GPU's own FP32 distances agree with FP64
        np.testing.assert_allclose(gdist[t, 1:], gd, rtol=1e-5, atol=TIE)
        # every chosen block is among the K best up to the tie tolerance
        assert np.all(gd <= od[K - 1] + TIE), (t, gd.max(), od[K - 1])
        # order: nondecreasing up to ties
        assert np.all(np.diff(gd) >= -TIE)
        if od[K] - od[K - 1] > TIE:
            assert set(g.tolist()) == set(oidx[t, :K].tolist()), t
            for r in range(1, K):
                lo_gap = od[r] - od[r - 1]
                hi_gap = od[r + 1] - od[r]
                if lo_gap > TIE and hi_gap > TIE:
                    assert g[r] == oidx[t, r], (t, r)
        exact += int(np.array_equal(g, oidx[t, :K]))
    return exact / len(refs)


def grid_refs(orc, H, W, N=8, s=3):
    return [(int(i), int(j)) for i in orc.grid(H, N, s) for j in orc.grid(W, N, s)]


@pytest.mark.parametrize("H,W,sigma,K", [(64, 72, 25, 16), (100, 83, 25, 32), (13, 13, 50, 32), (13, 45, 15, 16),
                                         (40, 40, 0, 32)])
def test_match_parity(orc, H, W, sigma, K):
    _, X = synth.make_pair(H, W, sigma / 255, 2)
    p = gbm3d.params_default()
    gidx, gdist = gbm3d.match(gpu(X), K, p, with_dist=True)
    oidx, odist = orc.match(X, K=K + 1, nthreads=NT)
    frac = check_match(X, gidx.cpu().numpy(), gdist.cpu().numpy(), oidx, odist, W, K, grid_refs(orc, H, W))
    assert frac > 0.9


def test_match_exact_ties_flat_image(orc):
    """sigma = 0 piecewise-constant image: many exact zero distances, broken by (row, col)."""
    X = np.zeros((48, 56), np.float32)
    X[:, 28:] = 0.5
    X[20:30, 10:20] = 0.25
    gidx, _ = gbm3d.match(gpu(X), 32, with_dist=True)
    oidx, _ = orc.match(X, K=32, nthreads=NT)
    np.testing.assert_array_equal(gidx.cpu().numpy(), oidx)


@pytest.mark.parametrize("H,W,K", [(1024, 1024, 16), (1024, 1024, 32), (2048, 2048, 16), (4096, 4096, 16),
                                   (4096, 4096, 32)])
def test_match_parity_full_size_sampled(orc, H, W, K):
    """Full-size launch (as the benchmark runs it); oracle on a sample of references."""
    _, X = synth.make_pair(H, W, 25 / 255, 1)
    gidx, gdist = gbm3d.match(gpu(X), K, with_dist=True)
    gy, gx = orc.grid(H, 8, 3), orc.grid(W, 8, 3)
    rs = np.random.default_rng(7)
    sel = list(rs.choice(len(gy) * len(gx), 300, replace=False)) + [0, len(gx) - 1, len(gy) * len(gx) - 1]
    refs = [(int(gy[s // len(gx)]), int(gx[s % len(gx)])) for s in sel]
    oidx, odist = orc.match_refs(X, [r[0] for r in refs], [r[1] for r in refs], K=K + 1, nthreads=NT)
    frac = check_match(X, gidx.cpu().numpy()[sel], gdist.cpu().numpy()[sel], oidx, odist, W, K, refs)
    assert frac > 0.9


@pytest.mark.parametrize("H,W,sigma,C", [(64, 72, 25, 2), (100, 83, 50, 2), (13, 13, 25, 2), (48, 48, 15, 1),
                                         (56, 40, 25, 3), (64, 56, 25, 4)])
def test_filter_ht_parity(orc, H, W, sigma, C):
    _, X = synth.make_pair(H, W, sigma / 255, 3)
    p = gbm3d.params_default().replace(cycle_spins=C)
    z = gpu(X)
    idx, _ = gbm3d.match(z, p.k1, p)
    groups, w = gbm3d.filter_ht(z, idx, sigma / 255, p)
    by, bx = gbm3d.grid_dims(H, W, p)
    og, ow = orc.filter_ht(X, idx.cpu().numpy(), sigma / 255, by, bx, C=C)
    assert np.abs(groups.cpu().numpy() - og).max() <= ATOL
    np.testing.assert_allclose(w.cpu().numpy(), ow, rtol=ATOL)


def test_filter_ht_levels_and_k8(orc):
    _, X = synth.make_pair(64, 64, 0.1, 1)
    for levels, k1 in ((1, 16), (2, 16), (3, 8), (3, 32)):
        p = gbm3d.params_default().replace(levels=levels, k1=k1)
        z = gpu(X)
        idx, _ = gbm3d.match(z, k1, p)
        groups, w = gbm3d.filter_ht(z, idx, 0.1, p)
        by, bx = gbm3d.grid_dims(64, 64, p)
        og, ow = orc.filter_ht(X, idx.cpu().numpy(), 0.1, by, bx, K=k1, L=levels)
        assert np.abs(groups.cpu().numpy() - og).max() <= ATOL, (levels, k1)
        np.testing.assert_allclose(w.cpu().numpy(), ow, rtol=ATOL)


@pytest.mark.parametrize("H,W,sigma,K", [(64, 72, 25, 32), (100, 83, 50, 16), (13, 13, 15, 8)])
def test_filter_wiener_parity(orc, H, W, sigma, K):
    clean, X = synth.make_pair(H, W, sigma / 255, 1)
    pilot = (clean + 0.01 * np.sin(np.arange(W))[None, :]).astype(np.float32)
    p = gbm3d.params_default().replace(k2=K)
    idx, _ = gbm3d.match(gpu(pilot), K, p)
    groups, w = gbm3d.filter_wiener(gpu(X), gpu(pilot), idx, sigma / 255, p)
    og, ow = orc.filter_wiener(X, pilot, idx.cpu().numpy(), sigma / 255, K=K, nthreads=NT)
    assert np.abs(groups.cpu().numpy() - og).max() <= ATOL
    np.testing.assert_allclose(w.cpu().numpy(), ow, rtol=ATOL)


@pytest.mark.parametrize("beta,K", [(0.0, 16), (2.0, 32)])
def test_aggregate_parity(orc, beta, K):
    H, W = 77, 64
    _, X = synth.make_pair(H, W, 0.1, 2)
    idx, _ = gbm3d.match(gpu(X), K)
    G = idx.shape[0]
    rs = np.random.default_rng(3)
    groups = rs.standard_normal((G, K, 8, 8)).astype(np.float32)
    w = (rs.random(G) + 0.1).astype(np.float32)
    out = gbm3d.aggregate(gpu(groups), gpu(w), idx, H, W, window_beta=beta)
    ref = orc.aggregate(groups, w, idx.cpu().numpy(), H, W, beta=beta)
    assert np.abs(out.cpu().numpy() - ref).max() <= ATOL


def test_aggregate_deterministic():
    _, X = synth.make_pair(96, 96, 0.1, 2)
    idx, _ = gbm3d.match(gpu(X), 32)
    rs = np.random.default_rng(4)
    groups = gpu(rs.random((idx.shape[0], 32, 8, 8)))
    w = gpu(rs.random(idx.shape[0]) + 0.5)
    a = gbm3d.aggregate(groups, w, idx, 96, 96, window_beta=2.0)
    b = gbm3d.aggregate(groups, w, idx, 96, 96, window_beta=2.0)
    assert torch.equal(a, b)


@pytest.mark.parametrize("H,W,sigma", [(64, 72, 25), (100, 83, 50), (13, 40, 15)])
def test_chained_two_stage_parity(orc, H, W, sigma):
    """Oracle filters driven by the GPU's own match lists, stage by stage."""
    s = sigma / 255
    _, X = synth.make_pair(H, W, s, 2)
    p = gbm3d.params_default()
    z = gpu(X)
    y1 = gbm3d.denoise(z, s, p.replace(stages=1))
    idx1, _ = gbm3d.match(z, p.k1, p)
    by, bx = gbm3d.grid_dims(H, W, p)
    og, ow = orc.filter_ht(X, idx1.cpu().numpy(), s, by, bx)
    oy1 = orc.aggregate(og, ow, idx1.cpu().numpy(), H, W)
    assert np.abs(y1.cpu().numpy() - oy1).max() <= ATOL
    y2 = gbm3d.denoise(z, s, p)
    idx2, _ = gbm3d.match(y1, p.k2, p)
    og2, ow2 = orc.filter_wiener(X, y1.cpu().numpy(), idx2.cpu().numpy(), s, K=p.k2, nthreads=NT)
    oy2 = orc.aggregate(og2, ow2, idx2.cpu().numpy(), H, W, beta=2.0)
    assert np.abs(y2.cpu().numpy() - oy2).max() <= ATOL


@pytest.mark.parametrize("H,W,sigma", [(256, 256, 25), (512, 512, 15), (512, 512, 25), (512, 512, 50)])
def test_end_to_end_psnr(orc, H, W, sigma):
    s = sigma / 255
    clean, X = synth.make_pair(H, W, s, 1)
    out = gbm3d.denoise(gpu(X), s).cpu().numpy()
    ref = orc.denoise(X, s, nthreads=NT)
    pg, po = orc.psnr(out, clean), orc.psnr(ref, clean)
    assert abs(pg - po) <= 0.01, (pg, po)
    assert pg > orc.psnr(X, clean) + 5


@pytest.mark.parametrize("k1,k2", [(8, 16), (32, 32)])
def test_group_sizes_end_to_end(orc, k1, k2):
    # stage-1 groups of 8 and 32 blocks through the whole denoise (the TV
    # weights and the planar permutation for every group size), stage 2 at 16 / 32
    s = 25 / 255
    clean, X = synth.make_pair(72, 64, s, 5)
    p = gbm3d.params_default().replace(k1=k1, k2=k2)
    out = gbm3d.denoise(gpu(X), s, p).cpu().numpy()
    ref = orc.denoise(X, s, params=orc.Params(k1=k1, k2=k2), nthreads=NT)
    assert abs(orc.psnr(out, clean) - orc.psnr(ref, clean)) <= 0.01


@pytest.mark.parametrize("T,stages,C", [(2, 2, 2), (3, 1, 1), (1, 1, 2)])
def test_variants_end_to_end(orc, T, stages, C):
    s = 25 / 255
    clean, X = synth.make_pair(64, 80, s, 3)
    p = gbm3d.params_default().replace(translations=T, stages=stages, cycle_spins=C)
    out = gbm3d.denoise(gpu(X), s, p).cpu().numpy()
    ref = orc.denoise(X, s, params=orc.Params(translations=T, stages=stages, cycle_spins=C), nthreads=NT)
    assert abs(orc.psnr(out, clean) - orc.psnr(ref, clean)) <= 0.01


def test_sigma_zero_and_constant(orc):
    _, X = synth.make_pair(48, 56, 0.0, 1)
    out = gbm3d.denoise(gpu(X), 0.0).cpu().numpy()
    assert np.abs(out - X).max() <= 1e-5
    c, s = 0.6, 25 / 255
    out = gbm3d.denoise(gpu(synth.constant_image(40, 48, c)), s).cpu().numpy()
    P = c * 8 * np.sqrt(32)
    assert np.abs(out - c * P ** 2 / (P ** 2 + s ** 2)).max() <= 1e-5


def test_pitched_input_matches_contiguous():
    _, X = synth.make_pair(64, 70, 0.1, 1)
    big = torch.zeros((64, 96), device=DEV)
    big[:, :70] = gpu(X)
    view = big[:, :70]
    a = gbm3d.denoise(gpu(X), 0.1)
    b = gbm3d.denoise(view, 0.1, out=torch.zeros((64, 96), device=DEV)[:, :70])
    assert torch.equal(a, b)


def test_denoise_4096_runs():
    """The 4096 x 4096 grayscale configuration end to end (33 GB workspace):
    finite output, and far closer to the clean scene than the noisy input."""
    clean, X = synth.make_pair(4096, 4096, 25 / 255, 3)
    out = gbm3d.denoise(gpu(X), 25 / 255).cpu().numpy().astype(np.float64)
    assert np.isfinite(out).all()
    c = clean.astype(np.float64)
    p_noisy = 10 * np.log10(1 / np.mean((X.astype(np.float64) - c) ** 2))
    p_out = 10 * np.log10(1 / np.mean((out - c) ** 2))
    assert p_out > p_noisy + 8, (p_noisy, p_out)


# ---- the Sec. 5 parameter list: 16 x 16 tiling blocks in stage 1, 8 x 8 in stage 2

def paper_stage(stage, **kw):
    return gbm3d.params_stage(gbm3d.params_default(1), stage).replace(**kw)


@pytest.mark.parametrize("H,W,sigma,K,s", [(64, 72, 25, 16, 16), (100, 83, 25, 32, 5), (37, 45, 50, 16, 3),
                                           (16, 40, 15, 8, 16), (48, 48, 0, 16, 16)])
def test_match_n16_parity(orc, H, W, sigma, K, s):
    _, X = synth.make_pair(H, W, sigma / 255, 2)
    p = paper_stage(1, step=s)
    gidx, gdist = gbm3d.match(gpu(X), K, p, with_dist=True)
    oidx, odist = orc.match(X, N=16, s=s, R=16, K=K + 1, nthreads=NT)
    frac = check_match(X, gidx.cpu().numpy(), gdist.cpu().numpy(), oidx, odist, W, K,
                       grid_refs(orc, H, W, 16, s), N=16)
    assert frac > 0.9


@pytest.mark.parametrize("H,W,sigma,C,K", [(64, 80, 25, 2, 16), (100, 83, 50, 2, 16), (48, 48, 15, 1, 8),
                                           (32, 32, 25, 2, 32), (16, 40, 25, 3, 16), (48, 64, 25, 4, 16)])
def test_filter_ht_n16_parity(orc, H, W, sigma, C, K):
    _, X = synth.make_pair(H, W, sigma / 255, 3)
    p = paper_stage(1, cycle_spins=C, k1=K)
    z = gpu(X)
    idx, _ = gbm3d.match(z, K, p)
    groups, w = gbm3d.filter_ht(z, idx, sigma / 255, p)
    assert groups.shape[2:] == (16, 16)
    by, bx = gbm3d.grid_dims(H, W, p)
    og, ow = orc.filter_ht(X, idx.cpu().numpy(), sigma / 255, by, bx, N=16, K=K, C=C)
    assert np.abs(groups.cpu().numpy() - og).max() <= ATOL
    np.testing.assert_allclose(w.cpu().numpy(), ow, rtol=ATOL)


@pytest.mark.parametrize("beta,s", [(0.0, 16), (2.0, 5)])
def test_aggregate_n16_parity(orc, beta, s):
    H, W = 77, 64
    _, X = synth.make_pair(H, W, 0.1, 2)
    p = paper_stage(1, step=s)
    idx, _ = gbm3d.match(gpu(X), 16, p)
    G = idx.shape[0]
    rs = np.random.default_rng(3)
    groups = rs.standard_normal((G, 16, 16, 16)).astype(np.float32)
    w = (rs.random(G) + 0.1).astype(np.float32)
    out = gbm3d.aggregate(gpu(groups), gpu(w), idx, H, W, p, window_beta=beta)
    ref = orc.aggregate(groups, w, idx.cpu().numpy(), H, W, N=16, beta=beta)
    assert np.abs(out.cpu().numpy() - ref).max() <= ATOL


@pytest.mark.parametrize("H,W,sigma", [(64, 80, 25), (100, 83, 50)])
def test_paper_preset_chained_parity(orc, H, W, sigma):
    """Each stage of the Sec. 5 preset against the oracle's filter and
    aggregation driven by the GPU's own match lists."""
    s = sigma / 255
    _, X = synth.make_pair(H, W, s, 2)
    q = gbm3d.params_default(1).replace(translations=1)
    z = gpu(X)
    y1 = gbm3d.denoise(z, s, q.replace(stages=1))
    p1, p2 = gbm3d.params_stage(q, 1), gbm3d.params_stage(q, 2)
    idx1, _ = gbm3d.match(z, q.k1, p1)
    by, bx = gbm3d.grid_dims(H, W, p1)
    og, ow = orc.filter_ht(X, idx1.cpu().numpy(), s, by, bx, N=16, K=q.k1)
    oy1 = orc.aggregate(og, ow, idx1.cpu().numpy(), H, W, N=16)
    assert np.abs(y1.cpu().numpy() - oy1).max() <= ATOL
    y2 = gbm3d.denoise(z, s, q)
    idx2, _ = gbm3d.match(y1, q.k2, p2)
    og2, ow2 = orc.filter_wiener(X, y1.cpu().numpy(), idx2.cpu().numpy(), s, N=8, K=q.k2, nthreads=NT)
    oy2 = orc.aggregate(og2, ow2, idx2.cpu().numpy(), H, W, N=8, beta=2.0)
    assert np.abs(y2.cpu().numpy() - oy2).max() <= ATOL


@pytest.mark.parametrize("H,W,sigma", [(96, 128, 25), (256, 256, 15), (512, 512, 50), (1024, 1024, 25)])
def test_paper_preset_end_to_end_psnr(orc, H, W, sigma):
    """The whole Sec. 5 preset (both stages, 2 translations with each stage's
    own shifts) within 0.01 dB of the FP64 oracle."""
    s = sigma / 255
    clean, X = synth.make_pair(H, W, s, 1)
    out = gbm3d.denoise(gpu(X), s, gbm3d.params_default(1)).cpu().numpy()
    ref = orc.denoise(X, s, params=orc.Params.paper(), nthreads=NT)
    pg, po = orc.psnr(out, clean), orc.psnr(ref, clean)
    assert abs(pg - po) <= 0.01, (pg, po)
    assert pg > orc.psnr(X, clean) + 5


def test_paper_preset_sigma_zero_and_constant():
    q = gbm3d.params_default(1)
    _, X = synth.make_pair(48, 64, 0.0, 1)
    out = gbm3d.denoise(gpu(X), 0.0, q).cpu().numpy()
    assert np.abs(out - X).max() <= 1e-5
    c, s = 0.45, 25 / 255
    out = gbm3d.denoise(gpu(synth.constant_image(48, 40, c)), s, q).cpu().numpy()
    P = c * 8 * np.sqrt(16)
    assert np.abs(out - c * P ** 2 / (P ** 2 + s ** 2)).max() <= 1e-5


# ---- box-sum matching engine (match_engine = 3)

@pytest.mark.parametrize("H,W,sigma,K,s,R", [(64, 72, 25, 16, 3, 19), (100, 83, 25, 32, 3, 19), (13, 13, 50, 32, 3, 19),
                                             (40, 40, 0, 32, 3, 19), (57, 131, 15, 8, 1, 5), (70, 66, 25, 16, 2, 9),
                                             (90, 77, 50, 32, 3, 12), (48, 48, 25, 2, 3, 3)])
def test_box_engine_parity(orc, H, W, sigma, K, s, R):
    _, X = synth.make_pair(H, W, sigma / 255, 2)
    p = gbm3d.params_default().replace(match_engine=3, step=s, search_radius=R)
    gidx, gdist = gbm3d.match(gpu(X), K, p, with_dist=True)
    oidx, odist = orc.match(X, N=8, s=s, R=R, K=K + 1, nthreads=NT)
    frac = check_match(X, gidx.cpu().numpy(), gdist.cpu().numpy(), oidx, odist, W, K, grid_refs(orc, H, W, 8, s))
    assert frac > 0.9


def test_box_engine_exact_ties_flat_image(orc):
    X = np.zeros((48, 56), np.float32)
    X[:, 28:] = 0.5
    X[20:30, 10:20] = 0.25
    p = gbm3d.params_default().replace(match_engine=3)
    gidx, _ = gbm3d.match(gpu(X), 32, p, with_dist=True)
    oidx, _ = orc.match(X, K=32, nthreads=NT)
    np.testing.assert_array_equal(gidx.cpu().numpy(), oidx)


@pytest.mark.parametrize("K", [16, 32])
def test_box_engine_full_size_sampled(orc, K):
    H = W = 1024
    _, X = synth.make_pair(H, W, 25 / 255, 1)
    p = gbm3d.params_default().replace(match_engine=3)
    gidx, gdist = gbm3d.match(gpu(X), K, p, with_dist=True)
    gidx2, _ = gbm3d.match(gpu(X), K, p, with_dist=True)
    assert torch.equal(gidx, gidx2)  # deterministic
    gy, gx = orc.grid(H, 8, 3), orc.grid(W, 8, 3)
    rs = np.random.default_rng(8)
    sel = list(rs.choice(len(gy) * len(gx), 300, replace=False)) + [0, len(gx) - 1, len(gy) * len(gx) - 1]
    refs = [(int(gy[t // len(gx)]), int(gx[t % len(gx)])) for t in sel]
    oidx, odist = orc.match_refs(X, [r[0] for r in refs], [r[1] for r in refs], K=K + 1, nthreads=NT)
    frac = check_match(X, gidx.cpu().numpy()[sel], gdist.cpu().numpy()[sel], oidx, odist, W, K, refs)
    assert frac > 0.9


def test_box_engine_denoise_psnr(orc):
    s = 25 / 255
    clean, X = synth.make_pair(256, 256, s, 1)
    out = gbm3d.denoise(gpu(X), s, gbm3d.params_default().replace(match_engine=3)).cpu().numpy()
    ref = orc.denoise(X, s, nthreads=NT)
    assert abs(orc.psnr(out, clean) - orc.psnr(ref, clean)) <= 0.01
