"""Tensor-core block matching (Theorem 1 norm expansion on tcgen05, exact
FP32 re-rank of the certified survivors) against the direct FP32 engine: the
two must agree bit for bit -- indices and distances -- on every reference,
including the ones the tensor-core pass hands back to the direct kernel
(near-ties, constant images).  The direct engine is itself pinned to the FP64
oracle by test_gpu_parity.py."""
import numpy as np
import pytest
import torch

from paper_2103_10765_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_2103_10765_gb300 import gbm3d
    gbm3d.load()
    return gbm3d


def _both(g, img, K, **kw):
    p = g.params_default()
    if kw:
        p = p.replace(**kw)
    i1, d1 = g.match(img, K, p.replace(match_engine=1), with_dist=True)
    i2, d2 = g.match(img, K, p.replace(match_engine=2), with_dist=True)
    # the same engine without a distance output returns the same indices
    i3, _ = g.match(img, K, p.replace(match_engine=2), with_dist=False)
    torch.cuda.synchronize()
    nd = int((i3 != i2).any(dim=1).sum())
    assert nd == 0, f"{nd} references differ without distances"
    return i1, d1, i2, d2


def _assert_same(i1, d1, i2, d2):
    bad = (i1 != i2).any(dim=1) | (d1.view(torch.int32) != d2.view(torch.int32)).any(dim=1)
    n = int(bad.sum())
    assert n == 0, f"{n} of {i1.shape[0]} references differ; first {torch.nonzero(bad)[:5].flatten().tolist()}"


def _noisy(H, W, sigma, seed=1):
    _, z = synth.make_pair(H, W, sigma, seed)
    return torch.from_numpy(np.ascontiguousarray(z)).cuda()


def _clean(H, W, seed=1):
    c, _ = synth.make_pair(H, W, 0.1, seed)
    return torch.from_numpy(np.ascontiguousarray(c)).cuda()


@pytest.mark.parametrize("H,W", [(64, 72), (37, 101), (101, 37), (256, 256), (300, 260)])
@pytest.mark.parametrize("K", [16, 32])
def test_engines_identical_noisy(g, H, W, K):
    _assert_same(*_both(g, _noisy(H, W, 25 / 255), K))


@pytest.mark.parametrize("sigma", [5, 15, 50])
def test_engines_identical_sigmas(g, sigma):
    _assert_same(*_both(g, _noisy(256, 256, sigma / 255, seed=2), 16))


@pytest.mark.parametrize("K", [2, 8, 16, 32])
def test_engines_identical_clean(g, K):
    # noise-free piecewise-smooth scene: many near-ties, some references go back to the direct kernel
    _assert_same(*_both(g, _clean(200, 232), K))


def test_engines_identical_constant(g):
    # every distance is 0: no list can be certified, every reference is re-matched directly
    img = torch.full((96, 80), 0.5, device="cuda")
    _assert_same(*_both(g, img, 16))


def test_engines_identical_other_geometry(g):
    img = _noisy(160, 144, 25 / 255, seed=3)
    for kw in (dict(step=1, search_radius=12), dict(step=2, search_radius=16), dict(step=4, search_radius=10),
               dict(step=3, search_radius=2)):
        _assert_same(*_both(g, img, 8, **kw))


def test_engines_identical_pitched_and_offset(g):
    base = _noisy(140, 200, 25 / 255, seed=4)
    view = base[3:131, 5:181]  # pitch 200, unaligned start
    _assert_same(*_both(g, view, 16))


@pytest.mark.parametrize("pitch", [200, 201, 204])
def test_engines_identical_region_load_paths(g, pitch):
    """The search region of a tile arrives by one TMA box where the image
    allows it (16-byte aligned start, row pitch a multiple of 16 bytes: pitch
    200 and 204 here) and by thread loads otherwise (pitch 201); the lists
    are the direct engine's either way."""
    base = torch.zeros((150, pitch), device="cuda")
    base[:, :176] = _noisy(150, 176, 25 / 255, seed=6)
    view = base[:, :176]
    _assert_same(*_both(g, view, 16))
    _assert_same(*_both(g, view, 32))


def test_engines_identical_scaled_and_shifted(g):
    # the power-of-two scaling and centring must not change the ranking
    z = _noisy(128, 128, 25 / 255, seed=5)
    for img in (z * 1e4 + 3e4, z * 1e-3 - 7.0, z - 100.0):
        _assert_same(*_both(g, img.contiguous(), 16))


@pytest.mark.parametrize("K", [16, 32])
def test_engines_identical_full_size(g, K):
    # the bench workload (1024^2, sigma 25/255): every one of the 115,600 lists
    _assert_same(*_both(g, _noisy(1024, 1024, 25 / 255), K))


@pytest.mark.parametrize("K", [16, 32])
def test_engines_identical_4096(g, K):
    # the 4096^2 grayscale configuration: all 1,860,496 lists
    img = _noisy(4096, 4096, 25 / 255, seed=4) if K == 16 else _clean(4096, 4096, seed=4)
    _assert_same(*_both(g, img, K))


def test_engines_identical_full_size_smooth(g):
    # a stage-2-like input (smooth estimate) at full size
    _assert_same(*_both(g, _clean(1024, 1024, seed=2), 32))


def test_full_size_rarely_rematches(g):
    # on the noisy bench input almost every list certifies: under 1 % of the
    # references go back to the direct kernel (a cost, never a change of result)
    img = _noisy(1024, 1024, 25 / 255, seed=6)
    p = g.params_default().replace(match_engine=2)
    t0, r0 = g.match_stats()
    g.match(img, 16, p)
    g.match(img, 32, p)
    t1, r1 = g.match_stats()
    assert t1 == t0
    assert r1 - r0 <= 115600 * 2 // 100  # < 1 %


def test_no_timeouts(g):
    assert g.match_stats()[0] == 0
