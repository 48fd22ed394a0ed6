"""The C-ABI library loads, exports every symbol include/gbm3d.h declares, and
its host-side logic (presets, grid sizes, workspace sizes, argument
validation) behaves as documented.  No call here reaches the GPU: every
validation failure returns before any launch."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def g():
    from paper_2103_10765_gb300 import build, gbm3d
    build.build_library()
    return gbm3d


@pytest.fixture
def no_gpu():
    """These tests pass fake device pointers that validation must reject before
    any launch; where a GPU is visible they are skipped, so that a validation
    regression can never turn into a launch on a bogus address."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("fake-pointer validation tests run where no GPU is visible")
    except ImportError:
        pass


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gbm3d.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gbm3d_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(g):
    lib = g.load()
    names = declared_functions()
    assert "gbm3d_denoise" in names and len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_version(g):
    assert b"gbm3d" in g.load().gbm3d_version()


def test_presets(g):
    p = g.params_default(0)
    assert (p.patch, p.step, p.search_radius, p.k1, p.k2, p.levels, p.cycle_spins, p.translations, p.stages) == \
        (8, 3, 19, 16, 32, 3, 2, 1, 2)
    assert abs(p.tau_a - 3.6) < 1e-6 and abs(p.tau_b - 0.3) < 1e-6 and p.kaiser_beta == 2.0
    assert p.match_engine == 0
    assert (p.patch2, p.step2) == (8, 3)
    # Sec. 5: 16 x 16 tiling blocks in stage 1, 8 x 8 in stage 2, 32-pixel window, K = 16, 2 translations
    q = g.params_default(1)
    assert (q.patch, q.step, q.patch2, q.step2, q.search_radius, q.k1, q.k2, q.levels, q.cycle_spins,
            q.translations, q.stages) == (16, 16, 8, 8, 16, 16, 16, 3, 2, 2, 2)
    with pytest.raises(g.Gbm3dError):
        g.params_default(7)


def test_params_stage(g, orc):
    q = g.params_default(1)
    s1, s2 = g.params_stage(q, 1), g.params_stage(q, 2)
    assert (s1.patch, s1.step, s1.patch2, s1.step2) == (16, 16, 0, 0)
    assert (s2.patch, s2.step, s2.patch2, s2.step2) == (8, 8, 0, 0)
    assert (s1.k1, s1.k2, s1.translations) == (q.k1, q.k2, q.translations)
    assert g.grid_dims(1024, 1024, s1) == (64, 64) and g.grid_dims(1024, 1024, s2) == (128, 128)
    for H, W in ((100, 77), (48, 40)):
        assert g.grid_dims(H, W, s1) == (len(orc.grid(H, 16, 16)), len(orc.grid(W, 16, 16)))
    p0 = g.params_default(0)
    t = g.params_stage(p0, 2)
    assert (t.patch, t.step) == (8, 3)
    with pytest.raises(g.Gbm3dError):
        g.params_stage(q, 3)


def test_workspace_covers_both_stage_geometries(g):
    q = g.params_default(1)
    n = g.workspace_bytes(1024, 1024, q)
    # stage-1 mosaic pyramid (64*16)^2 * 16 floats plus stage-2 blocks 128^2 * 16 * 64 floats
    assert n > (1024 * 1024 * 16 + 128 * 128 * 16 * 64) * 4
    assert g.workspace_bytes(1024, 1024) > n  # s = 3 overlapping grids need far more


def test_grid_dims_closed_form(g, orc):
    for H, W in ((256, 256), (512, 512), (1024, 1024), (37, 101), (8, 8)):
        assert g.grid_dims(H, W) == (len(orc.grid(H, 8, 3)), len(orc.grid(W, 8, 3)))
    assert g.grid_dims(1024, 1024) == (340, 340)


def test_workspace_monotone(g):
    a = g.workspace_bytes(256, 256)
    b = g.workspace_bytes(512, 512)
    c = g.workspace_bytes(1024, 1024)
    assert 0 < a < b < c
    # groups buffer alone: G * K2 * 64 floats
    assert c >= 340 * 340 * 32 * 64 * 4
    assert g.workspace_bytes(256, 256, g.params_default().replace(translations=3)) > a


def _status(fn, *args):
    return fn(*args)


def test_validation_errors(g, no_gpu):
    lib = g.load()
    p = g.params_default()
    P = ctypes.byref(p)
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: validation fails first
    # image smaller than a block
    assert lib.gbm3d_match(fake, 7, 64, 64, P, 16, fake, None, None, None) == g.EINVAL
    # pitch < W
    assert lib.gbm3d_match(fake, 64, 64, 32, P, 16, fake, None, None, None) == g.EINVAL
    # null pointers
    assert lib.gbm3d_match(None, 64, 64, 64, P, 16, fake, None, None, None) == g.EINVAL
    assert lib.gbm3d_denoise(fake, 64, 64, 64, ctypes.c_float(0.1), P, None, fake, None) == g.EINVAL
    # out aliasing noisy
    assert lib.gbm3d_denoise(fake, 64, 64, 64, ctypes.c_float(0.1), P, fake, fake, None) == g.EINVAL
    # negative or non-finite sigma
    assert lib.gbm3d_denoise(fake, 64, 64, 64, ctypes.c_float(-1.0), P, ctypes.c_void_p(0x2000), fake,
                             None) == g.EINVAL
    assert lib.gbm3d_denoise(fake, 64, 64, 64, ctypes.c_float(float("nan")), P, ctypes.c_void_p(0x2000), fake,
                             None) == g.EINVAL
    # search window too small for K: 9 x 9 image has 2 x 2 block positions
    assert lib.gbm3d_match(fake, 9, 9, 9, P, 16, fake, None, None, None) == g.EINVAL
    # unsupported parameters
    # (cycle spins 1..4: the level-1 analysis is instantiated for spin shifts 0..3)
    for bad in (dict(patch=12), dict(patch2=4), dict(step2=-1), dict(k1=64), dict(levels=4), dict(k2=12),
                dict(translations=4), dict(cycle_spins=0), dict(cycle_spins=5)):
        q = p.replace(**bad)
        st = lib.gbm3d_match(fake, 64, 64, 64, ctypes.byref(q), 16, fake, None, None, None)
        assert st in (g.EINVAL, g.EUNSUPPORTED), bad
    assert b"" != lib.gbm3d_last_error_string()
    # matching engine: out of range; tensor cores where the window union is too wide
    q = p.replace(match_engine=7)
    assert lib.gbm3d_match(fake, 64, 64, 64, ctypes.byref(q), 16, fake, None, None, None) == g.EINVAL
    q = p.replace(match_engine=3, step=4)  # box sums: s <= 3
    assert lib.gbm3d_match(fake, 64, 64, 64, ctypes.byref(q), 16, fake, None, None, None) == g.EUNSUPPORTED
    q = p.replace(match_engine=4)
    assert lib.gbm3d_match(fake, 64, 64, 64, ctypes.byref(q), 16, fake, None, None, None) == g.EINVAL
    q = p.replace(match_engine=2, search_radius=30)
    assert lib.gbm3d_match(fake, 64, 64, 64, ctypes.byref(q), 16, fake, None, None, None) == g.EUNSUPPORTED
    assert lib.gbm3d_denoise(fake, 64, 64, 64, ctypes.c_float(0.1), ctypes.byref(q), ctypes.c_void_p(0x2000),
                             ctypes.c_void_p(0x4000), None) == g.EUNSUPPORTED
    assert lib.gbm3d_match_stats(None, None) == g.EINVAL
    # misaligned workspace
    assert lib.gbm3d_filter_ht(fake, 64, 64, 64, fake, ctypes.c_float(0.1), P, ctypes.c_void_p(0x3000), fake,
                               ctypes.c_void_p(0x1004), None) == g.EINVAL
    # unsupported group size for aggregation
    assert lib.gbm3d_aggregate(fake, fake, fake, 12, 64, 64, 64, P, ctypes.c_float(0.0), fake, fake,
                               None) == g.EUNSUPPORTED
    # the Wiener filter is built for 8 x 8 blocks: 16 x 16 in stage 2 is refused before any launch
    q = p.replace(patch=16, patch2=16)
    assert lib.gbm3d_denoise(fake, 64, 64, 64, ctypes.c_float(0.1), ctypes.byref(q), ctypes.c_void_p(0x2000),
                             ctypes.c_void_p(0x4000), None) == g.EUNSUPPORTED
    assert lib.gbm3d_filter_wiener(fake, fake, 64, 64, 64, fake, ctypes.c_float(0.1), ctypes.byref(q),
                                   ctypes.c_void_p(0x3000), fake, None, None) == g.EUNSUPPORTED
    # tensor-core matching is for 8 x 8 blocks
    q = g.params_default(1).replace(match_engine=2)
    assert lib.gbm3d_match(fake, 64, 64, 64, ctypes.byref(q), 16, fake, None, None, None) == g.EUNSUPPORTED
    # the image must hold the largest block of the stages
    q = g.params_default(1)
    assert lib.gbm3d_denoise(fake, 12, 64, 64, ctypes.c_float(0.1), ctypes.byref(q), ctypes.c_void_p(0x2000),
                             ctypes.c_void_p(0x4000), None) == g.EINVAL


def test_color_validation(g, no_gpu):
    lib = g.load()
    p = g.params_default()
    P = ctypes.byref(p)
    fake, fake2, ws = ctypes.c_void_p(0x100000), ctypes.c_void_p(0x900000), ctypes.c_void_p(0x2000000)
    sig = ctypes.c_float(0.1)
    # planes overlapping (plane stride below one plane)
    assert lib.gbm3d_denoise_color(fake, 64, 64, 64, 64 * 63, sig, P, fake2, ws, None) == g.EINVAL
    # out overlapping noisy
    assert lib.gbm3d_denoise_color(fake, 64, 64, 64, 64 * 64, sig, P, ctypes.c_void_p(0x100000 + 4 * 64 * 64),
                                   ws, None) == g.EINVAL
    # translations other than 1
    q = p.replace(translations=2)
    assert lib.gbm3d_denoise_color(fake, 64, 64, 64, 64 * 64, sig, ctypes.byref(q), fake2, ws, None) == g.EUNSUPPORTED
    n = ctypes.c_size_t()
    assert lib.gbm3d_workspace_bytes_color(64, 64, ctypes.byref(q), ctypes.byref(n)) == g.EUNSUPPORTED
    # the colour workspace is the grayscale one plus six planes
    assert g.workspace_bytes_color(256, 256) == g.workspace_bytes(256, 256) + 6 * 256 * 256 * 4


def test_empty_image_rejected(g):
    lib = g.load()
    p = g.params_default()
    by, bx = ctypes.c_int(), ctypes.c_int()
    assert lib.gbm3d_grid_dims(0, 0, ctypes.byref(p), ctypes.byref(by), ctypes.byref(bx)) == g.EINVAL
    n = ctypes.c_size_t()
    assert lib.gbm3d_workspace_bytes(0, 64, ctypes.byref(p), ctypes.byref(n)) == g.EINVAL


def test_binding_fails_loudly_without_library(g, monkeypatch, tmp_path):
    from paper_2103_10765_gb300 import build
    monkeypatch.setattr(g, "_lib", None)
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        g.load(build_if_missing=False)


def test_pnp_host_validation(g, no_gpu):
    """Plug-and-play plan arguments are checked on the host before any launch."""
    lib = g.load()
    p = g.params_default()
    shapes = [(128, 136), (64, 72)]
    n = g.pnp_workspace_bytes(shapes, p)
    per = sum(g.workspace_bytes(h, w, p) + 6 * h * w * 4 for h, w in shapes)
    assert n >= per  # plus the transform tables of sides 64, 72, 128, 136
    assert n - per >= 4 * (64 * 64 + 72 * 72 + 128 * 128 + 136 * 136)
    with pytest.raises(g.Gbm3dError):
        g.pnp_workspace_bytes([(100, 64)], p)  # sides must be multiples of 8
    ci, cf, vp = ctypes.c_int, ctypes.c_float, ctypes.c_void_p
    H, W = (ci * 1)(64), (ci * 1)(64)
    ptrs = (vp * 1)(0x1000)
    outs = (vp * 1)(0x2000)
    pitch = (ci * 1)(64)
    sig = (cf * 1)(0.1)
    good = [0.25, 0.5, 1.0, 0.5, 0.25]
    ws = vp(0x10000000)
    big = 1 << 40

    def create(psf=good, q=None, wsb=big, sigma=sig):
        arr = (cf * len(psf))(*psf)
        h = vp()
        return lib.gbm3d_pnp_plan_create(1, H, W, ptrs, pitch, outs, pitch, sigma, arr, len(psf), ctypes.byref(p),
                                         ctypes.byref(q or g.PnpParams()), ws, wsb, None, ctypes.byref(h))
    assert create(psf=[0.5, 0.5]) == g.EINVAL             # even length
    assert create(psf=[0.2, 0.5, 0.3]) == g.EINVAL        # not symmetric
    assert create(q=g.PnpParams(rho=0.0)) == g.EINVAL
    assert create(q=g.PnpParams(iters=0)) == g.EINVAL
    assert create(wsb=1024) == g.ENOMEM
    assert create(sigma=(cf * 1)(-1.0)) == g.EINVAL
    assert lib.gbm3d_pnp_run(None, None) == g.EINVAL
    assert lib.gbm3d_pnp_plan_destroy(None) == g.OK
