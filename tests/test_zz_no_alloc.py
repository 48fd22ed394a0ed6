"""gbm3d_aggregate_noalloc: the aggregation entry point for callers that cannot
allocate device memory (it uses the library's fixed device scratch instead of
a caller-provided workspace).

Checked through the C ABI against gbm3d_aggregate on two calls in a row with
different inputs (the shared scratch keeps the previous call's contents, so
the second call shows that it clears what it must), plus the size limit.
This file is collected last on purpose; it passes alone in a fresh process
and after the other tests."""
import ctypes

import numpy as np
import pytest

from paper_2103_10765_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2103_10765_gb300 import gbm3d  # noqa: E402

ATOL = 1e-4


def _case(H, W, K, seed):
    _, X = synth.make_pair(H, W, 0.1, seed)
    img = torch.from_numpy(X).cuda()
    idx, _ = gbm3d.match(img, K)
    rs = np.random.default_rng(seed)
    groups = torch.from_numpy(rs.random((idx.shape[0], K, 8, 8), dtype=np.float32)).cuda()
    w = torch.from_numpy((rs.random(idx.shape[0]) + 0.1).astype(np.float32)).cuda()
    return groups, w, idx


def _call_noalloc(groups, w, idx, H, W, beta, out):
    lib = gbm3d.load()
    p = gbm3d.params_default()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.gbm3d_aggregate_noalloc(ctypes.c_void_p(groups.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                     ctypes.c_void_p(idx.data_ptr()), idx.shape[1], H, W, out.stride(0),
                                     ctypes.byref(p), ctypes.c_float(beta), ctypes.c_void_p(out.data_ptr()), stream)
    return st


def test_noalloc_matches_workspace_aggregation_twice():
    # a larger image after a smaller one and the reverse, so that both a stale
    # tail and a fresh region of the shared scratch are exercised; 512 x 512
    # with K = 32 fills the fixed scratch to about 85 %
    cases = [(96, 80, 32, 2.0, 1), (61, 77, 16, 0.0, 2), (512, 512, 32, 2.0, 3), (40, 48, 32, 0.0, 4)]
    for H, W, K, beta, seed in cases:
        groups, w, idx = _case(H, W, K, seed)
        want = gbm3d.aggregate(groups, w, idx, H, W, window_beta=beta)
        out = torch.full((H, W), float("nan"), device="cuda")
        assert _call_noalloc(groups, w, idx, H, W, beta, out) == gbm3d.OK
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert float((out - want).abs().max()) <= ATOL


def test_noalloc_rejects_sizes_beyond_its_scratch():
    H = W = 1024
    out = torch.empty((8, 8), device="cuda")  # never written: the call fails before any launch
    groups = w = idx = torch.empty(1, device="cuda")
    lib = gbm3d.load()
    p = gbm3d.params_default()
    st = lib.gbm3d_aggregate_noalloc(ctypes.c_void_p(groups.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                     ctypes.c_void_p(idx.data_ptr()), 32, H, W, W, ctypes.byref(p),
                                     ctypes.c_float(0.0), ctypes.c_void_p(out.data_ptr()), None)
    assert st == gbm3d.ENOMEM
    assert b"fixed" in lib.gbm3d_last_error_string()


def test_noalloc_python_wrapper():
    """The binding's aggregate_noalloc checks its arguments and gives the
    workspace aggregation's result."""
    H, W, K = 72, 64, 16
    groups, w, idx = _case(H, W, K, 5)
    want = gbm3d.aggregate(groups, w, idx, H, W)
    out = gbm3d.aggregate_noalloc(groups, w, idx, H, W, torch.empty((H, W), device="cuda"))
    torch.cuda.synchronize()
    assert float((out - want).abs().max()) <= ATOL
    with pytest.raises(ValueError):
        gbm3d.aggregate_noalloc(groups, w, idx, H, W, torch.empty((H - 1, W), device="cuda"))
    with pytest.raises(ValueError):
        gbm3d.aggregate_noalloc(groups.double(), w, idx, H, W, torch.empty((H, W), device="cuda"))
