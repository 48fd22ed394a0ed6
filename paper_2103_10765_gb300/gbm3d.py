"""Thin Python binding of libgbm3d (the C ABI in include/gbm3d.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Tensors are torch CUDA tensors (torch provides device memory
and the current stream); outputs are allocated here with torch.  There is no
CPU fallback: if the library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = range(6)
_lib = None


class Gbm3dError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"gbm3d status {status}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    """Mirror of gbm3d_params."""
    _fields_ = [(n, ctypes.c_int) for n in
                ("patch", "step", "search_radius", "k1", "k2", "levels", "cycle_spins", "translations", "stages")] + \
               [(n, ctypes.c_float) for n in ("tau_a", "tau_b", "kaiser_beta", "eps_w")] + \
               [(n, ctypes.c_int) for n in ("match_engine", "patch2", "step2")]

    def replace(self, **kw) -> "Params":
        q = Params()
        ctypes.memmove(ctypes.byref(q), ctypes.byref(self), ctypes.sizeof(Params))
        for k, v in kw.items():
            setattr(q, k, v)
        return q

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class PnpParams(ctypes.Structure):
    """Mirror of gbm3d_pnp_params (defaults: 50 iterations, rho 0.1, graph, autotune)."""
    _fields_ = [("iters", ctypes.c_int), ("rho", ctypes.c_float), ("use_graph", ctypes.c_int),
                ("autotune", ctypes.c_int)]

    def __init__(self, iters=50, rho=0.1, use_graph=1, autotune=1):
        super().__init__(iters, rho, use_graph, autotune)


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgbm3d.so (building it first if it is missing and allowed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libgbm3d not built: {path} is missing (run __graft_entry__.build())")
        _build.build_library()
    lib = ctypes.CDLL(path)
    vp, ci, cf, P = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.POINTER(Params)
    lib.gbm3d_params_default.argtypes = [P, ci]
    lib.gbm3d_params_stage.argtypes = [P, ci, P]
    lib.gbm3d_grid_dims.argtypes = [ci, ci, P, ctypes.POINTER(ci), ctypes.POINTER(ci)]
    lib.gbm3d_workspace_bytes.argtypes = [ci, ci, P, ctypes.POINTER(ctypes.c_size_t)]
    lib.gbm3d_match.argtypes = [vp, ci, ci, ci, P, ci, vp, vp, vp, vp]
    lib.gbm3d_filter_ht.argtypes = [vp, ci, ci, ci, vp, cf, P, vp, vp, vp, vp]
    lib.gbm3d_filter_wiener.argtypes = [vp, vp, ci, ci, ci, vp, cf, P, vp, vp, vp, vp]
    lib.gbm3d_aggregate.argtypes = [vp, vp, vp, ci, ci, ci, ci, P, cf, vp, vp, vp]
    lib.gbm3d_denoise.argtypes = [vp, ci, ci, ci, cf, P, vp, vp, vp]
    lib.gbm3d_aggregate_noalloc.argtypes = [vp, vp, vp, ci, ci, ci, ci, P, cf, vp, vp]
    lib.gbm3d_set_match_events.argtypes = [vp]
    lib.gbm3d_measure_fp32_peak.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp]
    lib.gbm3d_workspace_bytes_color.argtypes = [ci, ci, P, ctypes.POINTER(ctypes.c_size_t)]
    lib.gbm3d_denoise_color.argtypes = [vp, ci, ci, ci, ctypes.c_longlong, cf, P, vp, vp, vp]
    lib.gbm3d_match_stats.argtypes = [ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_ulonglong)]
    ip, fpp = ctypes.POINTER(ci), ctypes.POINTER(ctypes.c_void_p)
    lib.gbm3d_pnp_workspace_bytes.argtypes = [ci, ip, ip, P, ctypes.POINTER(ctypes.c_size_t)]
    lib.gbm3d_pnp_plan_create.argtypes = [ci, ip, ip, fpp, ip, fpp, ip, ctypes.POINTER(cf), ctypes.POINTER(cf), ci, P,
                                          ctypes.POINTER(PnpParams), vp, ctypes.c_size_t, vp,
                                          ctypes.POINTER(ctypes.c_void_p)]
    lib.gbm3d_pnp_run.argtypes = [vp, vp]
    lib.gbm3d_pnp_plan_destroy.argtypes = [vp]
    lib.gbm3d_pnp_gemm_config.argtypes = [vp, ci, ip, ip]
    lib.gbm3d_pilot_param_count.argtypes = []
    lib.gbm3d_pilot_workspace_bytes.argtypes = [ci, ci, ci, ci, ctypes.POINTER(ctypes.c_size_t)]
    lib.gbm3d_pilot_forward.argtypes = [vp, ci, ci, ci, vp, vp, vp, vp, vp]
    lib.gbm3d_pilot_loss_grad.argtypes = [vp, vp, ci, ci, ci, vp, vp, vp, vp, vp, vp]
    lib.gbm3d_pilot_train_step.argtypes = [vp, vp, ci, ci, ci, vp, vp, vp, vp, ci, cf, vp, vp, vp]
    lib.gbm3d_workspace_bytes_learned.argtypes = [ci, ci, P, ctypes.POINTER(ctypes.c_size_t)]
    lib.gbm3d_denoise_learned.argtypes = [vp, ci, ci, ci, cf, P, vp, vp, vp, vp]
    lib.gbm3d_last_error_string.restype = ctypes.c_char_p
    lib.gbm3d_version.restype = ctypes.c_char_p
    for name in ("gbm3d_params_default", "gbm3d_params_stage", "gbm3d_grid_dims", "gbm3d_workspace_bytes", "gbm3d_match",
                 "gbm3d_filter_ht", "gbm3d_filter_wiener", "gbm3d_aggregate", "gbm3d_denoise",
                 "gbm3d_aggregate_noalloc", "gbm3d_match_stats", "gbm3d_set_match_events",
                 "gbm3d_workspace_bytes_color", "gbm3d_denoise_color", "gbm3d_pnp_workspace_bytes",
                 "gbm3d_pnp_plan_create", "gbm3d_pnp_run", "gbm3d_pnp_plan_destroy", "gbm3d_pnp_gemm_config",
                 "gbm3d_pilot_param_count", "gbm3d_pilot_workspace_bytes", "gbm3d_pilot_forward",
                 "gbm3d_pilot_loss_grad", "gbm3d_pilot_train_step", "gbm3d_workspace_bytes_learned",
                 "gbm3d_denoise_learned", "gbm3d_measure_fp32_peak"):
        getattr(lib, name).restype = ci
    _lib = lib
    return lib


def _check(status: int):
    if status != OK:
        raise Gbm3dError(status, load().gbm3d_last_error_string().decode())


def params_default(preset: int = 0) -> Params:
    p = Params()
    _check(load().gbm3d_params_default(ctypes.byref(p), preset))
    return p


def params_stage(p: Params, stage: int) -> Params:
    """The block-level parameters of stage 1 or 2 of the whole method
    (gbm3d_params_stage: patch / step set to that stage's block side and stride)."""
    q = Params()
    _check(load().gbm3d_params_stage(ctypes.byref(p), stage, ctypes.byref(q)))
    return q


def grid_dims(H: int, W: int, p: Params | None = None):
    p = p or params_default()
    by, bx = ctypes.c_int(), ctypes.c_int()
    _check(load().gbm3d_grid_dims(H, W, ctypes.byref(p), ctypes.byref(by), ctypes.byref(bx)))
    return by.value, bx.value


def workspace_bytes(H: int, W: int, p: Params | None = None) -> int:
    p = p or params_default()
    n = ctypes.c_size_t()
    _check(load().gbm3d_workspace_bytes(H, W, ctypes.byref(p), ctypes.byref(n)))
    return n.value


def workspace(H: int, W: int, p: Params | None = None, device=None) -> torch.Tensor:
    """Device scratch for any call on an H x W image (torch allocations are 256-byte aligned)."""
    return torch.empty(max(workspace_bytes(H, W, p), 1), dtype=torch.uint8, device=device or "cuda")


def _stream(t: torch.Tensor):
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _img(t: torch.Tensor, name: str):
    if not (t.is_cuda and t.dtype == torch.float32 and t.dim() == 2 and t.stride(1) == 1):
        raise ValueError(f"{name} must be a 2-D float32 CUDA tensor with unit column stride")
    return t.shape[0], t.shape[1], t.stride(0)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def match(img: torch.Tensor, K: int, p: Params | None = None, with_dist: bool = False):
    """Block matching: (idx int32 [G, K], dist float32 [G, K] or None)."""
    p = p or params_default()
    H, W, pitch = _img(img, "img")
    by, bx = grid_dims(H, W, p)
    idx = torch.empty((by * bx, K), dtype=torch.int32, device=img.device)
    dist = torch.empty((by * bx, K), dtype=torch.float32, device=img.device) if with_dist else None
    _check(load().gbm3d_match(_ptr(img), H, W, pitch, ctypes.byref(p), K, _ptr(idx), _ptr(dist), None,
                              _stream(img)))
    return idx, dist


def workspace_bytes_color(H: int, W: int, p: Params | None = None) -> int:
    p = p or params_default()
    n = ctypes.c_size_t()
    _check(load().gbm3d_workspace_bytes_color(H, W, ctypes.byref(p), ctypes.byref(n)))
    return n.value


def denoise_color(noisy: torch.Tensor, sigma: float, p: Params | None = None, ws: torch.Tensor | None = None,
                  out: torch.Tensor | None = None) -> torch.Tensor:
    """Colour G-BM3D of a (3, H, W) float32 CUDA tensor of R, G, B planes
    (rows contiguous; any row pitch and plane stride)."""
    p = p or params_default()
    if not (noisy.is_cuda and noisy.dtype == torch.float32 and noisy.dim() == 3 and noisy.shape[0] == 3
            and noisy.stride(2) == 1):
        raise ValueError("noisy must be a (3, H, W) float32 CUDA tensor with unit column stride")
    _, H, W = noisy.shape
    if ws is None:
        ws = torch.empty(max(workspace_bytes_color(H, W, p), 1), dtype=torch.uint8, device=noisy.device)
    if out is None:  # the same row pitch and plane stride as noisy (one pair for both in the ABI)
        out = torch.empty_strided(noisy.shape, noisy.stride(), dtype=torch.float32, device=noisy.device)
    if out.stride() != noisy.stride() or out.shape != noisy.shape:
        raise ValueError("out must have the shape and strides of noisy")
    _check(load().gbm3d_denoise_color(_ptr(noisy), H, W, noisy.stride(1), noisy.stride(0), float(sigma),
                                      ctypes.byref(p), _ptr(out), _ptr(ws), _stream(noisy)))
    return out


_match_events_keep = None


def set_match_events(events=None):
    """Record 4 torch.cuda.Events around the two matching launches of every
    gbm3d_denoise on this thread (None: off).  events[0..1] bracket stage 1,
    events[2..3] stage 2."""
    global _match_events_keep
    if events is None:
        _match_events_keep = None
        _check(load().gbm3d_set_match_events(None))
        return
    if len(events) != 4:
        raise ValueError("need 4 events")
    arr = (ctypes.c_void_p * 4)(*[ctypes.c_void_p(e.cuda_event) for e in events])
    _match_events_keep = (arr, events)
    _check(load().gbm3d_set_match_events(ctypes.cast(arr, ctypes.c_void_p)))


def measure_fp32_peak(device=None):
    """(scalar, packed) FP32 FMA throughput of the device in TFLOP/s,
    measured by the library's FMA-chain kernels (synchronous)."""
    dev = torch.device(device or "cuda")
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().gbm3d_measure_fp32_peak(ctypes.byref(a), ctypes.byref(b),
                                          ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)))
    return a.value, b.value


def match_stats():
    """(timeouts, rematched) counters of the tensor-core matcher on the current device."""
    t, r = ctypes.c_ulonglong(), ctypes.c_ulonglong()
    _check(load().gbm3d_match_stats(ctypes.byref(t), ctypes.byref(r)))
    return t.value, r.value


def filter_ht(noisy: torch.Tensor, idx: torch.Tensor, sigma: float, p: Params | None = None,
              ws: torch.Tensor | None = None):
    """Stage-1 global hard thresholding: (groups [G, K1, N, N], w [G]), N = p.patch."""
    p = p or params_default()
    H, W, pitch = _img(noisy, "noisy")
    G = idx.shape[0]
    ws = ws if ws is not None else workspace(H, W, p, noisy.device)
    groups = torch.empty((G, p.k1, p.patch, p.patch), dtype=torch.float32, device=noisy.device)
    w = torch.empty(G, dtype=torch.float32, device=noisy.device)
    _check(load().gbm3d_filter_ht(_ptr(noisy), H, W, pitch, _ptr(idx.contiguous()), float(sigma), ctypes.byref(p),
                                  _ptr(groups), _ptr(w), _ptr(ws), _stream(noisy)))
    return groups, w


def filter_wiener(noisy: torch.Tensor, pilot: torch.Tensor, idx: torch.Tensor, sigma: float,
                  p: Params | None = None):
    """Stage-2 empirical Wiener filter: (groups [G, K2, 8, 8], w [G])."""
    p = p or params_default()
    H, W, pitch = _img(noisy, "noisy")
    if _img(pilot, "pilot") != (H, W, pitch):
        raise ValueError("noisy and pilot must share shape and pitch")
    G = idx.shape[0]
    groups = torch.empty((G, p.k2, 8, 8), dtype=torch.float32, device=noisy.device)
    w = torch.empty(G, dtype=torch.float32, device=noisy.device)
    _check(load().gbm3d_filter_wiener(_ptr(noisy), _ptr(pilot), H, W, pitch, _ptr(idx.contiguous()), float(sigma),
                                      ctypes.byref(p), _ptr(groups), _ptr(w), None, _stream(noisy)))
    return groups, w


def aggregate(groups: torch.Tensor, w: torch.Tensor, idx: torch.Tensor, H: int, W: int,
              p: Params | None = None, window_beta: float = 0.0, ws: torch.Tensor | None = None,
              out: torch.Tensor | None = None) -> torch.Tensor:
    """Weighted aggregation of filtered blocks into an H x W image."""
    p = p or params_default()
    K = idx.shape[1]
    out = out if out is not None else torch.empty((H, W), dtype=torch.float32, device=groups.device)
    _, _, pitch = _img(out, "out")
    ws = ws if ws is not None else workspace(H, W, p, groups.device)
    _check(load().gbm3d_aggregate(_ptr(groups.contiguous()), _ptr(w.contiguous()), _ptr(idx.contiguous()), K, H, W,
                                  pitch, ctypes.byref(p), float(window_beta), _ptr(out), _ptr(ws), _stream(groups)))
    return out


def aggregate_noalloc(groups: torch.Tensor, w: torch.Tensor, idx: torch.Tensor, H: int, W: int, out: torch.Tensor,
                      p: Params | None = None, window_beta: float = 0.0) -> torch.Tensor:
    """gbm3d_aggregate_noalloc: aggregation into a caller-provided `out` using
    the library's fixed device scratch (no workspace, no allocation)."""
    p = p or params_default()
    oh, ow, pitch = _img(out, "out")
    if (oh, ow) != (H, W):
        raise ValueError(f"out is {oh} x {ow}, the image {H} x {W}")
    for t, name, dt in ((groups, "groups", torch.float32), (w, "w", torch.float32), (idx, "idx", torch.int32)):
        if t.dtype != dt or t.device != out.device:
            raise ValueError(f"{name} must be a {dt} tensor on {out.device}")
    if idx.dim() != 2 or w.numel() != idx.shape[0] or groups.numel() != idx.numel() * p.patch * p.patch:
        raise ValueError("groups [G, K, N, N], w [G] and idx [G, K] disagree")
    groups, w, idx = groups.contiguous(), w.contiguous(), idx.contiguous()
    _check(load().gbm3d_aggregate_noalloc(_ptr(groups), _ptr(w), _ptr(idx), idx.shape[1], H, W, pitch,
                                          ctypes.byref(p), float(window_beta), _ptr(out), _stream(out)))
    return out


def denoise(noisy: torch.Tensor, sigma: float, p: Params | None = None, ws: torch.Tensor | None = None,
            out: torch.Tensor | None = None) -> torch.Tensor:
    """Two-stage (or stage-1-only) G-BM3D of a device image."""
    p = p or params_default()
    H, W, pitch = _img(noisy, "noisy")
    out = out if out is not None else torch.empty_like(noisy)
    if _img(out, "out")[2] != pitch:
        raise ValueError("out must have the same pitch as noisy")
    ws = ws if ws is not None else workspace(H, W, p, noisy.device)
    _check(load().gbm3d_denoise(_ptr(noisy), H, W, pitch, float(sigma), ctypes.byref(p), _ptr(out), _ptr(ws),
                                _stream(noisy)))
    return out


class HostDenoiser:
    """End-to-end use from host memory: pinned host -> device copy, denoise,
    device -> host copy, on one stream.  Buffers are allocated once per shape.
    channels = 3: colour (R, G, B planes, gbm3d_denoise_color)."""

    def __init__(self, H: int, W: int, p: Params | None = None, device="cuda", channels: int = 1):
        self.p = p or params_default()
        self.H, self.W, self.C = H, W, channels
        shape = (H, W) if channels == 1 else (channels, H, W)
        self.dev_in = torch.empty(shape, dtype=torch.float32, device=device)
        self.dev_out = torch.empty(shape, dtype=torch.float32, device=device)
        self.host_out = torch.empty(shape, dtype=torch.float32, pin_memory=True)
        if channels == 1:
            self.ws = workspace(H, W, self.p, device)
        else:
            n = workspace_bytes_color(H, W, self.p)
            self.ws = torch.empty(max(n, 1), dtype=torch.uint8, device=device)

    @property
    def h2d_bytes(self) -> int:
        return self.C * self.H * self.W * 4

    d2h_bytes = h2d_bytes

    def __call__(self, host_noisy: torch.Tensor, sigma: float) -> torch.Tensor:
        self.dev_in.copy_(host_noisy, non_blocking=True)
        if self.C == 1:
            denoise(self.dev_in, sigma, self.p, self.ws, self.dev_out)
        else:
            denoise_color(self.dev_in, sigma, self.p, self.ws, self.dev_out)
        self.host_out.copy_(self.dev_out, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        return self.host_out


def _int_array(v):
    return (ctypes.c_int * len(v))(*[int(x) for x in v])


def pnp_workspace_bytes(shapes, p: Params | None = None) -> int:
    """Scratch bytes of a plug-and-play plan over images of the given (H, W) shapes."""
    p = p or params_default()
    n = ctypes.c_size_t()
    _check(load().gbm3d_pnp_workspace_bytes(len(shapes), _int_array([h for h, _ in shapes]),
                                            _int_array([w for _, w in shapes]), ctypes.byref(p), ctypes.byref(n)))
    return n.value


class PnpPlan:
    """gbm3d_pnp_plan over a batch of blurred noisy device images ys[i] (2-D
    float32 CUDA tensors, any sizes with sides multiples of 8) with noise
    deviations sigmas[i]; psf is the 1-D factor g of the separable blur
    (odd length, symmetric).  run() executes the whole ADMM loop on the
    current stream; results land in self.outs.  The inputs are bound: write
    new data into ys and call run() again."""

    def __init__(self, ys, sigmas, psf, p: Params | None = None, q: PnpParams | None = None):
        self.p = p or params_default()
        self.q = q or PnpParams()
        self.ys = list(ys)
        dev = self.ys[0].device
        shapes = []
        for y in self.ys:
            shapes.append(_img(y, "y")[:2])
        self.outs = [torch.empty_like(y) for y in self.ys]
        n = len(self.ys)
        nbytes = pnp_workspace_bytes(shapes, self.p)
        self.ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
        g = [float(v) for v in psf]
        H, W = _int_array([h for h, _ in shapes]), _int_array([w for _, w in shapes])
        yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in self.ys])
        op = (ctypes.c_void_p * n)(*[o.data_ptr() for o in self.outs])
        ypitch = _int_array([y.stride(0) for y in self.ys])
        opitch = _int_array([o.stride(0) for o in self.outs])
        sig = (ctypes.c_float * n)(*[float(s) for s in sigmas])
        psf_arr = (ctypes.c_float * len(g))(*g)
        handle = ctypes.c_void_p()
        _check(load().gbm3d_pnp_plan_create(n, H, W, yp, ypitch, op, opitch, sig, psf_arr, len(g),
                                            ctypes.byref(self.p), ctypes.byref(self.q), _ptr(self.ws), nbytes,
                                            _stream(self.ys[0]), ctypes.byref(handle)))
        self._handle = handle

    def run(self):
        _check(load().gbm3d_pnp_run(self._handle, _stream(self.ys[0])))
        return self.outs

    def gemm_configs(self, i: int):
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(load().gbm3d_pnp_gemm_config(self._handle, i, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def close(self):
        if getattr(self, "_handle", None):
            load().gbm3d_pnp_plan_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pilot_param_count() -> int:
    return int(load().gbm3d_pilot_param_count())


def _pilot_ws(B, H, W, train, device):
    n = ctypes.c_size_t()
    _check(load().gbm3d_pilot_workspace_bytes(B, H, W, int(train), ctypes.byref(n)))
    return torch.empty(max(n.value, 1), dtype=torch.uint8, device=device)


class PilotNet:
    """The learned pilot's parameters on the device (theta, FP32) with its
    Adam state.  Batches are (B, H, W) float32 CUDA tensors, sigmas a
    sequence of B noise levels."""

    def __init__(self, theta, device="cuda"):
        theta = torch.as_tensor(theta, dtype=torch.float32)
        if theta.numel() != pilot_param_count():
            raise ValueError(f"theta has {theta.numel()} values, the network {pilot_param_count()}")
        self.theta = theta.to(device).contiguous()
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.step = 0
        self._ws = {}

    def _workspace(self, shape, train):
        key = (tuple(shape), bool(train))
        if key not in self._ws:
            self._ws[key] = _pilot_ws(*shape, train, self.theta.device)
        return self._ws[key]

    @staticmethod
    def _batch(Z):
        if not (Z.is_cuda and Z.dtype == torch.float32 and Z.dim() == 3 and Z.is_contiguous()):
            raise ValueError("a batch is a contiguous (B, H, W) float32 CUDA tensor")
        return Z.shape

    def _sig(self, sigmas, B):
        s = torch.as_tensor(list(sigmas), dtype=torch.float32).to(self.theta.device)
        if s.numel() != B:
            raise ValueError("one sigma per image")
        return s

    def forward(self, Z, sigmas):
        B, H, W = self._batch(Z)
        s = self._sig(sigmas, B)
        out = torch.empty_like(Z)
        _check(load().gbm3d_pilot_forward(_ptr(Z), B, H, W, _ptr(s), _ptr(self.theta), _ptr(out),
                                          _ptr(self._workspace((B, H, W), False)), _stream(Z)))
        return out

    def loss_grad(self, Z, Y1, sigmas):
        B, H, W = self._batch(Z)
        s = self._sig(sigmas, B)
        grad = torch.empty_like(self.theta)
        loss = torch.empty(1, dtype=torch.float32, device=Z.device)
        _check(load().gbm3d_pilot_loss_grad(_ptr(Z), _ptr(Y1.contiguous()), B, H, W, _ptr(s), _ptr(self.theta),
                                            _ptr(grad), _ptr(loss), _ptr(self._workspace((B, H, W), True)),
                                            _stream(Z)))
        return loss, grad

    def train_step(self, Z, Y1, sigmas, lr=1e-3):
        """One Adam step; returns the loss before it (device scalar)."""
        B, H, W = self._batch(Z)
        s = self._sig(sigmas, B)
        self.step += 1
        loss = torch.empty(1, dtype=torch.float32, device=Z.device)
        _check(load().gbm3d_pilot_train_step(_ptr(Z), _ptr(Y1.contiguous()), B, H, W, _ptr(s), _ptr(self.theta),
                                             _ptr(self.m), _ptr(self.v), self.step, float(lr), _ptr(loss),
                                             _ptr(self._workspace((B, H, W), True)), _stream(Z)))
        return loss


def workspace_bytes_learned(H: int, W: int, p: Params | None = None) -> int:
    p = p or params_default()
    n = ctypes.c_size_t()
    _check(load().gbm3d_workspace_bytes_learned(H, W, ctypes.byref(p), ctypes.byref(n)))
    return n.value


def denoise_learned(noisy: torch.Tensor, sigma: float, net: PilotNet, p: Params | None = None,
                    ws: torch.Tensor | None = None, out: torch.Tensor | None = None) -> torch.Tensor:
    """Stage 2 with the learned pilot in place of stage 1."""
    p = p or params_default()
    H, W, pitch = _img(noisy, "noisy")
    out = out if out is not None else torch.empty_like(noisy)
    if ws is None:
        ws = torch.empty(max(workspace_bytes_learned(H, W, p), 1), dtype=torch.uint8, device=noisy.device)
    _check(load().gbm3d_denoise_learned(_ptr(noisy), H, W, pitch, float(sigma), ctypes.byref(p), _ptr(net.theta),
                                        _ptr(out), _ptr(ws), _stream(noisy)))
    return out
