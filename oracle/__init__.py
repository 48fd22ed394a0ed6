"""FP64 CPU oracle for the G-BM3D hot path (arXiv 2103.10765).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The CUDA library and its
Python binding never import this package.  The arithmetic lives in
``gbm3d_oracle.c`` (plain C, double precision); this module compiles it with
gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gbm3d_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_gbm3d.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available).  Returns the .so path."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _get():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


class _Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in
                ("patch", "step", "search_radius", "k1", "k2", "levels", "cycle_spins", "translations", "stages")] + \
               [(n, ctypes.c_double) for n in ("tau_a", "tau_b", "kaiser_beta", "eps_w")] + \
               [(n, ctypes.c_int) for n in ("patch2", "step2")]


def _declare(lib):
    c_int, c_double, vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    lib.orc_grid.argtypes = [c_int, c_int, c_int, vp]
    lib.orc_grid.restype = c_int
    lib.orc_patch_dist.argtypes = [_f64p, c_int, c_int, c_int, c_int, c_int, c_int, c_int]
    lib.orc_patch_dist.restype = c_double
    lib.orc_match_refs.argtypes = [_f64p, c_int, c_int, c_int, c_int, c_int, _i32p, _i32p, c_int, _i32p, vp, c_int]
    lib.orc_match.argtypes = [_f64p, c_int, c_int, c_int, c_int, c_int, c_int, _i32p, vp, c_int]
    lib.orc_bior15_filters.argtypes = [vp, vp]
    lib.orc_bior15_filters.restype = None
    lib.orc_dwt1.argtypes = [_f64p, c_int, c_int, _f64p, _f64p]
    lib.orc_idwt1.argtypes = [_f64p, _f64p, c_int, c_int, _f64p]
    lib.orc_upsilon.argtypes = [c_double, c_double]
    lib.orc_upsilon.restype = c_double
    lib.orc_dwt3.argtypes = [_f64p, c_int, c_int, c_int, c_int, vp, c_int]
    lib.orc_idwt3.argtypes = [_f64p, c_int, c_int, c_int, c_int, c_int]
    lib.orc_filter_ht.argtypes = [_f64p, c_int, c_int, _i32p, c_int, c_int, c_int, c_int, c_double, c_int, c_int,
                                  c_double, c_double, c_double, _f64p, _f64p, c_int]
    lib.orc_tv_weights.argtypes = [_f64p, c_int, c_int, c_int, c_double, _f64p]
    lib.orc_dct2.argtypes = [_f64p, c_int, c_int]
    lib.orc_haar.argtypes = [_f64p, c_int, c_int]
    lib.orc_filter_wiener.argtypes = [_f64p, _f64p, c_int, c_int, _i32p, c_int, c_int, c_int, c_double, c_double,
                                      _f64p, _f64p, c_int]
    lib.orc_bessel_i0.argtypes = [c_double]
    lib.orc_bessel_i0.restype = c_double
    lib.orc_kaiser.argtypes = [c_int, c_double, _f64p]
    lib.orc_aggregate.argtypes = [_f64p, _f64p, _i32p, c_int, c_int, c_int, c_int, c_int, c_double, _f64p, c_int]
    lib.orc_denoise.argtypes = [_f64p, c_int, c_int, c_double, ctypes.POINTER(_Params), _f64p, vp, c_int]
    lib.orc_max_threads.argtypes = []
    lib.orc_opp.argtypes = [_f64p, ctypes.c_size_t, c_int, _f64p]
    lib.orc_opp_sigma_scale.argtypes = [c_int]
    lib.orc_opp_sigma_scale.restype = c_double
    lib.orc_denoise_color.argtypes = [_f64p, c_int, c_int, c_double, ctypes.POINTER(_Params), _f64p, c_int]


class OracleError(RuntimeError):
    pass


def _check(st, what):
    if st != 0:
        raise OracleError(f"{what} failed with status {st}")


@dataclass
class Params:
    """Method parameters (field meaning as in the C-ABI's gbm3d_params)."""
    patch: int = 8
    step: int = 3
    search_radius: int = 19
    k1: int = 16
    k2: int = 32
    levels: int = 3
    cycle_spins: int = 2
    translations: int = 1
    stages: int = 2
    tau_a: float = 3.6
    tau_b: float = 0.3
    kaiser_beta: float = 2.0
    eps_w: float = 1e-8
    patch2: int = 0  # stage-2 block side (0: patch)
    step2: int = 0   # stage-2 grid stride (0: step)

    @classmethod
    def paper(cls) -> "Params":
        """The Sec. 5 parameter list: N = 16 tiling blocks in stage 1, N = 8 in
        stage 2 (s = N in both), a 32-pixel search window read as R = 16,
        K = 16 in both stages, 3 levels, 2 cycle spins, 2 translations."""
        return cls(patch=16, step=16, search_radius=16, k1=16, k2=16, translations=2, patch2=8, step2=8)

    def c(self):
        return _Params(self.patch, self.step, self.search_radius, self.k1, self.k2, self.levels, self.cycle_spins,
                       self.translations, self.stages, self.tau_a, self.tau_b, self.kaiser_beta, self.eps_w,
                       self.patch2, self.step2)


def max_threads() -> int:
    return int(_get().orc_max_threads())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def grid(M: int, N: int, s: int) -> np.ndarray:
    lib = _get()
    n = lib.orc_grid(M, N, s, None)
    out = np.zeros(max(n, 1), dtype=np.int32)
    lib.orc_grid(M, N, s, out.ctypes.data_as(ctypes.c_void_p))
    return out[:n]


def patch_dist(X, N, i, j, k, l) -> float:
    X = _f64(X)
    return float(_get().orc_patch_dist(X, X.shape[0], X.shape[1], N, i, j, k, l))


def match(X, N=8, s=3, R=19, K=16, nthreads=1):
    """(idx[By*Bx, K] int32, dist[By*Bx, K] float64) for every grid reference."""
    X = _f64(X)
    H, W = X.shape
    By, Bx = len(grid(H, N, s)), len(grid(W, N, s))
    idx = np.zeros((By * Bx, K), dtype=np.int32)
    dist = np.zeros((By * Bx, K), dtype=np.float64)
    _check(_get().orc_match(X, H, W, N, s, R, K, idx, dist.ctypes.data_as(ctypes.c_void_p), nthreads), "orc_match")
    return idx, dist


def match_refs(X, refs_i, refs_j, N=8, R=19, K=16, nthreads=1):
    X = _f64(X)
    H, W = X.shape
    ri = np.ascontiguousarray(refs_i, dtype=np.int32)
    rj = np.ascontiguousarray(refs_j, dtype=np.int32)
    idx = np.zeros((len(ri), K), dtype=np.int32)
    dist = np.zeros((len(ri), K), dtype=np.float64)
    _check(_get().orc_match_refs(X, H, W, N, R, K, ri, rj, len(ri), idx, dist.ctypes.data_as(ctypes.c_void_p),
                                 nthreads), "orc_match_refs")
    return idx, dist


def bior15_filters():
    h0 = np.zeros(10)
    g1 = np.zeros(10)
    _get().orc_bior15_filters(h0.ctypes.data_as(ctypes.c_void_p), g1.ctypes.data_as(ctypes.c_void_p))
    return h0, g1


HAAR, BIOR15 = 0, 1


def dwt1(x, kind=BIOR15):
    x = _f64(x)
    lo = np.zeros(len(x) // 2)
    hi = np.zeros(len(x) // 2)
    _check(_get().orc_dwt1(x, len(x), kind, lo, hi), "orc_dwt1")
    return lo, hi


def idwt1(lo, hi, kind=BIOR15):
    lo, hi = _f64(lo), _f64(hi)
    x = np.zeros(2 * len(lo))
    _check(_get().orc_idwt1(lo, hi, 2 * len(lo), kind, x), "orc_idwt1")
    return x


def upsilon(a, lam):
    return float(_get().orc_upsilon(float(a), float(lam)))


def dwt3(v, L=3, tau=None, nthreads=1):
    """Forward 3-D transform of v[y][x][z] (Mallat layout), thresholded if tau given."""
    v = _f64(v).copy()
    Y, X, Z = v.shape
    tp = None
    if tau is not None:
        t = _f64(tau)
        tp = t.ctypes.data_as(ctypes.c_void_p)
    _check(_get().orc_dwt3(v, Y, X, Z, L, tp, nthreads), "orc_dwt3")
    return v


def idwt3(v, L=3, nthreads=1):
    v = _f64(v).copy()
    Y, X, Z = v.shape
    _check(_get().orc_idwt3(v, Y, X, Z, L, nthreads), "orc_idwt3")
    return v


def filter_ht(Z, idx, sigma, By, Bx, N=8, K=16, L=3, C=2, tau_a=3.6, tau_b=0.3, eps_w=1e-8, nthreads=1):
    Z = _f64(Z)
    H, W = Z.shape
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    groups = np.zeros((By * Bx, K, N, N))
    w = np.zeros(By * Bx)
    _check(_get().orc_filter_ht(Z, H, W, idx, By, Bx, N, K, float(sigma), L, C, tau_a, tau_b, eps_w, groups, w,
                                nthreads), "orc_filter_ht")
    return groups, w


def tv_weights(groups, eps_w=1e-8):
    """w[g] = 1 / max(TV(groups[g]), eps_w) for groups [G, K, N, N] (the
    stage-1 weight rule of orc_filter_ht)."""
    groups = _f64(groups)
    G, K, N = groups.shape[0], groups.shape[1], groups.shape[2]
    w = np.zeros(G)
    _check(_get().orc_tv_weights(groups, G, K, N, float(eps_w), w), "orc_tv_weights")
    return w


def dct2(blk, inverse=False):
    b = _f64(blk).copy()
    _check(_get().orc_dct2(b, b.shape[0], int(inverse)), "orc_dct2")
    return b


def haar(x, inverse=False):
    x = _f64(x).copy()
    _check(_get().orc_haar(x, len(x), int(inverse)), "orc_haar")
    return x


def filter_wiener(Z, Yp, idx, sigma, N=8, K=32, eps_w=1e-8, nthreads=1):
    Z, Yp = _f64(Z), _f64(Yp)
    H, W = Z.shape
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    G = idx.size // K
    groups = np.zeros((G, K, N, N))
    w = np.zeros(G)
    _check(_get().orc_filter_wiener(Z, Yp, H, W, idx, G, N, K, float(sigma), eps_w, groups, w, nthreads),
           "orc_filter_wiener")
    return groups, w


def bessel_i0(x):
    return float(_get().orc_bessel_i0(float(x)))


def kaiser(N, beta):
    out = np.zeros(N)
    _check(_get().orc_kaiser(N, float(beta), out), "orc_kaiser")
    return out


def aggregate(groups, w, idx, H, W, N=8, beta=0.0, require_cover=True):
    """Weighted aggregation; with require_cover=False pixels that no block
    covers are 0 instead of an error (aggregating a subset of the groups)."""
    groups = _f64(groups)
    w = _f64(w)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    G = w.size
    K = idx.size // G
    out = np.zeros((H, W))
    _check(_get().orc_aggregate(groups, w, idx, G, K, H, W, N, float(beta), out, int(require_cover)),
           "orc_aggregate")
    return out


def denoise(Z, sigma, params: Params | None = None, nthreads=1, return_y1=False):
    params = params or Params()
    Z = _f64(Z)
    H, W = Z.shape
    out = np.zeros((H, W))
    y1 = np.zeros((H, W))
    p = params.c()
    _check(_get().orc_denoise(Z, H, W, float(sigma), ctypes.byref(p), out, y1.ctypes.data_as(ctypes.c_void_p),
                              nthreads), "orc_denoise")
    return (out, y1) if return_y1 else out


def opp(x, inverse=False):
    """Opponent colour transform of a (3, H, W) array (reading C1), or its inverse."""
    x = _f64(x)
    y = np.zeros_like(x)
    _check(_get().orc_opp(x, x[0].size, int(inverse), y), "orc_opp")
    return y


def opp_sigma_scale(c: int) -> float:
    """Noise deviation of opponent channel c per unit deviation in R, G, B (reading C2)."""
    return float(_get().orc_opp_sigma_scale(c))


def denoise_color(Z, sigma, params: Params | None = None, nthreads=1):
    """Colour G-BM3D of a (3, H, W) RGB array (readings C1-C4)."""
    params = params or Params()
    Z = _f64(Z)
    _, H, W = Z.shape
    out = np.zeros_like(Z)
    p = params.c()
    _check(_get().orc_denoise_color(Z, H, W, float(sigma), ctypes.byref(p), out, nthreads), "orc_denoise_color")
    return out


def psnr(x, ref) -> float:
    """10 log10(1 / MSE) for images with peak 1 (no clipping)."""
    mse = float(np.mean((np.asarray(x, np.float64) - np.asarray(ref, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)
