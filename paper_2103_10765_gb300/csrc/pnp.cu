// pnp.cu -- plug-and-play ADMM deconvolution with G-BM3D as the denoiser,
// for a batch of images of uneven sizes (Sec. 1: plug-and-play priors couple
// a denoiser with inverse problems such as deconvolution, one denoiser call
// per iteration; Sec. 6: real-time plug-and-play use).
//
// Per image, with y = h * x + n (circular blur by a separable, symmetric
// point-spread function h = g g^T) and fixed penalty rho:
//   x <- (H^T H + rho I)^-1 (H^T y + rho (v - u))
//   v <- G-BM3D(x + u, sigma_n / sqrt(rho))
//   u <- u + x - v
// starting from v = y, u = 0; the result is v.
//
// x-update.  For an even 1-D kernel g, circular convolution along one axis
// is diagonal in the discrete Hartley basis cas(2 pi k n / N) = cos + sin,
// with the real eigenvalues lam_N[k] = sum_t g[t] cos(2 pi k t / N); the
// separable transform T(X) = C_H X C_W (C_N[k][n] = cas(2 pi k n / N),
// symmetric, C_N C_N = N I) therefore diagonalises the 2-D blur, and
//   x = T( T(b) / ((lam_H[k] lam_W[l])^2 + rho) ) / (H W).
// Each T is two dense FP32 matrix products, so any image size works (sizes
// with large prime factors included) at 8 H W (H + W) FLOP per x-update.
// The products run in a register-tiled SIMT kernel; an autotuner times four
// tile shapes per (M, N, K) on the plan's own buffers and keeps the fastest.
//
// Per iteration and image: 4 products (the eigenvalue division and the
// "x + u" of the denoiser input fused into their epilogues), one G-BM3D
// denoise, and one update kernel (u' = t - v with t = x + u; b = H^T y +
// rho (2 v - t), the next iteration's right-hand side).  With use_graph the
// plan captures one iteration of every image, each on its own stream
// branch, as a CUDA graph and replays it `iters` times; without it the same
// launches run image after image on the caller's stream.  Both give the same
// bits.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <tuple>
#include <vector>

#include "internal.cuh"

namespace gbm3d {
namespace {

// ---- dense FP32 products ---------------------------------------------------
// C = epilogue(A[M][K] B[K][N]), row-major with leading dimensions.  CTA tile
// BM x BN, 256 threads as 16 x 16, each with a TM x TN micro-tile split in two
// halves (rows ty*TM/2 + i and BM/2 + ty*TM/2 + i, likewise columns) so that
// the shared-memory reads of a half-warp are contiguous.  BK = 8, one tile of
// A and B prefetched into registers while the current one is multiplied.
struct Epi {
    int mode;              // 0: alpha acc; 1: acc / ((lamM[r] lamN[c])^2 + rho); 2: alpha acc + add[r][c]
    float alpha, rho;
    const float *lamM, *lamN;
    const float *add;
    int ldadd;
};

template <int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__(256)
k_sgemm(const float *__restrict__ A, int lda, const float *__restrict__ B, int ldb, float *__restrict__ C, int ldc,
        int M, int N, int K, Epi epi)
{
    constexpr int BK = 8, HM = TM / 2, HN = TN / 2;
    constexpr int LA = BM * BK / 256, LB = BN * BK / 256; // elements each thread loads per tile
    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Bs[2][BK][BN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    // load maps: A as BM rows of BK/LA groups; B as BK rows of BN/LB groups
    const int ar = tid / (BK / LA), ak = (tid % (BK / LA)) * LA;
    const int bk = tid / (BN / LB), bn = (tid % (BN / LB)) * LB;
    float ra[LA], rb[LB];
    auto load = [&](int k0) {
#pragma unroll
        for (int i = 0; i < LA; i++) {
            const int r = m0 + ar, k = k0 + ak + i;
            ra[i] = (r < M && k < K) ? __ldg(A + (size_t)r * lda + k) : 0.f;
        }
#pragma unroll
        for (int i = 0; i < LB; i++) {
            const int k = k0 + bk, c = n0 + bn + i;
            rb[i] = (k < K && c < N) ? __ldg(B + (size_t)k * ldb + c) : 0.f;
        }
    };
    auto store = [&](int s) {
#pragma unroll
        for (int i = 0; i < LA; i++) As[s][ak + i][ar] = ra[i];
#pragma unroll
        for (int i = 0; i < LB; i++) Bs[s][bk][bn + i] = rb[i];
    };
    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; i++)
#pragma unroll
        for (int j = 0; j < TN; j++) acc[i][j] = 0.f;
    load(0);
    store(0);
    __syncthreads();
    const int nk = (K + BK - 1) / BK;
    for (int t = 0; t < nk; t++) {
        const int s = t & 1;
        if (t + 1 < nk) load((t + 1) * BK);
#pragma unroll
        for (int k = 0; k < BK; k++) {
            float a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < HM; i++) {
                a[i] = As[s][k][ty * HM + i];
                a[HM + i] = As[s][k][BM / 2 + ty * HM + i];
            }
#pragma unroll
            for (int j = 0; j < HN; j++) {
                b[j] = Bs[s][k][tx * HN + j];
                b[HN + j] = Bs[s][k][BN / 2 + tx * HN + j];
            }
#pragma unroll
            for (int i = 0; i < TM; i++)
#pragma unroll
                for (int j = 0; j < TN; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (t + 1 < nk) {
            store(s ^ 1);
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < TM; i++) {
        const int r = m0 + (i < HM ? ty * HM + i : BM / 2 + ty * HM + (i - HM));
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; j++) {
            const int c = n0 + (j < HN ? tx * HN + j : BN / 2 + tx * HN + (j - HN));
            if (c >= N) continue;
            float v = acc[i][j];
            if (epi.mode == 1) {
                const float l = __ldg(epi.lamM + r) * __ldg(epi.lamN + c);
                v = v / fmaf(l, l, epi.rho);
            } else if (epi.mode == 2) {
                v = fmaf(epi.alpha, v, __ldg(epi.add + (size_t)r * epi.ldadd + c));
            } else {
                v *= epi.alpha;
            }
            C[(size_t)r * ldc + c] = v;
        }
    }
}

struct GemmCfg {
    int bm, bn;
    void (*fn)(const float *, int, const float *, int, float *, int, int, int, int, Epi);
};

const GemmCfg kGemmCfgs[] = {
    {128, 128, k_sgemm<128, 128, 8, 8>},
    {128, 64, k_sgemm<128, 64, 8, 4>},
    {64, 128, k_sgemm<64, 128, 4, 8>},
    {64, 64, k_sgemm<64, 64, 4, 4>},
};
constexpr int kNumCfgs = sizeof(kGemmCfgs) / sizeof(kGemmCfgs[0]);

cudaError_t gemm(int cfg, const float *A, int lda, const float *B, int ldb, float *C, int ldc, int M, int N, int K,
                 const Epi &epi, cudaStream_t st)
{
    const GemmCfg &g = kGemmCfgs[cfg];
    dim3 grid((N + g.bn - 1) / g.bn, (M + g.bm - 1) / g.bm);
    g.fn<<<grid, 256, 0, st>>>(A, lda, B, ldb, C, ldc, M, N, K, epi);
    return cudaGetLastError();
}

// ---- transform tables -------------------------------------------------------
// C_N[k][n] = cas(2 pi k n / N) with the product k n reduced mod N exactly.
__global__ void k_cas(int N, float *__restrict__ C)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)N * N) return;
    const int k = (int)(e / N), n = (int)(e - (long long)k * N);
    const int r = (int)(((long long)k * n) % N);
    float s, c;
    sincospif(2.f * (float)r / (float)N, &s, &c);
    C[e] = c + s;
}

// lam_N[k] = g[0] + 2 sum_{t=1..R} g[t] cos(2 pi k t / N): the Hartley (= DFT,
// g being even) eigenvalues of circular convolution with g along an axis of N.
__global__ void k_lambda(int N, const float *__restrict__ g, int R, float *__restrict__ lam)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    float acc = g[0];
    for (int t = 1; t <= R; t++) {
        const int r = (int)(((long long)k * t) % N);
        acc = fmaf(2.f * g[t], cospif(2.f * (float)r / (float)N), acc);
    }
    lam[k] = acc;
}

// ---- elementwise ------------------------------------------------------------
// Circular convolution with the even kernel g (taps g[0..R], g[-t] = g[t])
// along rows (axis 0: out[i][j] = sum_t g[t] in[i][j - t]) or columns.
__global__ void k_conv1(const float *__restrict__ src, int sp, float *__restrict__ dst, int dp, int H, int W,
                        const float *__restrict__ g, int R, int axis)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= W || y >= H) return;
    float acc = g[0] * src[(size_t)y * sp + x];
    for (int t = 1; t <= R; t++) {
        float a, b;
        if (axis == 0) {
            int xm = x - t, xp = x + t;
            xm = ((xm % W) + W) % W;
            xp %= W;
            a = src[(size_t)y * sp + xm];
            b = src[(size_t)y * sp + xp];
        } else {
            int ym = y - t, yp = y + t;
            ym = ((ym % H) + H) % H;
            yp %= H;
            a = src[(size_t)ym * sp + x];
            b = src[(size_t)yp * sp + x];
        }
        acc = fmaf(g[t], a + b, acc);
    }
    dst[(size_t)y * dp + x] = acc;
}

// Start: v = y, u = 0, b = H^T y + rho y.
__global__ void k_pnp_init(const float *__restrict__ y, int yp, const float *__restrict__ hty, float *__restrict__ v,
                           float *__restrict__ u, float *__restrict__ b, int H, int W, float rho)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31), r = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= W || r >= H) return;
    const size_t e = (size_t)r * W + x;
    const float yv = y[(size_t)r * yp + x];
    v[e] = yv;
    u[e] = 0.f;
    b[e] = fmaf(rho, yv, hty[e]);
}

// After the denoiser: u = t - v (t = x + u_old), b = H^T y + rho (v - u).
__global__ void k_pnp_update(const float *__restrict__ t, const float *__restrict__ v, const float *__restrict__ hty,
                             float *__restrict__ u, float *__restrict__ b, long long n, float rho)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float vv = v[e], un = t[e] - vv;
    u[e] = un;
    b[e] = fmaf(rho, vv - un, hty[e]);
}

__global__ void k_copy2d(const float *__restrict__ src, int sp, float *__restrict__ dst, int dp, int H, int W)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= W || y >= H) return;
    dst[(size_t)y * dp + x] = src[(size_t)y * sp + x];
}

} // namespace
} // namespace gbm3d

// ---- host side ----------------------------------------------------------------
namespace gbm3d {
namespace {

constexpr int kMaxPsf = 63; // longest 1-D factor of the point-spread function

struct PnpImage {
    int H, W, ypitch, opitch;
    float sigma_d;
    const float *y;
    float *out;
    char *dws;                          // denoiser workspace
    float *hty, *b, *t1, *t, *u, *v;    // H x W planes, pitch W
    const float *casH, *casW, *lamH, *lamW;
    int cfg1, cfg2;                     // GEMM tile shape for K = H and for K = W
};

size_t plane_bytes(int H, int W) { return align_up((size_t)H * W * sizeof(float)); }

// Distinct transform sizes of the batch, ascending.
std::vector<int> distinct_sizes(int n, const int *H, const int *W)
{
    std::map<int, int> m;
    for (int i = 0; i < n; i++) m[H[i]] = m[W[i]] = 1;
    std::vector<int> v;
    for (auto &kv : m) v.push_back(kv.first);
    return v;
}

size_t tables_bytes(const std::vector<int> &sizes)
{
    size_t o = align_up(kMaxPsf * sizeof(float)); // the kernel's half g[0..R]
    for (int N : sizes) o += align_up((size_t)N * N * sizeof(float)) + align_up((size_t)N * sizeof(float));
    return o;
}

// Fastest tile shape per (M, N, K), cached for the process (all shapes give
// the same bits: every output is the same sequential FMA chain over k).
std::map<std::tuple<int, int, int>, int> g_tuned;

int autotune(const float *A, const float *B, float *C, int M, int N, int K, cudaStream_t st, bool enabled)
{
    if (!enabled) return 0;
    const auto key = std::make_tuple(M, N, K);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) return it->second;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return 0;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return 0;
    }
    Epi epi{0, 1.f, 0.f, nullptr, nullptr, nullptr, 0};
    int best = 0;
    float best_ms = 1e30f;
    for (int c = 0; c < kNumCfgs; c++) {
        if (gemm(c, A, K, B, N, C, N, M, N, K, epi, st) != cudaSuccess) continue; // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3; r++) gemm(c, A, K, B, N, C, N, M, N, K, epi, st);
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) continue;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g_tuned[key] = best;
    return best;
}

void launch_grid(dim3 &grid, int H, int W) { grid = dim3((W + 31) / 32, (H + 7) / 8); }

} // namespace
} // namespace gbm3d

using namespace gbm3d;

struct gbm3d_pnp_plan_st {
    std::vector<PnpImage> img;
    gbm3d_params p;
    gbm3d_pnp_params q;
    const float *g; // device, g[0..R]
    int R;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaStream_t origin = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

int pnp_fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return set_error(code, buf);
}

int pnp_cuda_fail(cudaError_t e, const char *where)
{
    return pnp_fail(GBM3D_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// One ADMM iteration of image m on stream st (readings in the file header).
int pnp_iteration(const gbm3d_pnp_plan_st &P, const PnpImage &m, cudaStream_t st)
{
    const int H = m.H, W = m.W;
    const float rho = P.q.rho;
    const Epi plain{0, 1.f, 0.f, nullptr, nullptr, nullptr, 0};
    const Epi divide{1, 1.f, rho, m.lamH, m.lamW, nullptr, 0};
    const Epi finish{2, 1.f / ((float)H * (float)W), 0.f, nullptr, nullptr, m.u, W};
    cudaError_t e;
    // T(b) = C_H b C_W, divided by the eigenvalues, transformed back (+ u)
    if ((e = gemm(m.cfg1, m.casH, H, m.b, W, m.t1, W, H, W, H, plain, st)) != cudaSuccess) return pnp_cuda_fail(e, "pnp gemm");
    if ((e = gemm(m.cfg2, m.t1, W, m.casW, W, m.b, W, H, W, W, divide, st)) != cudaSuccess) return pnp_cuda_fail(e, "pnp gemm");
    if ((e = gemm(m.cfg1, m.casH, H, m.b, W, m.t1, W, H, W, H, plain, st)) != cudaSuccess) return pnp_cuda_fail(e, "pnp gemm");
    if ((e = gemm(m.cfg2, m.t1, W, m.casW, W, m.t, W, H, W, W, finish, st)) != cudaSuccess) return pnp_cuda_fail(e, "pnp gemm");
    // v = G-BM3D(x + u)
    int s = gbm3d_denoise(m.t, H, W, W, m.sigma_d, &P.p, m.v, m.dws, (gbm3d_stream_t)st);
    if (s != GBM3D_OK) return s;
    const long long n = (long long)H * W;
    k_pnp_update<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m.t, m.v, m.hty, m.u, m.b, n, rho);
    if ((e = cudaGetLastError()) != cudaSuccess) return pnp_cuda_fail(e, "pnp update");
    return GBM3D_OK;
}

int check_pnp_args(int n, const int *H, const int *W, const gbm3d_params *p, const float *psf, int psf_len,
                   const gbm3d_pnp_params *q)
{
    if (n < 1 || !H || !W || !p) return pnp_fail(GBM3D_EINVAL, "pnp: n >= 1 and non-null H, W, params required");
    if (q) {
        if (q->iters < 1) return pnp_fail(GBM3D_EINVAL, "pnp: iters %d < 1", q->iters);
        if (!(q->rho > 0.f) || !isfinite(q->rho)) return pnp_fail(GBM3D_EINVAL, "pnp: rho must be positive");
    }
    if (psf) {
        if (psf_len < 1 || psf_len > kMaxPsf || !(psf_len & 1))
            return pnp_fail(GBM3D_EINVAL, "pnp: psf length %d: odd, 1..%d", psf_len, kMaxPsf);
        const int R = psf_len / 2;
        for (int t = 0; t <= R; t++)
            if (!isfinite(psf[R + t]) || psf[R + t] != psf[R - t])
                return pnp_fail(GBM3D_EINVAL, "pnp: the psf factor must be finite and symmetric");
    }
    for (int i = 0; i < n; i++) {
        if (H[i] % 8 || W[i] % 8)
            return pnp_fail(GBM3D_EINVAL, "pnp: image %d is %dx%d; sides must be multiples of 8", i, H[i], W[i]);
        size_t b = 0;
        const int st = gbm3d_workspace_bytes(H[i], W[i], p, &b);
        if (st != GBM3D_OK) return st;
    }
    return GBM3D_OK;
}

} // namespace

extern "C" {

int gbm3d_pnp_workspace_bytes(int n, const int *H, const int *W, const gbm3d_params *p, size_t *bytes)
{
    int st = check_pnp_args(n, H, W, p, nullptr, 0, nullptr);
    if (st) return st;
    if (!bytes) return pnp_fail(GBM3D_EINVAL, "pnp: bytes is NULL");
    size_t o = tables_bytes(distinct_sizes(n, H, W));
    for (int i = 0; i < n; i++) {
        size_t b = 0;
        gbm3d_workspace_bytes(H[i], W[i], p, &b);
        o += align_up(b) + 6 * plane_bytes(H[i], W[i]);
    }
    *bytes = o;
    return GBM3D_OK;
}

int gbm3d_pnp_plan_create(int n, const int *H, const int *W, const float *const *y, const int *ypitch,
                          float *const *out, const int *opitch, const float *sigma, const float *psf, int psf_len,
                          const gbm3d_params *p, const gbm3d_pnp_params *q, void *ws, size_t ws_bytes,
                          gbm3d_stream_t stream, gbm3d_pnp_plan *plan)
{
    if (!plan) return pnp_fail(GBM3D_EINVAL, "pnp: plan is NULL");
    *plan = nullptr;
    if (!q || !psf || !y || !ypitch || !out || !opitch || !sigma || !ws)
        return pnp_fail(GBM3D_EINVAL, "pnp: null argument");
    int st = check_pnp_args(n, H, W, p, psf, psf_len, q);
    if (st) return st;
    size_t need = 0;
    if ((st = gbm3d_pnp_workspace_bytes(n, H, W, p, &need))) return st;
    if (ws_bytes < need) return pnp_fail(GBM3D_ENOMEM, "pnp: workspace %zu bytes, need %zu", ws_bytes, need);
    if (((uintptr_t)ws) % kAlign) return pnp_fail(GBM3D_EINVAL, "pnp: ws must be 256-byte aligned");
    for (int i = 0; i < n; i++) {
        if (!y[i] || !out[i] || ypitch[i] < W[i] || opitch[i] < W[i])
            return pnp_fail(GBM3D_EINVAL, "pnp: image %d: null pointer or pitch < W", i);
        if (!(sigma[i] >= 0.f) || !isfinite(sigma[i])) return pnp_fail(GBM3D_EINVAL, "pnp: sigma must be >= 0");
    }
    cudaStream_t s0 = (cudaStream_t)stream;
    auto *P = new gbm3d_pnp_plan_st();
    P->p = *p;
    P->q = *q;
    P->R = psf_len / 2;
    // tables: g[0..R], then per size the cas matrix and the eigenvalues
    char *base = (char *)ws;
    float *g = (float *)base;
    cudaError_t e = cudaMemcpyAsync(g, psf + P->R, (P->R + 1) * sizeof(float), cudaMemcpyHostToDevice, s0);
    P->g = g;
    size_t o = align_up(kMaxPsf * sizeof(float));
    std::map<int, std::pair<const float *, const float *>> tab;
    for (int N : distinct_sizes(n, H, W)) {
        float *C = (float *)(base + o);
        o += align_up((size_t)N * N * sizeof(float));
        float *lam = (float *)(base + o);
        o += align_up((size_t)N * sizeof(float));
        if (e == cudaSuccess) {
            k_cas<<<(unsigned)(((long long)N * N + 255) / 256), 256, 0, s0>>>(N, C);
            k_lambda<<<(N + 127) / 128, 128, 0, s0>>>(N, g, P->R, lam);
            e = cudaGetLastError();
        }
        tab[N] = {C, lam};
    }
    for (int i = 0; i < n; i++) {
        PnpImage m{};
        m.H = H[i];
        m.W = W[i];
        m.ypitch = ypitch[i];
        m.opitch = opitch[i];
        m.sigma_d = sigma[i] / sqrtf(q->rho);
        m.y = y[i];
        m.out = out[i];
        size_t b = 0;
        gbm3d_workspace_bytes(m.H, m.W, p, &b);
        m.dws = base + o;
        o += align_up(b);
        float **planes[6] = {&m.hty, &m.b, &m.t1, &m.t, &m.u, &m.v};
        for (float **pl : planes) {
            *pl = (float *)(base + o);
            o += plane_bytes(m.H, m.W);
        }
        m.casH = tab[m.H].first;
        m.lamH = tab[m.H].second;
        m.casW = tab[m.W].first;
        m.lamW = tab[m.W].second;
        P->img.push_back(m);
    }
    // autotune the two product shapes of every image on its own buffers
    for (PnpImage &m : P->img) {
        if (e != cudaSuccess) break;
        m.cfg1 = autotune(m.casH, m.b, m.t1, m.H, m.W, m.H, s0, q->autotune != 0);
        m.cfg2 = autotune(m.t1, m.casW, m.t, m.H, m.W, m.W, s0, q->autotune != 0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s0);
    if (e != cudaSuccess) {
        delete P;
        return pnp_cuda_fail(e, "pnp plan setup");
    }
    if (q->use_graph) {
        // one iteration of every image, each on its own branch, as a graph
        e = cudaStreamCreateWithFlags(&P->origin, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming);
        for (int i = 0; i < n && e == cudaSuccess; i++) {
            cudaStream_t sti;
            cudaEvent_t ev;
            e = cudaStreamCreateWithFlags(&sti, cudaStreamNonBlocking);
            if (e != cudaSuccess) break;
            P->streams.push_back(sti);
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) break;
            P->joins.push_back(ev);
        }
        int ist = GBM3D_OK;
        if (e == cudaSuccess) {
            cudaEvent_t *hook = swap_match_events(nullptr);
            e = cudaStreamBeginCapture(P->origin, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                e = cudaEventRecord(P->fork, P->origin);
                for (int i = 0; i < n && e == cudaSuccess && ist == GBM3D_OK; i++) {
                    e = cudaStreamWaitEvent(P->streams[i], P->fork, 0);
                    if (e == cudaSuccess) ist = pnp_iteration(*P, P->img[i], P->streams[i]);
                    if (e == cudaSuccess && ist == GBM3D_OK) e = cudaEventRecord(P->joins[i], P->streams[i]);
                    if (e == cudaSuccess && ist == GBM3D_OK) e = cudaStreamWaitEvent(P->origin, P->joins[i], 0);
                }
                cudaGraph_t graph = nullptr;
                const cudaError_t e2 = cudaStreamEndCapture(P->origin, &graph);
                if (e == cudaSuccess) e = e2;
                P->graph = graph;
            }
            swap_match_events(hook);
            if (e == cudaSuccess && ist == GBM3D_OK) e = cudaGraphInstantiate(&P->exec, P->graph, 0);
        }
        if (e != cudaSuccess || ist != GBM3D_OK) {
            gbm3d_pnp_plan_destroy(P);
            return ist != GBM3D_OK ? ist : pnp_cuda_fail(e, "pnp graph capture");
        }
    }
    *plan = P;
    return GBM3D_OK;
}

int gbm3d_pnp_run(gbm3d_pnp_plan plan, gbm3d_stream_t stream)
{
    if (!plan) return pnp_fail(GBM3D_EINVAL, "pnp: plan is NULL");
    const gbm3d_pnp_plan_st &P = *plan;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    dim3 grid;
    for (const PnpImage &m : P.img) { // H^T y (h symmetric: the blur itself), v = y, u = 0, b
        launch_grid(grid, m.H, m.W);
        k_conv1<<<grid, 256, 0, st>>>(m.y, m.ypitch, m.t1, m.W, m.H, m.W, P.g, P.R, 0);
        k_conv1<<<grid, 256, 0, st>>>(m.t1, m.W, m.hty, m.W, m.H, m.W, P.g, P.R, 1);
        k_pnp_init<<<grid, 256, 0, st>>>(m.y, m.ypitch, m.hty, m.v, m.u, m.b, m.H, m.W, P.q.rho);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return pnp_cuda_fail(e, "pnp init");
    for (int it = 0; it < P.q.iters; it++) {
        if (P.exec) {
            if ((e = cudaGraphLaunch(P.exec, st)) != cudaSuccess) return pnp_cuda_fail(e, "pnp graph launch");
        } else {
            for (const PnpImage &m : P.img) {
                const int s = pnp_iteration(P, m, st);
                if (s != GBM3D_OK) return s;
            }
        }
    }
    for (const PnpImage &m : P.img) {
        launch_grid(grid, m.H, m.W);
        k_copy2d<<<grid, 256, 0, st>>>(m.v, m.W, m.out, m.opitch, m.H, m.W);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return pnp_cuda_fail(e, "pnp output");
    return GBM3D_OK;
}

int gbm3d_pnp_plan_destroy(gbm3d_pnp_plan plan)
{
    if (!plan) return GBM3D_OK;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    for (cudaEvent_t ev : plan->joins) cudaEventDestroy(ev);
    for (cudaStream_t s : plan->streams) cudaStreamDestroy(s);
    if (plan->fork) cudaEventDestroy(plan->fork);
    if (plan->origin) cudaStreamDestroy(plan->origin);
    delete plan;
    return GBM3D_OK;
}

int gbm3d_pnp_gemm_config(gbm3d_pnp_plan plan, int image, int *cfg_k_h, int *cfg_k_w)
{
    if (!plan || !cfg_k_h || !cfg_k_w || image < 0 || image >= (int)plan->img.size())
        return pnp_fail(GBM3D_EINVAL, "pnp: bad plan, image or pointer");
    *cfg_k_h = plan->img[image].cfg1;
    *cfg_k_w = plan->img[image].cfg2;
    return GBM3D_OK;
}

} // extern "C"
