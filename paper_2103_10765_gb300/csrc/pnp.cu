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
// Each T is two dense matrix products, so any image size works (sizes with
// large prime factors included) at 8 H W (H + W) FLOP per x-update.  The
// products run on the tensor cores (tcgen05.mma kind::tf32, each FP32
// operand split into two tf32 parts, three products accumulated in FP32 in
// tensor memory); an autotuner times the two tile shapes per (M, N, K) on
// the plan's own buffers and keeps the faster.
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

// ---- dense products on the tensor cores ------------------------------------
// C = epilogue(A[M][K] B[K][N]) with FP32 inputs and an FP32-accurate result
// from the 5th-generation tensor cores: every operand is split as
// v = hi + lo with hi = tf32(v) and lo = tf32(v - hi) (tf32: 10 stored
// mantissa bits, round to nearest), and the three products hi.hi + hi.lo +
// lo.hi accumulate in FP32 in tensor memory (tcgen05.mma kind::tf32); the
// dropped lo.lo term is below 2^-22 of |a| |b|.  CTA tile 128 x BN (BN = 128
// or 64), K in stages of 32 with two stages in flight; 8 warps split the
// operands as they load them (thread = one row of the K-major tile; the next
// tile's row is fetched into registers while the current one is split and
// multiplied), one thread issues the 12 MMAs of a stage, and after the last
// stage the warps read the accumulators back (tcgen05.ld) and apply the
// epilogue.
struct Epi {
    int mode;              // 0: alpha acc; 1: acc / ((lamM[r] lamN[c])^2 + rho); 2: alpha acc + add[r][c]
    float alpha, rho;
    const float *lamM, *lamN;
    const float *add;
    int ldadd;
    int trans;             // 1: store C transposed (C^T[c][r], leading dimension ldc)
};

constexpr int kGM = 128, kGK = 32, kGThreads = 256;
constexpr int kGSpin = 1 << 22; // bounded mbarrier polls

__device__ unsigned long long g_gemm_timeouts = 0; // bounded waits of the product kernel that gave up

__device__ __forceinline__ uint32_t g_smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool g_mbar_test(uint32_t a, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(a), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Waits for phase `parity` (at most kGSpin polls); false on a timeout.
__device__ __forceinline__ bool g_mbar_wait(uint32_t a, uint32_t parity)
{
    for (int it = 0; it < kGSpin; it++)
        if (g_mbar_test(a, parity)) return true;
    return false;
}

// K-major operand tile of ROWS x kGK tf32 in core matrices of 8 rows x 16
// bytes: (row r, K chunk c of 4 values) at c * ROWS * 16 + r * 16, i.e.
// leading (K) byte offset ROWS * 16, stride (8-row) byte offset 128.
template <int ROWS>
__device__ __forceinline__ uint64_t g_desc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((ROWS * 16) >> 4) << 16) | ((uint64_t)(128 >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ uint32_t to_tf32(float v)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
}

// Splits 4 values into tf32 high and low parts and stores both 16-byte rows.
__device__ __forceinline__ void split4(float4 v, unsigned char *hi, unsigned char *lo)
{
    const uint32_t h0 = to_tf32(v.x), h1 = to_tf32(v.y), h2 = to_tf32(v.z), h3 = to_tf32(v.w);
    const uint32_t l0 = to_tf32(v.x - __uint_as_float(h0)), l1 = to_tf32(v.y - __uint_as_float(h1));
    const uint32_t l2 = to_tf32(v.z - __uint_as_float(h2)), l3 = to_tf32(v.w - __uint_as_float(h3));
    *reinterpret_cast<uint4 *>(hi) = make_uint4(h0, h1, h2, h3);
    *reinterpret_cast<uint4 *>(lo) = make_uint4(l0, l1, l2, l3);
}

// Instruction descriptor of tcgen05.mma kind::tf32: D FP32 (bits 4-5 = 1),
// A and B TF32 (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
template <int BN>
__host__ __device__ constexpr uint32_t g_idesc()
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kGM >> 4) << 24);
}

template <int BN>
constexpr int g_smem_bytes()
{
    return 2 * (2 * kGM * kGK * 4 + 2 * BN * kGK * 4) + 64;
}

// B arrives transposed, as Bt[n][k] = B[k][n] (rows along K, like A), so both
// operands load as 16-byte rows.  M, N, K are multiples of 8.  A wait that
// gives up fills the CTA's output tile with NaN (and counts
// g_gemm_timeouts), so a failure cannot pass unseen.
template <int BN>
__global__ void __launch_bounds__(kGThreads, 1)
k_gemm_tc(const float *__restrict__ A, int lda, const float *__restrict__ Bt, int ldb, float *__restrict__ C,
          int ldc, int M, int N, int K, Epi epi)
{
    constexpr int kA = kGM * kGK * 4, kB = BN * kGK * 4; // bytes of one split part of a stage
    constexpr int kStage = 2 * kA + 2 * kB;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *ready = reinterpret_cast<uint64_t *>(smem + 2 * kStage); // [2] operands built (kGThreads arrivals)
    uint64_t *done = ready + 2;                                         // [2] products of the stage complete
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(done + 2);
    volatile int *s_err = reinterpret_cast<volatile int *>(s_tmem + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kGM, n0 = blockIdx.x * BN;
    const int nk = (K + kGK - 1) / kGK;
    const uint32_t sb = g_smem_u32(smem);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(g_smem_u32(s_tmem)),
                     "r"((uint32_t)BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < 2; b++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(g_smem_u32(&ready[b])), "r"(kGThreads)
                         : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(g_smem_u32(&done[b])), "r"(1) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_err = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_tmem;
    int issued = -1; // thread 0: the last stage whose products were issued

    // this thread's operand row of a k-tile (A row, or B column as a K-major
    // row): 8 chunks of 4 values, zero outside the matrices
    const bool arow = tid < kGM, brow = !arow && tid - kGM < BN;
    const int ar = m0 + tid, nn = tid - kGM, cn = n0 + nn;
    auto fetch = [&](int kt, float4 (&v)[kGK / 4]) {
        const int k0 = kt * kGK;
#pragma unroll
        for (int c = 0; c < kGK / 4; c++) {
            const int k = k0 + 4 * c; // K is a multiple of 8: k < K covers all four
            v[c] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (arow && ar < M && k < K) {
                v[c] = __ldg(reinterpret_cast<const float4 *>(A + (size_t)ar * lda + k));
            } else if (brow && cn < N && k < K) {
                v[c] = __ldg(reinterpret_cast<const float4 *>(Bt + (size_t)cn * ldb + k));
            }
        }
    };
    float4 nxt[kGK / 4];
    fetch(0, nxt);
    for (int kt = 0; kt < nk; kt++) {
        const int st = kt & 1;
        unsigned char *stg = smem + st * kStage;
        float4 cur[kGK / 4];
#pragma unroll
        for (int c = 0; c < kGK / 4; c++) cur[c] = nxt[c];
        if (kt + 1 < nk) fetch(kt + 1, nxt); // in flight while this tile is split and multiplied
        // this stage's buffers were read by the products of k-tile kt - 2
        if (kt >= 2 && !*s_err && !g_mbar_wait(g_smem_u32(&done[st]), ((kt - 2) >> 1) & 1)) {
            *s_err = 1;
            atomicAdd(&g_gemm_timeouts, 1ull);
        }
        if (!*s_err) {
            if (arow) {
#pragma unroll
                for (int c = 0; c < kGK / 4; c++)
                    split4(cur[c], stg + c * kGM * 16 + tid * 16, stg + kA + c * kGM * 16 + tid * 16);
            } else if (brow) {
#pragma unroll
                for (int c = 0; c < kGK / 4; c++)
                    split4(cur[c], stg + 2 * kA + c * BN * 16 + nn * 16, stg + 2 * kA + kB + c * BN * 16 + nn * 16);
            }
        }
        // the generic-proxy stores become visible to the tensor cores' reads
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(g_smem_u32(&ready[st])) : "memory");
        if (tid == 0 && !*s_err) {
            if (!g_mbar_wait(g_smem_u32(&ready[st]), (kt >> 1) & 1)) {
                *s_err = 1;
                atomicAdd(&g_gemm_timeouts, 1ull);
            } else {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t base = sb + st * kStage;
#pragma unroll
                for (int j = 0; j < kGK / 8; j++) { // K = 8 per instruction: two chunks
                    const uint64_t ah = g_desc<kGM>(base + j * 2 * kGM * 16);
                    const uint64_t al = g_desc<kGM>(base + kA + j * 2 * kGM * 16);
                    const uint64_t bh = g_desc<BN>(base + 2 * kA + j * 2 * BN * 16);
                    const uint64_t bl = g_desc<BN>(base + 2 * kA + kB + j * 2 * BN * 16);
                    const uint32_t first = (kt > 0 || j > 0) ? 1u : 0u;
#define GEMM_MMA(ad, bd, acc)                                                                               \
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"                                          \
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),                \
                 "l"(ad), "l"(bd), "r"(g_idesc<BN>()), "r"(acc)                                             \
                 : "memory")
                    GEMM_MMA(ah, bh, first);
                    GEMM_MMA(ah, bl, 1u);
                    GEMM_MMA(al, bh, 1u);
#undef GEMM_MMA
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 g_smem_u32(&done[st]))
                             : "memory");
                issued = kt;
            }
        }
    }
    // thread 0 waits for the last products it issued (also after an error:
    // tensor memory and shared memory must not be released under them)
    if (tid == 0 && issued >= 0 && !g_mbar_wait(g_smem_u32(&done[issued & 1]), (issued >> 1) & 1)) {
        *s_err = 1;
        atomicAdd(&g_gemm_timeouts, 1ull);
    }
    if (tid == 0 && issued != nk - 1) *s_err = 1; // not every stage was multiplied
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool ok = !*s_err;

    // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. (rows of the
    // tile) and half w / 4 of the columns, 32 at a time
    const int q = warp & 3, half = warp >> 2;
    const int r = m0 + 32 * q + lane;
    for (int cc = half * (BN / 2); cc < (half + 1) * (BN / 2); cc += 32) {
        uint32_t v[32];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                     "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                     "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
                     "tcgen05.wait::ld.sync.aligned;"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                       "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                       "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
                       "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                       "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                     : "r"(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)cc)
                     : "memory");
        if (r >= M) continue;
        const int c0 = n0 + cc;
        float o[32];
#pragma unroll
        for (int j = 0; j < 32; j++) {
            float val = __uint_as_float(v[j]);
            const int c = c0 + j;
            if (!ok) {
                val = __int_as_float(0x7fc00000); // NaN: the tile was not computed
            } else if (epi.mode == 1) {
                const float l = __ldg(epi.lamM + r) * __ldg(epi.lamN + (c < N ? c : N - 1));
                val = val / fmaf(l, l, epi.rho);
            } else if (epi.mode == 2) {
                val = fmaf(epi.alpha, val, c < N ? __ldg(epi.add + (size_t)r * epi.ldadd + c) : 0.f);
            } else {
                val *= epi.alpha;
            }
            o[j] = val;
        }
        if (epi.trans) { // lanes hold consecutive rows: each column's 32 stores are coalesced
#pragma unroll
            for (int j = 0; j < 32; j++)
                if (c0 + j < N) C[(size_t)(c0 + j) * ldc + r] = o[j];
            continue;
        }
        float *dst = C + (size_t)r * ldc + c0;
        if (c0 + 32 <= N) {
#pragma unroll
            for (int j = 0; j < 32; j += 4)
                *reinterpret_cast<float4 *>(dst + j) = make_float4(o[j], o[j + 1], o[j + 2], o[j + 3]);
        } else {
#pragma unroll
            for (int j = 0; j < 32; j++)
                if (c0 + j < N) dst[j] = o[j];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN)
                     : "memory");
    }
}

struct GemmCfg {
    int bn;
    void (*fn)(const float *, int, const float *, int, float *, int, int, int, int, Epi);
    int smem;
};

const GemmCfg kGemmCfgs[] = {
    {128, k_gemm_tc<128>, g_smem_bytes<128>()},
    {64, k_gemm_tc<64>, g_smem_bytes<64>()},
};
constexpr int kNumCfgs = sizeof(kGemmCfgs) / sizeof(kGemmCfgs[0]);

// C = epi(A B), A [M][K] row-major (lda), B given as Bt [N][K] row-major (ldb)
// (for a symmetric B, B itself).
cudaError_t gemm(int cfg, const float *A, int lda, const float *Bt, int ldb, float *C, int ldc, int M, int N, int K,
                 const Epi &epi, cudaStream_t st)
{
    const GemmCfg &g = kGemmCfgs[cfg];
    cudaError_t e = cudaFuncSetAttribute(g.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, g.smem);
    if (e != cudaSuccess) return e;
    dim3 grid((N + g.bn - 1) / g.bn, (M + kGM - 1) / kGM);
    g.fn<<<grid, kGThreads, g.smem, st>>>(A, lda, Bt, ldb, C, ldc, M, N, K, epi);
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
// the same bits: every output accumulates the same products in the same K
// order).
std::map<std::tuple<int, int, int>, int> g_tuned;

int autotune(const float *A, const float *Bt, float *C, int M, int N, int K, cudaStream_t st, bool enabled)
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
    Epi epi{0, 1.f, 0.f, nullptr, nullptr, nullptr, 0, 0};
    int best = 0;
    float best_ms = 1e30f;
    for (int c = 0; c < kNumCfgs; c++) {
        if (gemm(c, A, K, Bt, K, C, N, M, N, K, epi, st) != cudaSuccess) continue; // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3; r++) gemm(c, A, K, Bt, K, C, N, M, N, K, epi, st);
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
    const Epi plain_t{0, 1.f, 0.f, nullptr, nullptr, nullptr, 0, 1};
    const Epi divide{1, 1.f, rho, m.lamH, m.lamW, nullptr, 0, 0};
    const Epi finish{2, 1.f / ((float)H * (float)W), 0.f, nullptr, nullptr, m.u, W, 0};
    cudaError_t e;
    // T(b) = C_H (b C_W): the inner product is stored transposed (t1 as
    // [W][H]), so the outer one reads it, like the symmetric C_W, as rows
    // along its contraction; then the eigenvalue division, and the same two
    // products again back to the image domain (+ u)
    if ((e = gemm(m.cfg2, m.b, W, m.casW, W, m.t1, H, H, W, W, plain_t, st)) != cudaSuccess)
        return pnp_cuda_fail(e, "pnp gemm");
    if ((e = gemm(m.cfg1, m.casH, H, m.t1, H, m.b, W, H, W, H, divide, st)) != cudaSuccess)
        return pnp_cuda_fail(e, "pnp gemm");
    if ((e = gemm(m.cfg2, m.b, W, m.casW, W, m.t1, H, H, W, W, plain_t, st)) != cudaSuccess)
        return pnp_cuda_fail(e, "pnp gemm");
    if ((e = gemm(m.cfg1, m.casH, H, m.t1, H, m.t, W, H, W, H, finish, st)) != cudaSuccess)
        return pnp_cuda_fail(e, "pnp gemm");
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
        m.cfg1 = autotune(m.casH, m.t1, m.t, m.H, m.W, m.H, s0, q->autotune != 0);
        m.cfg2 = autotune(m.b, m.casW, m.t1, m.H, m.W, m.W, s0, q->autotune != 0);
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
