// match.cu -- block matching (Sec. 2 eq. dfg, Theorem 1, Algorithm 1;
// Sec. 3.1 S^K_pq).
//
// One warp per reference block, eight references (consecutive grid columns
// of one grid row) per CTA sharing one shared-memory copy of their search
// region.  The reference block lives in registers (64 floats per lane, the
// same in every lane); each lane takes four vertically stacked candidates at
// a time, so every 8-pixel image row it loads from shared memory serves up
// to four candidate rows (11 row loads per 4 candidates instead of 32).
// Distances are the exact sum of squared differences in FP32 -- the direct
// form, not the norm expansion of eq. (expand), which cancels badly in FP32.
//
// Selection keeps the K-1 best (distance, k*W+l) keys in a warp-distributed
// sorted list: lane t holds the t-th best.  Each batch of candidates is
// compared against the current K-1-th key; the few that qualify (ballot) are
// inserted one at a time with a shuffle-based shift.  The reference block
// itself is excluded and written to slot 0.
#include <float.h>
#include <limits.h>

#include "internal.cuh"

namespace gbm3d {
namespace {

constexpr int kRefsPerCta = 8;
constexpr int kVB = 4;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ bool key_less(float da, int ia, float db, int ib)
{
    return da < db || (da == db && ia < ib);
}

template <int N>
__global__ void __launch_bounds__(kRefsPerCta * 32)
k_match(const float *__restrict__ img, int H, int W, int pitch, int Bx, int s, int R, int K,
        int32_t *__restrict__ idx, float *__restrict__ dist)
{
    extern __shared__ float sm[];
    const int p = blockIdx.y;
    const int q0 = blockIdx.x * kRefsPerCta;
    const int i = grid_pos(p, s, H, N);
    const int qlast = min(q0 + kRefsPerCta - 1, Bx - 1);
    const int jf = grid_pos(q0, s, W, N), jl = grid_pos(qlast, s, W, N);
    const int ry0 = max(0, i - R), ry1 = min(H - N, i + R) + N;
    const int rx0 = max(0, jf - R), rx1 = min(W - N, jl + R) + N;
    const int rw = rx1 - rx0, rh = ry1 - ry0;
    const int rhp = rh + kVB; // zero rows below absorb the last vertical block
    for (int e = threadIdx.x; e < rhp * rw; e += blockDim.x) {
        const int y = e / rw, x = e - y * rw;
        sm[e] = (y < rh) ? __ldg(img + (size_t)(ry0 + y) * pitch + rx0 + x) : 0.f;
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = q0 + warp;
    if (q >= Bx) return;
    const int j = grid_pos(q, s, W, N);

    float r[N][N];
#pragma unroll
    for (int a = 0; a < N; a++)
#pragma unroll
        for (int b = 0; b < N; b++) r[a][b] = sm[(i - ry0 + a) * rw + (j - rx0 + b)];

    const int k0 = ry0, k1 = min(H - N, i + R);
    const int l0 = max(0, j - R), l1 = min(W - N, j + R);
    const int ny = k1 - k0 + 1, nx = l1 - l0 + 1;
    const int nunits = ((ny + kVB - 1) / kVB) * nx;
    const int Kc = K - 1;
    const float kInf = __int_as_float(0x7f800000);

    float ld = kInf;  // this lane's list entry (lane t = t-th best)
    int li = INT_MAX;
    float thr_d = kInf; // current (K-1)-th best key
    int thr_i = INT_MAX;

    for (int u0 = 0; u0 < nunits; u0 += 32) {
        const int u = u0 + lane;
        const bool vu = u < nunits;
        int kb = 0, dl = 0;
        if (vu) {
            kb = u / nx;
            dl = u - kb * nx;
        }
        const int k = k0 + kb * kVB, l = l0 + dl;
        float d[kVB];
#pragma unroll
        for (int c = 0; c < kVB; c++) d[c] = 0.f;
        if (vu) {
            const float *base = sm + (k - ry0) * rw + (l - rx0);
#pragma unroll
            for (int t = 0; t < kVB + N - 1; t++) {
                float x[N];
#pragma unroll
                for (int b = 0; b < N; b++) x[b] = base[t * rw + b];
#pragma unroll
                for (int c = 0; c < kVB; c++) {
                    const int a = t - c;
                    if (a >= 0 && a < N) {
#pragma unroll
                        for (int b = 0; b < N; b++) {
                            const float df = r[a][b] - x[b];
                            d[c] = fmaf(df, df, d[c]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int c = 0; c < kVB; c++) {
            const int kc = k + c;
            const bool valid = vu && kc <= k1 && !(kc == i && l == j);
            const int cid = kc * W + l;
            const float cd = d[c];
            bool pend = valid && key_less(cd, cid, thr_d, thr_i);
            unsigned mask = __ballot_sync(kFull, pend);
            while (mask) {
                const int src = __ffs(mask) - 1;
                const float nd = __shfl_sync(kFull, cd, src);
                const int ni = __shfl_sync(kFull, cid, src);
                const float pd = __shfl_up_sync(kFull, ld, 1);
                const int pi = __shfl_up_sync(kFull, li, 1);
                if (lane < Kc && key_less(nd, ni, ld, li)) {
                    if (lane == 0 || key_less(pd, pi, nd, ni)) {
                        ld = nd;
                        li = ni;
                    } else {
                        ld = pd;
                        li = pi;
                    }
                }
                thr_d = __shfl_sync(kFull, ld, Kc - 1);
                thr_i = __shfl_sync(kFull, li, Kc - 1);
                if (lane == src) pend = false;
                pend = pend && key_less(cd, cid, thr_d, thr_i);
                mask = __ballot_sync(kFull, pend);
            }
        }
    }

    const size_t gi = ((size_t)p * Bx + q) * K;
    if (lane < Kc) {
        idx[gi + 1 + lane] = li;
        if (dist) dist[gi + 1 + lane] = ld;
    }
    if (lane == 0) {
        idx[gi] = i * W + j;
        if (dist) dist[gi] = 0.f;
    }
}

} // namespace

size_t match_smem_bytes(int s, int R)
{
    const int rows = 2 * R + kPatch + kVB;
    const int cols = (kRefsPerCta - 1) * s + 2 * R + kPatch;
    return (size_t)rows * cols * sizeof(float);
}

cudaError_t launch_match(const float *img, int H, int W, int pitch, int By, int Bx, int s, int R, int K,
                         int32_t *idx, float *dist, cudaStream_t st)
{
    const size_t smem = match_smem_bytes(s, R);
    cudaError_t e = cudaFuncSetAttribute(k_match<kPatch>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((Bx + kRefsPerCta - 1) / kRefsPerCta, By);
    k_match<kPatch><<<grid, kRefsPerCta * 32, smem, st>>>(img, H, W, pitch, Bx, s, R, K, idx, dist);
    return cudaGetLastError();
}

} // namespace gbm3d
