// match.cu -- block matching (Sec. 2 eq. dfg, Theorem 1, Algorithm 1;
// Sec. 3.1 S^K_pq).
//
// One warp per reference block, eight references (consecutive grid columns
// of one grid row) per CTA sharing one shared-memory copy of their search
// region.  The reference block lives in registers (64 floats per lane, the
// same in every lane; a 16 x 16 block, 256 floats, would not fit, so there
// the lanes hold 4 of its rows at a time and reload the next 4 from shared
// memory, a broadcast read); each lane takes four vertically stacked candidates at
// a time, so every 8-pixel image row it loads from shared memory serves up
// to four candidate rows (11 row loads per 4 candidates instead of 32).
// Distances are the exact sum of squared differences in FP32 -- the direct
// form, not the norm expansion of eq. (expand), which cancels badly in FP32 --
// computed with Blackwell's packed FP32 pairs (add/fma.rn.f32x2 on the
// negated reference): the even
// and odd columns of a block row are two independent FP32 partial sums, each
// rounded exactly as scalar FSUB/FFMA would be.
//
// Lane layout: a work unit is (block of kVB candidate rows, candidate
// column); units are numbered row-major with the column count padded to a
// multiple of 8 (col_pad), and the shared-memory row stride is chosen so that
// kVB * stride == col_pad (mod 32).  A warp's 32 consecutive units then read
// 32 distinct banks even where they straddle two unit rows.  Pixels are read
// as aligned float pairs straight into the packed registers: the region is
// stored twice, the second copy shifted by one float, and each lane reads
// whichever copy puts its row start on an even offset.
//
// Selection (K-1 best keys (distance, k*W+l)) follows the warp-select
// pattern: lane t holds the t-th best of a sorted 32-entry list; candidates
// that beat the current (K-1)-th key are handled per candidate row of the
// batch: all of a batch's keys are first tested against the threshold with
// one ballot per candidate row; rows without a qualifying lane (most of them
// once the list has filled) cost nothing more.  When at most kInsertMax lanes
// of a row qualify they are inserted one at a time with a shuffle-based
// shift, the threshold tightening after each; when more qualify (the first
// batches) they are appended to a per-warp buffer (ballot + prefix count)
// and every full 32 are bitonic-sorted across the warp and merged into the
// list by an out-of-line function.  The scan starts at the reference's own
// rows so that the threshold tightens early.  The reference block itself is excluded and written to
// slot 0.
#include <float.h>
#include <limits.h>

#include "internal.cuh"

namespace gbm3d {
namespace {

constexpr int kRefsPerCta = 8;
constexpr int kVB = 4;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kBuf = 64;       // per-warp candidate buffer: a partial batch + one step's appends
constexpr int kInsertMax = 4;  // at most this many qualifying candidates: insert one by one

typedef unsigned long long f2; // two packed FP32 values

__device__ __forceinline__ f2 pack2(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void unpack2(f2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// acc += (x + nr)^2 elementwise on both halves, with nr = -r the negated
// reference pixels: x + (-r) is exactly x - r, and (x - r)^2 = (r - x)^2.
__device__ __forceinline__ f2 sqdiff_acc2(f2 nr, f2 x, f2 acc)
{
    f2 e, o;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(e) : "l"(x), "l"(nr));
    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(o) : "l"(e), "l"(acc));
    return o;
}

__device__ __forceinline__ bool key_less(float da, int ia, float db, int ib)
{
    return da < db || (da == db && ia < ib);
}

// Compare-exchange across lanes lane and lane^j; `asc` selects the order of
// the enclosing bitonic block.
__device__ __forceinline__ void cmpx(float &d, int &i, int j, bool asc, int lane)
{
    const float od = __shfl_xor_sync(kFull, d, j);
    const int oi = __shfl_xor_sync(kFull, i, j);
    const bool lower = (lane & j) == 0;
    const bool take = (lower == asc) ? key_less(od, oi, d, i) : key_less(d, i, od, oi);
    if (take) {
        d = od;
        i = oi;
    }
}

// Sort 32 keys (one per lane) ascending by lane.
__device__ __forceinline__ void bitonic_sort32(float &d, int &i, int lane)
{
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) cmpx(d, i, j, (lane & k) == 0, lane);
}

// list (ascending by lane) <- the 32 smallest of list and b (ascending).
__device__ __forceinline__ void merge32(float &ld, int &li, float bd, int bi, int lane)
{
    const float rd = __shfl_sync(kFull, bd, 31 - lane);
    const int ri = __shfl_sync(kFull, bi, 31 - lane);
    if (key_less(rd, ri, ld, li)) {
        ld = rd;
        li = ri;
    }
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) cmpx(ld, li, j, true, lane);
}

// Three CTAs per SM (<= 85 registers): the extra warps hide the latency of
// the FP chains better than the registers the compiler gives up cost.
// The list, its threshold and the buffer fill, as passed to the out-of-line
// merge (the rare path; keeping it out of the unrolled loop keeps the loop
// body small).
struct ListState {
    float ld;
    int li;
    float thr_d;
    int thr_i;
    int cnt;
};

// Merges the first 32 buffered keys into the list, moves the rest of the
// buffer to its front and refreshes the threshold.  Called by the whole warp.
__device__ __noinline__ ListState merge_buffer(ListState s, float *wb_d, int *wb_i, int lane, int Kc)
{
    __syncwarp();
    float bd = wb_d[lane];
    int bi = wb_i[lane];
    bitonic_sort32(bd, bi, lane);
    merge32(s.ld, s.li, bd, bi, lane);
    s.cnt -= 32;
    float md = 0.f;
    int mi = 0;
    if (lane < s.cnt) {
        md = wb_d[32 + lane];
        mi = wb_i[32 + lane];
    }
    __syncwarp();
    if (lane < s.cnt) {
        wb_d[lane] = md;
        wb_i[lane] = mi;
    }
    __syncwarp();
    s.thr_d = __shfl_sync(kFull, s.ld, Kc - 1);
    s.thr_i = __shfl_sync(kFull, s.li, Kc - 1);
    return s;
}

// Arguments of one matching launch (the shared-memory geometry comes from
// match_geom on the host).
struct MatchArgs {
    const float *img;
    int H, W, pitch, Bx, s, R, K, col_pad, rw, copy_off, bufs_off;
    int32_t *idx;
    float *dist;
};

// Matches the references q0 .. q0+kRefs-1 of grid row p: one warp per
// reference, their common search region in shared memory sm.  kRefs ==
// kRefsPerCta (k_match): every thread of the CTA calls it (the region load
// ends in a __syncthreads).  kRefs == 1 with kSplit > 1 (k_match_fix): the
// CTA's kSplit warps share the one reference -- warp w scans candidate units
// w, w + kSplit, ..., and warp 0 merges their sorted lists (the same K - 1
// smallest (distance, index) pairs; the others return early).  kRefs ==
// kSplit == 1: one warp alone, with its own region (the load ends in a
// __syncwarp).
template <int N, int kRefs, int kSplit = 1>
__device__ __forceinline__ void match_group(const MatchArgs &A, int p, int q0, float *sm)
{
    const float *__restrict__ img = A.img;
    const int H = A.H, W = A.W, pitch = A.pitch, Bx = A.Bx, s = A.s, R = A.R, K = A.K;
    const int col_pad = A.col_pad, rw = A.rw, copy_off = A.copy_off, bufs_off = A.bufs_off;
    int32_t *__restrict__ idx = A.idx;
    float *__restrict__ dist = A.dist;
    const int i = grid_pos(p, s, H, N);
    const int qlast = min(q0 + kRefs - 1, Bx - 1);
    const int jf = grid_pos(q0, s, W, N), jl = grid_pos(qlast, s, W, N);
    const int ry0 = max(0, i - R), ry1 = min(H - N, i + R) + N;
    const int rx0 = max(0, jf - R), rx1 = min(W - N, jl + R) + N;
    const int rwd = rx1 - rx0, rh = ry1 - ry0;
    const int rhp = rh + kVB; // zero rows below absorb the last vertical block
    float *smB = sm + copy_off; // the region again, one float later: smB[e] = sm[e - 1]
    float *buf_d = sm + bufs_off;
    int *buf_i = reinterpret_cast<int *>(buf_d + (kRefs > kSplit ? kRefs : kSplit) * kBuf); // a buffer per warp
    constexpr bool kLone = kRefs == 1 && kSplit == 1; // one warp on its own
    const int t0 = kLone ? (threadIdx.x & 31) : threadIdx.x, nt = kLone ? 32 : blockDim.x;
    { // the region, eight loads per thread in flight before their stores; element
      // e = y rw + x advances by nt per load: dy = nt / rw rows and dx = nt mod rw
      // columns, with at most one carry from the columns into the rows
        constexpr int kLd = 8;
        const int total = rhp * rw, dy = nt / rw, dx = nt - dy * rw;
        int y = t0 / rw, x = t0 - y * rw;
        for (int e0 = t0; e0 < total; e0 += kLd * nt) {
            float v[kLd];
            int yy = y, xx = x;
#pragma unroll
            for (int u = 0; u < kLd; u++) {
                const int e = e0 + u * nt;
                v[u] = (e < total && yy < rh && xx < rwd) ? __ldg(img + (size_t)(ry0 + yy) * pitch + rx0 + xx) : 0.f;
                yy += dy;
                xx += dx;
                if (xx >= rw) {
                    xx -= rw;
                    yy++;
                }
            }
#pragma unroll
            for (int u = 0; u < kLd; u++) {
                const int e = e0 + u * nt;
                if (e < total) {
                    sm[e] = v[u];
                    smB[e + 1] = v[u];
                }
            }
            y = yy;
            x = xx;
        }
    }
    if (t0 == 0) smB[0] = 0.f;
    if (kLone)
        __syncwarp();
    else
        __syncthreads();

    const int warp = kRefs == 1 ? 0 : threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int part = kSplit > 1 ? threadIdx.x >> 5 : 0; // this warp's share of the units
    const int q = q0 + warp;
    if (q >= Bx) return; // (never with kSplit > 1: the reference exists)
    const int j = grid_pos(q, s, W, N);
    float *wb_d = buf_d + (kSplit > 1 ? part : warp) * kBuf;
    int *wb_i = buf_i + (kSplit > 1 ? part : warp) * kBuf;

    // negated reference block rows a0 .. a0+NA-1, column pairs (b, b+1) packed:
    // all of it for N = 8, four rows at a time for N = 16
    constexpr int NA = N <= 8 ? N : 4;
    f2 r[NA][N / 2];
    auto load_ref = [&](int a0) {
#pragma unroll
        for (int a = 0; a < NA; a++)
#pragma unroll
            for (int b = 0; b < N; b += 2)
                r[a][b / 2] = pack2(-sm[(i - ry0 + a0 + a) * rw + (j - rx0 + b)],
                                    -sm[(i - ry0 + a0 + a) * rw + (j - rx0 + b + 1)]);
    };
    if (NA == N) load_ref(0);

    const int k0 = ry0, k1 = min(H - N, i + R);
    const int l0 = max(0, j - R), l1 = min(W - N, j + R);
    const int ny = k1 - k0 + 1, nx = l1 - l0 + 1;
    const int nkb = (ny + kVB - 1) / kVB;
    const int nunits = nkb * col_pad;
    const int kb_start = (i - k0) / kVB; // scan the reference's own rows first
    const int Kc = K - 1;
    const float kInf = __int_as_float(0x7f800000);
    const unsigned lt_mask = (1u << lane) - 1u;

    float ld = kInf; // sorted list: lane t holds the t-th best key
    int li = INT_MAX;
    float thr_d = kInf;
    int thr_i = INT_MAX;
    int cnt = 0; // entries in the warp buffer (warp-uniform)

    for (int u0 = 32 * part; u0 < nunits; u0 += 32 * kSplit) {
        const int u = u0 + lane;
        const bool vu = u < nunits;
        int kb = 0, dl = 0;
        if (vu) {
            kb = u / col_pad;
            dl = u - kb * col_pad;
            kb += kb_start;
            if (kb >= nkb) kb -= nkb;
        }
        const int k = k0 + kb * kVB, l = l0 + dl;
        f2 dd[kVB]; // (even-column, odd-column) partial sums per candidate
#pragma unroll
        for (int c = 0; c < kVB; c++) dd[c] = 0ull;
        if (vu) {
            // 8-byte-aligned start of this lane's rows: even offsets in the
            // region, odd ones in the shifted copy (rw is even)
            const int cc = (k - ry0) * rw + (l - rx0);
            const f2 *base = reinterpret_cast<const f2 *>((cc & 1) ? smB + cc + 1 : sm + cc);
            // rows a of the block in ascending order for every candidate
#pragma unroll 1
            for (int a0 = 0; a0 < N; a0 += NA) {
                if (NA < N) load_ref(a0);
#pragma unroll
                for (int t = 0; t < kVB + NA - 1; t++) {
                    f2 x[N / 2];
#pragma unroll
                    for (int b = 0; b < N / 2; b++) x[b] = base[(a0 + t) * (rw / 2) + b];
#pragma unroll
                    for (int c = 0; c < kVB; c++) {
                        const int a = t - c;
                        if (a >= 0 && a < NA) {
#pragma unroll
                            for (int b = 0; b < N / 2; b++) dd[c] = sqdiff_acc2(r[a][b], x[b], dd[c]);
                        }
                    }
                }
            }
        }
        // keys of the batch (invalid: +inf, INT_MAX never qualify); test them all
        // against the threshold first -- once the list has filled, most batches
        // have no qualifying candidate and skip the selection loop
        float cdv[kVB];
        int cidv[kVB];
        unsigned mk[kVB], any = 0;
#pragma unroll
        for (int c = 0; c < kVB; c++) {
            const int kc = k + c;
            const bool valid = vu && dl < nx && kc <= k1 && !(kc == i && l == j);
            float d0, d1;
            unpack2(dd[c], d0, d1);
            cdv[c] = valid ? d0 + d1 : kInf;
            cidv[c] = valid ? kc * W + l : INT_MAX;
            mk[c] = __ballot_sync(kFull, key_less(cdv[c], cidv[c], thr_d, thr_i));
            any |= mk[c];
        }
        if (!any) continue;
        // only the candidate rows with a qualifying lane (warp-uniform tests)
#pragma unroll
        for (int c = 0; c < kVB; c++) {
            if (!mk[c]) continue;
            const float cd = cdv[c];
            const int cid = cidv[c];
            bool pend = key_less(cd, cid, thr_d, thr_i); // the threshold may have tightened
            unsigned mask = __ballot_sync(kFull, pend);
            const int nq = __popc(mask);
            if (nq > kInsertMax) { // many: buffer them, merge each full 32
                if (pend) {
                    const int pos = cnt + __popc(mask & lt_mask);
                    wb_d[pos] = cd;
                    wb_i[pos] = cid;
                }
                cnt += nq;
                if (cnt >= 32) {
                    ListState st{ld, li, thr_d, thr_i, cnt};
                    st = merge_buffer(st, wb_d, wb_i, lane, Kc);
                    ld = st.ld;
                    li = st.li;
                    thr_d = st.thr_d;
                    thr_i = st.thr_i;
                    cnt = st.cnt;
                }
            } else { // few: insert one at a time, tightening the threshold as we go
                while (mask) {
                    const int src = __ffs(mask) - 1;
                    const float nd = __shfl_sync(kFull, cd, src);
                    const int ni = __shfl_sync(kFull, cid, src);
                    const float pd = __shfl_up_sync(kFull, ld, 1);
                    const int pi = __shfl_up_sync(kFull, li, 1);
                    if (key_less(nd, ni, ld, li)) {
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
    }
    if (cnt > 0) { // flush the partial buffer
        __syncwarp();
        float bd = kInf;
        int bi = INT_MAX;
        if (lane < cnt) {
            bd = wb_d[lane];
            bi = wb_i[lane];
        }
        bitonic_sort32(bd, bi, lane);
        merge32(ld, li, bd, bi, lane);
    }
    if (kSplit > 1) { // the warps' lists, over the region (no longer read), merged by warp 0
        __syncthreads();
        float *md = sm;
        int *mi = reinterpret_cast<int *>(sm + kSplit * 32);
        md[part * 32 + lane] = ld;
        mi[part * 32 + lane] = li;
        __syncthreads();
        if (part != 0) return;
        for (int w = 1; w < kSplit; w++) merge32(ld, li, md[w * 32 + lane], mi[w * 32 + lane], lane);
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

template <int N>
__global__ void __launch_bounds__(kRefsPerCta * 32, N <= 8 ? 3 : 2) k_match(MatchArgs a)
{
    extern __shared__ float sm[];
    match_group<N, kRefsPerCta>(a, blockIdx.y, blockIdx.x * kRefsPerCta, sm);
}

// Re-matches the references the tensor-core pass marked (slot 0 = -1): CTA b
// scans references b, b + gridDim.x, ... (kFixThreads at a time; marked
// references cluster in space, so neighbours go to different CTAs) and matches
// every marked one it found with all its warps (match_group with kSplit =
// kFixThreads / 32).
constexpr int kFixThreads = 256;

template <int N>
__global__ void __launch_bounds__(kFixThreads) k_match_fix(MatchArgs a, int G)
{
    extern __shared__ float sm[];
    __shared__ int s_list[kFixThreads];
    __shared__ int s_n;
    for (long long j0 = 0; j0 * gridDim.x + blockIdx.x < G; j0 += kFixThreads) {
        if (threadIdx.x == 0) s_n = 0;
        __syncthreads();
        const long long g = blockIdx.x + (j0 + threadIdx.x) * gridDim.x;
        if (g < G && a.idx[g * a.K] < 0) s_list[atomicAdd(&s_n, 1)] = (int)g; // any order: outputs are per reference
        __syncthreads();
        const int n = s_n;
        for (int t = 0; t < n; t++) {
            const int gg = s_list[t];
            const int p = gg / a.Bx;
            match_group<N, 1, kFixThreads / 32>(a, p, gg - p * a.Bx, sm);
            __syncthreads();
        }
    }
}

struct MatchGeom {
    int col_pad, rw, rows;
    int copy_off, bufs_off; // floats: offset of the shifted copy, of the selection buffers
};

MatchGeom match_geom(int s, int R, int N, int nrefs = kRefsPerCta)
{
    MatchGeom g;
    g.col_pad = (2 * R + 1 + 7) / 8 * 8;
    // widest row a lane can touch: (l0 - rx0) <= (nrefs-1) s, plus the
    // padded column count, plus the block width
    int need = (nrefs - 1) * s + g.col_pad + N;
    const int data = (nrefs - 1) * s + 2 * R + N;
    if (data > need) need = data;
    g.rw = need; // kVB * rw == col_pad (mod 32)
    while ((kVB * g.rw - g.col_pad) % 32 != 0) g.rw++;
    g.rows = 2 * R + N + kVB;
    // the shifted copy starts 14 words (mod 32) after the region so that the
    // even-column lanes (region) and odd-column lanes (copy) of a half-warp
    // fall on disjoint banks
    g.copy_off = (g.rows * g.rw + 31) / 32 * 32 + 14;
    g.bufs_off = (g.copy_off + g.rows * g.rw + 2 + 3) / 4 * 4;
    return g;
}

} // namespace

size_t match_smem_bytes(int s, int R, int N)
{
    const MatchGeom g = match_geom(s, R, N);
    return (size_t)g.bufs_off * sizeof(float) + (size_t)kRefsPerCta * kBuf * (sizeof(float) + sizeof(int));
}

template <int N>
static cudaError_t launch_match_n(const float *img, int H, int W, int pitch, int By, int Bx, int s, int R, int K,
                                  int32_t *idx, float *dist, cudaStream_t st)
{
    const MatchGeom g = match_geom(s, R, N);
    const size_t smem = match_smem_bytes(s, R, N);
    cudaError_t e = cudaFuncSetAttribute(k_match<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((Bx + kRefsPerCta - 1) / kRefsPerCta, By);
    const MatchArgs a{img, H, W, pitch, Bx, s, R, K, g.col_pad, g.rw, g.copy_off, g.bufs_off, idx, dist};
    k_match<N><<<grid, kRefsPerCta * 32, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_match(const float *img, int H, int W, int pitch, int By, int Bx, int N, int s, int R, int K,
                         int32_t *idx, float *dist, cudaStream_t st)
{
    if (N == 16) return launch_match_n<16>(img, H, W, pitch, By, Bx, s, R, K, idx, dist, st);
    if (N == 8) return launch_match_n<8>(img, H, W, pitch, By, Bx, s, R, K, idx, dist, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_match_fix(const float *img, int H, int W, int pitch, int By, int Bx, int s, int R, int K,
                             int32_t *idx, float *dist, cudaStream_t st)
{
    const MatchGeom g = match_geom(s, R, kPatch, 1);
    const size_t smem =
        (size_t)g.bufs_off * sizeof(float) + (size_t)(kFixThreads / 32) * kBuf * (sizeof(float) + sizeof(int));
    cudaError_t e = cudaFuncSetAttribute(k_match_fix<kPatch>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int G = By * Bx;
    int blocks = 2 * nsm; // all resident at once (registers allow two CTAs per SM)
    if (blocks > G) blocks = G;
    if (blocks < 1) blocks = 1;
    const MatchArgs a{img, H, W, pitch, Bx, s, R, K, g.col_pad, g.rw, g.copy_off, g.bufs_off, idx, dist};
    k_match_fix<kPatch><<<blocks, kFixThreads, smem, st>>>(a, G);
    return cudaGetLastError();
}

} // namespace gbm3d
