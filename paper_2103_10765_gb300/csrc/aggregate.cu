// aggregate.cu -- weighted aggregation of filtered blocks (Sec. 3.1:
// Y = sum w U / sum w chi; stage 2 adds a Kaiser window).
//
// Deterministic owner-computes design: the match lists are inverted into a
// CSR index (block top-left position -> the (group, slot) entries placed
// there; counting sort, then each bucket sorted), and one thread per output
// pixel walks the N x N top-left positions that cover it (N = 8 or 16), in a fixed order,
// summing numerator and denominator with Kahan compensation.  No floating-
// point atomics: the result does not depend on scheduling.
#include <mutex>

#include "internal.cuh"

namespace gbm3d {

// Fixed device scratch for gbm3d_aggregate_noalloc (callers that cannot
// allocate device memory).  Every GPU that loads this library holds these
// bytes until the process exits; all calls on a device share them.
static __device__ __align__(256) unsigned char g_fixed_scratch[kFixedScratchBytes];
namespace {

constexpr int kScanBlock = 1024; // elements per scan block (256 threads x 4)

// Entries that are not valid block positions are skipped (never counted,
// never placed), so a bad caller-supplied list cannot write out of bounds.
__global__ void k_count(const int32_t *__restrict__ idx, int n, int H, int W, int N, int *__restrict__ cnt)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int pos = idx[e];
    if (block_ok(pos, H, W, N)) atomicAdd(cnt + pos, 1);
}

// Exclusive scan, phase 1: per-block scan of 1024 elements, block totals out.
__global__ void __launch_bounds__(256) k_scan_local(const int *__restrict__ in, int n, int *__restrict__ out,
                                                    int *__restrict__ bsum)
{
    __shared__ int warp_tot[8];
    const int base = blockIdx.x * kScanBlock + threadIdx.x * 4;
    int v[4];
#pragma unroll
    for (int i = 0; i < 4; i++) v[i] = base + i < n ? in[base + i] : 0;
    const int tsum = v[0] + v[1] + v[2] + v[3];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    int woff = 0;
    for (int i = 0; i < wid; i++) woff += warp_tot[i];
    int run = woff + incl - tsum;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == 255) bsum[blockIdx.x] = woff + incl;
}

// Phase 2: exclusive scan of the block totals (one CTA, sequential chunks).
__global__ void __launch_bounds__(1024) k_scan_bsum(int *__restrict__ bsum, int nb)
{
    __shared__ int warp_tot[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int c0 = 0; c0 < nb; c0 += 1024) {
        const int e = c0 + threadIdx.x;
        const int v = e < nb ? bsum[e] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        int woff = 0;
        for (int i = 0; i < wid; i++) woff += warp_tot[i];
        const int c = carry;
        if (e < nb) bsum[e] = c + woff + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = c + woff + incl;
        __syncthreads();
    }
}

__global__ void k_scan_add(int *__restrict__ out, int n, const int *__restrict__ bsum)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] += bsum[e / kScanBlock];
}

__global__ void k_fill(const int32_t *__restrict__ idx, int n, int H, int W, int N, const int *__restrict__ off,
                       int *__restrict__ cursor, int *__restrict__ list)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int pos = idx[e];
    if (!block_ok(pos, H, W, N)) return;
    const int slot = atomicAdd(cursor + pos, 1);
    list[off[pos] + slot] = e;
}

// Sort each bucket ascending (fixes the summation order).  A CTA of 256
// positions stages their entries (one contiguous range) in shared memory,
// each thread insertion-sorts its position's bucket there, and the CTA writes
// the range back; a range larger than kSortCap is sorted in place in global
// memory instead.  With slot_of (the planar layout's tables), each thread
// then writes, for its position's sorted entries, slot_of[entry] = its index
// in the sorted list and lpos[index] = the block column of the position; the
// sorted list itself is then not needed and is written back only without.
constexpr int kSortCap = 4096;

__device__ __forceinline__ void insertion_sort(int *v, int b0, int b1)
{
    for (int i = b0 + 1; i < b1; i++) {
        const int x = v[i];
        int j = i - 1;
        while (j >= b0 && v[j] > x) {
            v[j + 1] = v[j];
            j--;
        }
        v[j + 1] = x;
    }
}

__global__ void __launch_bounds__(256) k_sort(const int *__restrict__ off, int npos, int *__restrict__ list, int W,
                                              int *__restrict__ slot_of, int *__restrict__ lpos)
{
    __shared__ int sl[kSortCap];
    const int p0 = blockIdx.x * 256, p = p0 + threadIdx.x, pe = min(p0 + 256, npos);
    const int B0 = off[p0], n = off[pe] - B0;
    const bool tables = slot_of != nullptr;
    if (n <= kSortCap) {
        for (int i = threadIdx.x; i < n; i += 256) sl[i] = list[B0 + i];
        __syncthreads();
        if (p < npos) {
            const int b0 = off[p] - B0, b1 = off[p + 1] - B0;
            insertion_sort(sl, b0, b1);
            if (tables) {
                const int l = p % W;
                for (int i = b0; i < b1; i++) {
                    slot_of[sl[i]] = B0 + i;
                    lpos[B0 + i] = l;
                }
            }
        }
        if (tables) return;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += 256) list[B0 + i] = sl[i];
        return;
    }
    if (p >= npos) return;
    const int b0 = off[p], b1 = off[p + 1];
    insertion_sort(list, b0, b1);
    if (tables) {
        const int l = p % W;
        for (int i = b0; i < b1; i++) {
            slot_of[list[i]] = i;
            lpos[i] = l;
        }
    }
}

struct Win {
    float v[kMaxPatch];
};

__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// One thread per output pixel, eight lanes per 8-pixel row segment: the lanes
// of a segment walk the same block positions and entries together, so each
// patch-row read is a 32-byte sector shared by the 8 lanes (lanes the block
// does not cover sit the entry out).  Per pixel the order is fixed -- block
// rows k ascending, columns l ascending, entries ascending -- and numerator
// and denominator are Kahan-compensated FP32 sums.
constexpr int kSegX = 8, kSegRows = 4; // CTA: 8 segments (64 px) x 4 rows

template <int N>
__global__ void __launch_bounds__(256)
k_gather(const float *__restrict__ groups, const float *__restrict__ w, const int *__restrict__ off,
         const int *__restrict__ list, int log2K, int H, int W, int pitch, Win win, float *__restrict__ out)
{
    __shared__ float sw[N];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < N; i++) sw[i] = win.v[i];
    }
    __syncthreads();
    const int j = threadIdx.x & 7;
    const int x0 = blockIdx.x * (8 * kSegX) + ((threadIdx.x >> 3) & (kSegX - 1)) * 8;
    const int y = blockIdx.y * kSegRows + (threadIdx.x >> 6);
    if (x0 >= W || y >= H) return; // whole segment
    const int x = x0 + j;
    float num = 0.f, cn = 0.f, den = 0.f, cd = 0.f;
    const int ka = max(0, y - (N - 1)), kb = min(y, H - N);
    const int la = max(0, x0 - (N - 1)), lb = min(x0 + 7, W - N);
    for (int k = ka; k <= kb; k++) {
        const int a = y - k;
        const float wa = sw[a];
        const float *grow = groups + a * N;
        for (int l = la; l <= lb; l++) {
            const int b = x - l;
            const bool inb = b >= 0 && b < N && x < W;
            const float wab = inb ? wa * sw[b] : 0.f;
            const int pos = k * W + l;
            const int e0 = __ldg(off + pos), e1 = __ldg(off + pos + 1);
            for (int e = e0; e < e1; e++) {
                const int ent = __ldg(list + e);
                if (inb) {
                    const float wt = __ldg(w + (ent >> log2K)) * wab;
                    const float v = __ldg(grow + (size_t)ent * (N * N) + b);
                    kahan_add(num, cn, wt * v);
                    kahan_add(den, cd, wt);
                }
            }
        }
    }
    if (x < W) out[(size_t)y * pitch + x] = num / den;
}

// The same sums over the planar, position-sorted layout: row a of slot j is
// the N floats at planes + a * plane_stride + N j, its weight w_slot[j], its
// block column lpos[j].  For one block row k the slots of the blocks
// covering pixel x (positions k*W + x-N+1 .. k*W + x) are one contiguous range,
// walked in order (= columns ascending, entries ascending: the same
// per-pixel order as k_gather).
//
// One warp per 32 consecutive pixels of a row.  For each block row k the
// slots covering any of its pixels are again one contiguous range (about
// (N + 31) positions' entries); the warp stages it, up to kCap slots at a
// time, in shared memory (lane i loads slots c0 + i, c0 + i + 32, ...: their
// N values as float4, column and weight -- coalesced), then every lane walks
// the part of its own range inside the staged chunk.  kCap is sized so that
// one chunk holds the whole range in the common case: each lane's walk is
// then one pass, and the warp's time per k is its longest range.
constexpr int kGatherWarps = 8;

template <int N>
struct GatherCfg {
    static constexpr int kCap = N == 8 ? 144 : 88;                  // slots staged per warp (4 CTAs per SM)
    static constexpr int kRowS = N + 1;                              // staged value row stride (odd: fewer conflicts)
    static constexpr int kWarpFloats = kCap * kRowS + 2 * kCap;      // values; (column, weight) pairs
    static constexpr int kSmem = kGatherWarps * kWarpFloats * 4 + 64; // bytes, plus the window
};

// WIN: the window is not flat (stage 2's Kaiser window); stage 1's flat
// window skips the per-contribution lookup (its factors are all 1).
template <int N, bool WIN>
__global__ void __launch_bounds__(kGatherWarps * 32)
k_gather_planar(const float *__restrict__ planes, const float *__restrict__ w_slot, const int *__restrict__ off,
                const int *__restrict__ lpos, long long plane_stride, int H, int W, int pitch, Win win,
                float *__restrict__ out)
{
    constexpr int kCap = GatherCfg<N>::kCap, kRowS = GatherCfg<N>::kRowS;
    extern __shared__ __align__(16) float g_smem[];
    float *sw = g_smem; // window (16 floats)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *sv = g_smem + 16 + warp * GatherCfg<N>::kWarpFloats;
    float2 *scw = reinterpret_cast<float2 *>(sv + kCap * kRowS + (kCap * kRowS & 1)); // (column as int bits, w wa)
    if (threadIdx.x < N) sw[threadIdx.x] = win.v[threadIdx.x];
    __syncthreads();
    const int y = blockIdx.y;
    const int x0 = (blockIdx.x * kGatherWarps + warp) * 32, x = x0 + lane;
    if (x0 >= W) return; // whole warp
    const bool xin = x < W;
    float num = 0.f, cn = 0.f, den = 0.f, cd = 0.f;
    const int ka = max(0, y - (N - 1)), kb = min(y, H - N);
    // block columns covering this lane's pixel, and any pixel of the warp
    const int lo = max(0, x - (N - 1)), hi = min(x, W - N);
    const bool any = xin && lo <= hi;
    const int wlo = max(0, x0 - (N - 1)), whi = min(min(x0 + 31, W - 1), W - N);
    for (int k = ka; k <= kb; k++) {
        const int a = y - k;
        const float wa = sw[a];
        const float *plane = planes + a * plane_stride;
        const int S0 = __ldg(off + k * W + wlo), S1 = __ldg(off + k * W + whi + 1);
        const int s0 = any ? __ldg(off + k * W + lo) : 0, s1 = any ? __ldg(off + k * W + hi + 1) : 0;
        for (int c0 = S0; c0 < S1; c0 += kCap) {
            const int cn_ = min(kCap, S1 - c0);
            for (int i = lane; i < cn_; i += 32) {
                const float4 *src = reinterpret_cast<const float4 *>(plane + (size_t)(c0 + i) * N);
                float *dst = sv + i * kRowS;
#pragma unroll
                for (int v = 0; v < N / 4; v++) {
                    const float4 q = __ldg(src + v);
                    dst[4 * v] = q.x;
                    dst[4 * v + 1] = q.y;
                    dst[4 * v + 2] = q.z;
                    dst[4 * v + 3] = q.w;
                }
                // (w wa) kappa[b]: the same rounding as forming w wa first
                scw[i] = make_float2(__int_as_float(__ldg(lpos + c0 + i)), __ldg(w_slot + c0 + i) * wa);
            }
            __syncwarp();
            const int q0 = max(s0, c0), q1 = min(s1, c0 + cn_);
            for (int q = q0; q < q1; q++) {
                const int jj = q - c0;
                const float2 cw = scw[jj];
                const int b = x - __float_as_int(cw.x);
                const float wt = WIN ? cw.y * sw[b] : cw.y;
                kahan_add(num, cn, wt * sv[jj * kRowS + b]);
                kahan_add(den, cd, wt);
            }
            __syncwarp();
        }
    }
    if (xin) out[(size_t)y * pitch + x] = num / den;
}

} // namespace

// Device address of g_fixed_scratch on the current device.  In host code the
// symbol names a host-side stand-in, so the address is asked of the runtime
// once per device (with that device current) and cached.
cudaError_t fixed_scratch(void **ptr)
{
    constexpr int kMaxDev = 64;
    static std::mutex mu;
    static void *cache[kMaxDev] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < kMaxDev && cache[dev]) {
        *ptr = cache[dev];
        return cudaSuccess;
    }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_fixed_scratch);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDev) cache[dev] = p;
    *ptr = p;
    return cudaSuccess;
}

AggLayout agg_layout(int H, int W, int G, int K, bool with_slots)
{
    AggLayout L{};
    L.npos = H * W;
    const int nscan = L.npos + 1;
    L.nblk = (nscan + kScanBlock - 1) / kScanBlock;
    size_t o = 0;
    L.cnt = o;
    o += align_up((size_t)nscan * sizeof(int));
    L.off = o;
    o += align_up((size_t)nscan * sizeof(int));
    L.cursor = o;
    o += align_up((size_t)nscan * sizeof(int));
    L.list = o;
    o += align_up((size_t)G * K * sizeof(int));
    L.slot_of = o;
    if (with_slots) o += align_up((size_t)G * K * sizeof(int));
    L.lpos = o;
    if (with_slots) o += align_up((size_t)G * K * sizeof(int));
    L.bsum = o;
    o += align_up((size_t)L.nblk * sizeof(int));
    L.bytes = o;
    return L;
}

cudaError_t build_csr(const int32_t *idx, int G, int K, int H, int W, int N, void *agg_ws, bool with_slots,
                      cudaStream_t st)
{
    const AggLayout L = agg_layout(H, W, G, K, with_slots);
    char *base = (char *)agg_ws;
    int *cnt = (int *)(base + L.cnt), *off = (int *)(base + L.off), *cursor = (int *)(base + L.cursor);
    int *list = (int *)(base + L.list), *bsum = (int *)(base + L.bsum), *slot_of = (int *)(base + L.slot_of);
    const int n = G * K, nscan = L.npos + 1;
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)nscan * sizeof(int), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(cursor, 0, (size_t)nscan * sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_count<<<(n + 255) / 256, 256, 0, st>>>(idx, n, H, W, N, cnt);
    k_scan_local<<<L.nblk, 256, 0, st>>>(cnt, nscan, off, bsum);
    k_scan_bsum<<<1, 1024, 0, st>>>(bsum, L.nblk);
    k_scan_add<<<(nscan + 255) / 256, 256, 0, st>>>(off, nscan, bsum);
    k_fill<<<(n + 255) / 256, 256, 0, st>>>(idx, n, H, W, N, off, cursor, list);
    k_sort<<<(L.npos + 255) / 256, 256, 0, st>>>(off, L.npos, list, W, with_slots ? slot_of : nullptr,
                                                  with_slots ? (int *)(base + L.lpos) : nullptr);
    return cudaGetLastError();
}

static Win make_win(const float *window, int N)
{
    Win win{};
    for (int i = 0; i < N; i++) win.v[i] = window[i];
    return win;
}

cudaError_t launch_aggregate(const float *groups, const float *w, const int32_t *idx, int G, int K, int H, int W,
                             int N, int pitch, const float *window, float *out, void *agg_ws, cudaStream_t st)
{
    if (N != 8 && N != 16) return cudaErrorInvalidValue;
    cudaError_t e = build_csr(idx, G, K, H, W, N, agg_ws, false, st);
    if (e != cudaSuccess) return e;
    const AggLayout L = agg_layout(H, W, G, K, false);
    const char *base = (const char *)agg_ws;
    int log2K = 0;
    while ((1 << log2K) < K) log2K++;
    dim3 grid((W + 8 * kSegX - 1) / (8 * kSegX), (H + kSegRows - 1) / kSegRows);
    auto kern = N == 8 ? k_gather<8> : k_gather<16>;
    kern<<<grid, 256, 0, st>>>(groups, w, (const int *)(base + L.off), (const int *)(base + L.list), log2K, H, W,
                               pitch, make_win(window, N), out);
    return cudaGetLastError();
}

cudaError_t launch_aggregate_planar(const float *planes, const float *w_slot, int n_entries, int H, int W, int N,
                                    int pitch, const float *window, float *out, const void *agg_ws, cudaStream_t st)
{
    if (N != 8 && N != 16) return cudaErrorInvalidValue;
    const AggLayout L = agg_layout(H, W, n_entries, 1, true);
    const int *off = (const int *)((const char *)agg_ws + L.off);
    const int *lpos = (const int *)((const char *)agg_ws + L.lpos);
    dim3 grid((W + 32 * kGatherWarps - 1) / (32 * kGatherWarps), H);
    bool flat = true; // every window factor 1 (stage 1): no per-contribution lookup
    for (int i = 0; i < N; i++) flat = flat && window[i] == 1.f;
    auto kern = N == 8 ? (flat ? k_gather_planar<8, false> : k_gather_planar<8, true>)
                       : (flat ? k_gather_planar<16, false> : k_gather_planar<16, true>);
    const int smem = N == 8 ? GatherCfg<8>::kSmem : GatherCfg<16>::kSmem;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kGatherWarps * 32, smem, st>>>(planes, w_slot, off, lpos, (long long)n_entries * N, H, W, pitch,
                                                make_win(window, N), out);
    return cudaGetLastError();
}

} // namespace gbm3d
