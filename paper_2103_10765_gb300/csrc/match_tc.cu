// match_tc.cu -- block matching on the 5th-generation tensor cores
// (Theorem 1: d(a, b) = ||a||^2 + ||b||^2 - 2 a.b; Sec. 2 eq. dfg, Algorithm 1).
//
// The cross terms a.b of a tile of 128 references (16 grid rows x 8 grid
// columns) against every candidate of the union of their search windows form
// one dense product.  It runs as tcgen05.mma (kind::f16, FP32 accumulators in
// tensor memory): M = 128 references, N = 128 candidates per chunk (two
// candidate rows of 64 columns), K = 64 pixels.  The selection warps read the
// accumulators back with tcgen05.ld, one reference per lane.
//
// Exactness.  The product only ranks; the returned list is the exact one of
// the direct FP32 sum (match.cu), bit for bit:
//  1. Pixels are centred on the tile mean and scaled by a power of two so the
//     largest magnitude lies in [2^12, 2^13) (exact scaling), each block is
//     then centred on its own mean (values below 2^14) and split into two
//     FP16 halves v = hi + lo; three products hi.hi + hi.lo + lo.hi give the
//     product to about 2^-21 relative.
//  2. The mean terms of the distance are added per pair in FP32, and each
//     lane keeps its L (16 for
//     K <= 16, 32 for K <= 32) smallest keys in registers.  Keys below its
//     L-th key plus a margin wait in a small shared-memory queue and are
//     merged sixteen at a time by branch-free sorting networks (identical
//     work in all 32 lanes); merges also record the two smallest keys they
//     drop, the first of which joins the exact re-rank.
//  3. A rigorous bound delta on |key - e*| (e* = the exact-FP32 distance
//     minus the reference's centred norm) certifies the list: if every key
//     left out is provably larger than the (K-1)-th key kept, the true K-1
//     best are kept.  Their exact FP32 distances (same operation order as
//     match.cu) are then recomputed and sorted by (distance, k*W + l).
//  4. A reference that fails the test (near-ties wider than the margin,
//     non-finite input, a timed-out wait) is marked by slot 0 = -1 and
//     re-matched by the direct kernel (k_match_fix).
//
// Work split: a CTA of 4 selection warps and one issuing warp (two CTAs per
// SM); selection warp w owns tensor-memory lanes 32w..32w+31, i.e.
// references 32w..32w+31, an 8-row x 4-column block of the tile, and selects
// only on the chunks and 8-column steps that its references' windows reach.
// No CTA-wide barrier per chunk: the selection threads arrive on an
// mbarrier when they have built the next chunk's operand rows, each warp
// arrives on another when it has read a chunk's accumulators, and the
// issuing warp starts the product of chunk c + 1 once chunk c + 1 is built
// and the buffer it overwrites (chunk c - 1's) is consumed, so warps whose
// windows miss a chunk run ahead instead of waiting.  Every thread also builds
// one candidate row of the FP16 operand tiles (core-matrix layout, no
// swizzle) and thread 0 issues the MMAs.  Two accumulator buffers of 128
// columns alternate: the MMAs of chunk c+1 run while the warps select on
// chunk c.  Chunks are visited nearest-first to each warp's references so
// that thresholds tighten early.  Every mbarrier wait is bounded; on a
// timeout the tile falls back to the direct kernel.  Device counters record
// timeouts and re-matched references.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <float.h>
#include <limits.h>

#include <mutex>
#include <string.h>

#include "internal.cuh"

namespace gbm3d {

__device__ unsigned long long g_tc_timeouts = 0;  // bounded waits that gave up
__device__ unsigned long long g_tc_rematched = 0; // references handed to the direct kernel

namespace {

constexpr int kTileY = 16, kTileX = 8, kM = kTileY * kTileX; // references per tile (MMA M)
constexpr int kChunkRows = 2, kChunkCols = 64, kNc = kChunkRows * kChunkCols; // candidates per chunk (MMA N)
constexpr int kKd = kPatch * kPatch;                       // contraction length
constexpr int kRegStride = kChunkCols + kPatch;            // region row stride (floats)
constexpr int kOp = kM * kKd * 2;                          // bytes of one FP16 operand tile (128 x 64)
constexpr int kThreads = 128;                             // 4 selection warps: warp w owns tensor-memory lanes 32w..32w+31
constexpr int kCta = kThreads + 32;                        // + one warp that issues the products
constexpr int kDBuf = 2;                                   // accumulator buffers
constexpr uint32_t kTmemCols = 256;                        // power-of-two allocation >= kDBuf * kNc
constexpr int kPend = 24, kFlushAt = 16;                   // per-lane pending keys (checked every 8 columns)
static_assert(kFlushAt - 1 + 8 <= kPend && kPend - 1 - 16 < kFlushAt, "one 16-key merge per flush keeps the queue bounded");
constexpr int kSpin = 1 << 20;                             // bounded mbarrier polling
constexpr unsigned kFull = 0xffffffffu;

static_assert(kNc == kM, "operand tiles of A and B share one layout");
static_assert(kDBuf * kNc <= (int)kTmemCols, "accumulators exceed the tensor-memory allocation");

// Instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1),
// A and B FP16 (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kNc >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);

// Byte offset of element row n, K-chunk a (8 FP16 = one block row) in an
// operand tile: 8 x 16-byte core matrices, K-chunks 128 bytes apart (leading
// byte offset), 8-row groups 1024 bytes apart (stride byte offset).
__device__ __forceinline__ int op_off(int n, int a) { return (n >> 3) * 1024 + a * 128 + (n & 7) * 16; }

// Shared-memory matrix descriptor for a K-major, non-swizzled tile starting
// at shared address addr: start >> 4 (bits 0-13), leading byte offset 128
// (bits 16-29), stride byte offset 1024 (bits 32-45), fixed 0b001 at 46-48,
// base offset 0, swizzle none (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t a)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t a, uint32_t parity)
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

// Waits for the phase of parity `parity` to complete; gives up (returns
// false, sets *err, counts the timeout) after kSpin polls, or at once when
// *err is already set (err may be null: no early exit).
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int *err)
{
    for (int it = 0; it < kSpin; it++) {
        if (err && *err) return false;
        if (mbar_test(a, parity)) return true;
    }
    if (err) *err = 1;
    atomicAdd(&g_tc_timeouts, 1ull);
    return false;
}

// One tiled TMA load of a 2-D box of the image (coordinates: column x,
// row y; x * 4 bytes is a multiple of 16) into shared memory at dst,
// completing on the mbarrier at bar, which expects `bytes`.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar,
                                            uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                 "[%4];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                 "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(acc)
                 : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 lanes (lane t: row
// 32 (warp % 4) + t), waited for inside the same statement so that no use of
// the registers can be scheduled before the load completes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                 "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                   "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                   "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
                   "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                   "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr)
                 : "memory");
}

// 8 consecutive accumulator columns of this warp's 32 lanes (see tmem_ld32).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr)
                 : "memory");
}

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

__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// The direct kernel's step: acc += (x + nr)^2 on both halves (nr = -r).
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

__device__ __forceinline__ unsigned range_mask(int lo, int hi)
{
    lo = lo < 0 ? 0 : lo;
    hi = hi > 31 ? 31 : hi;
    if (lo > hi) return 0u;
    return (kFull >> (31 - hi)) & (kFull << lo);
}

// Splits 8 scaled values into FP16 high and low halves (v = hi + lo + O(2^-22 v)).
__device__ __forceinline__ void split8(const float (&v)[8], uint4 &hi, uint4 &lo)
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int t = 0; t < 4; t++) {
        const __half2 hh = __floats2half2_rn(v[2 * t], v[2 * t + 1]);
        const float2 hf = __half22float2(hh);
        const __half2 ll = __floats2half2_rn(v[2 * t] - hf.x, v[2 * t + 1] - hf.y);
        h[t] = *reinterpret_cast<const uint32_t *>(&hh);
        l[t] = *reinterpret_cast<const uint32_t *>(&ll);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Compare-exchange: (a, ia) <= (b, ib) by key afterwards (ties: either order;
// the certified re-rank decides ties exactly).
__device__ __forceinline__ void cex(float &a, int &ia, float &b, int &ib)
{
    const bool sw = b < a;
    const float ta = sw ? b : a, tb = sw ? a : b;
    const int tia = sw ? ib : ia, tib = sw ? ia : ib;
    a = ta;
    b = tb;
    ia = tia;
    ib = tib;
}

// Batcher's odd-even merge sort of 16 keys (63 compare-exchanges).
__device__ __forceinline__ void sort16(float (&k)[16], int (&v)[16])
{
#define CX(i, j) cex(k[i], v[i], k[j], v[j])
    CX(0, 1); CX(2, 3); CX(0, 2); CX(1, 3);
    CX(1, 2); CX(4, 5); CX(6, 7); CX(4, 6);
    CX(5, 7); CX(5, 6); CX(0, 4); CX(2, 6);
    CX(2, 4); CX(1, 5); CX(3, 7); CX(3, 5);
    CX(1, 2); CX(3, 4); CX(5, 6); CX(8, 9);
    CX(10, 11); CX(8, 10); CX(9, 11); CX(9, 10);
    CX(12, 13); CX(14, 15); CX(12, 14); CX(13, 15);
    CX(13, 14); CX(8, 12); CX(10, 14); CX(10, 12);
    CX(9, 13); CX(11, 15); CX(11, 13); CX(9, 10);
    CX(11, 12); CX(13, 14); CX(0, 8); CX(4, 12);
    CX(4, 8); CX(2, 10); CX(6, 14); CX(6, 10);
    CX(2, 4); CX(6, 8); CX(10, 12); CX(1, 9);
    CX(5, 13); CX(5, 9); CX(3, 11); CX(7, 15);
    CX(7, 11); CX(3, 5); CX(7, 9); CX(11, 13);
    CX(1, 2); CX(3, 4); CX(5, 6); CX(7, 8);
    CX(9, 10); CX(11, 12); CX(13, 14);
#undef CX
}

// lk (ascending, LP keys) <- the LP smallest of lk and the 16 keys pk:
// sort pk, take min(lk[LP-16+t], pk[15-t]) (a bitonic sequence holding the
// LP smallest), then a bitonic merge.  (x1, i1) and x2 track the smallest
// key ever dropped (with its candidate) and the second smallest.
// Branch-free, identical work in every lane.
template <int LP>
__device__ __forceinline__ void merge16(float (&lk)[LP], int (&li)[LP], float (&pk)[16], int (&pi)[16],
                                        float &x1, int &i1, float &x2)
{
    sort16(pk, pi);
#pragma unroll
    for (int t = 0; t < 16; t++) {
        const float a = lk[LP - 16 + t], b = pk[15 - t];
        const int ia = li[LP - 16 + t], ib = pi[15 - t];
        const bool sw = b < a;
        lk[LP - 16 + t] = sw ? b : a;
        li[LP - 16 + t] = sw ? ib : ia;
        const float d = sw ? a : b; // dropped
        const int id = sw ? ia : ib;
        const bool lt = d < x1;
        x2 = lt ? x1 : fminf(x2, d);
        i1 = lt ? id : i1;
        x1 = lt ? d : x1;
    }
#pragma unroll
    for (int st = LP / 2; st > 0; st >>= 1)
#pragma unroll
        for (int i = 0; i < LP; i++)
            if ((i & st) == 0) cex(lk[i], li[i], lk[i + st], li[i + st]);
}

} // namespace

// Shared-memory layout of one tile (byte offsets from the 1024-aligned base).
struct TcLayout {
    int reg_rows, L;
    int a_hi, a_lo, b_hi, b_lo, reg, nb, nbm, ntb, pk, pi, misc, bytes;
    int lk, li; // after the main loop the lists reuse the operand tiles
};

namespace {

// LP: register list capacity (power of two); LT: keys kept per reference.
template <int LP, int LT>
__global__ void __launch_bounds__(kCta, 2)
k_match_tc(const float *__restrict__ img, int H, int W, int pitch, int By, int Bx, int s, int R, int K,
           TcLayout lay, int32_t *__restrict__ idx, float *__restrict__ dist,
           const __grid_constant__ CUtensorMap tmap, int use_tma)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int L = LT;
    const int p0 = blockIdx.y * kTileY, q0 = blockIdx.x * kTileX;
    const int nP = min(kTileY, By - p0), nQ = min(kTileX, Bx - q0);
    const int iF = grid_pos(p0, s, H, kPatch), iL = grid_pos(p0 + nP - 1, s, H, kPatch);
    const int jF = grid_pos(q0, s, W, kPatch), jL = grid_pos(q0 + nQ - 1, s, W, kPatch);
    // union of the tile's search windows (candidate top-lefts)
    const int uy0 = max(0, iF - R), uy1 = min(H - kPatch, iL + R);
    const int ux0 = max(0, jF - R), ux1 = min(W - kPatch, jL + R);
    const int UH = uy1 - uy0 + 1, UW = ux1 - ux0 + 1; // UW <= kChunkCols (host check)
    const int nch = (UH + kChunkRows - 1) / kChunkRows;
    const int rrows = nch * kChunkRows + kPatch - 1; // region rows read by the chunks (<= lay.reg_rows)

    // region row y, column x (image pixel (uy0 + y, ux0 + x)) at reg[y * kRegStride + x];
    // a TMA box starts at the 16-byte aligned column xa <= ux0, so the
    // region begins ux0 - xa floats into the buffer (the host admits TMA only
    // where the columns read, x <= UW + 6, stay inside the box)
    const int xa = ux0 & ~3;
    float *reg = reinterpret_cast<float *>(smem + lay.reg) + (use_tma ? ux0 - xa : 0);
    // per candidate of the last three chunks: centred norm, -8 mean, -(8 mean + sum / 4)
    float *nbs = reinterpret_cast<float *>(smem + lay.nb);  // [3][kNc]
    float *nbm = reinterpret_cast<float *>(smem + lay.nbm); // [3][kNc]
    float *ntb = reinterpret_cast<float *>(smem + lay.ntb); // [3][kNc]
    float *pk = reinterpret_cast<float *>(smem + lay.pk);    // [kPend][kM] pending keys
    unsigned short *pi = reinterpret_cast<unsigned short *>(smem + lay.pi); // their candidate numbers
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + lay.misc);        // [2] products done
    uint64_t *mb_built = reinterpret_cast<uint64_t *>(smem + lay.misc + 16); // next chunk's operand built
    uint64_t *mb_used = reinterpret_cast<uint64_t *>(smem + lay.misc + 40);  // [2] accumulators read
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + lay.misc + 32);
    volatile int *s_err = reinterpret_cast<volatile int *>(smem + lay.misc + 36);
    float *s_red = reinterpret_cast<float *>(smem + lay.misc + 64); // [4]
    int *s_order = reinterpret_cast<int *>(smem + lay.misc + 128);  // chunk processing order
    uint64_t *mb_tma = reinterpret_cast<uint64_t *>(smem + lay.misc + 56); // region loaded
    const uint32_t sbase = smem_u32(smem);

    if (warp == 0) tmem_alloc(smem_u32(s_tmem), kTmemCols);
    const bool selw = tid < kThreads; // a selection thread (else the issuing warp)
    if (tid == 0) {
        for (int b = 0; b < kDBuf; b++) {
            mbar_init(smem_u32(&mbar[b]), 1);
            mbar_init(smem_u32(&mb_used[b]), kThreads / 32);
        }
        mbar_init(smem_u32(mb_built), kThreads);
        mbar_init(smem_u32(mb_tma), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_err = 0;
        // the search region: one TMA box of lay.reg_rows x kRegStride pixels
        // from (xa, uy0), zero outside the image
        if (use_tma)
            tma_load_2d(smem_u32(smem + lay.reg), &tmap, xa, uy0, smem_u32(mb_tma),
                        (uint32_t)(lay.reg_rows * kRegStride * 4));
    }

    // ---- search region (raw pixels, zero outside the image) and its mean
    const int vrows = UH + kPatch - 1, vcols = UW + kPatch - 1; // pixels of the union's blocks
    float sum = 0.f;
    if (!use_tma) { // eight loads per thread in flight before their stores
        constexpr int kLd = 8;
        const int total = rrows * kRegStride;
        for (int e0 = tid; selw && e0 < total; e0 += kLd * kThreads) {
            float v[kLd];
#pragma unroll
            for (int u = 0; u < kLd; u++) {
                const int e = e0 + u * kThreads;
                const int y = e / kRegStride, x = e - y * kRegStride;
                const int gy = uy0 + y, gx = ux0 + x;
                v[u] = (e < total && gy < H && gx < W) ? __ldg(img + (size_t)gy * pitch + gx) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kLd; u++) {
                const int e = e0 + u * kThreads;
                if (e < total) {
                    const int y = e / kRegStride, x = e - y * kRegStride;
                    reg[e] = v[u];
                    if (y < vrows && x < vcols) sum += v[u];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    bool tma_ok = true;
    if (use_tma) { // every thread waits for the box (bounded), then the sum
        tma_ok = __syncthreads_and(mbar_wait(smem_u32(mb_tma), 0, nullptr));
        for (int e = tid; tma_ok && selw && e < vrows * vcols; e += kThreads) {
            const int y = e / vcols, x = e - y * vcols;
            sum += reg[y * kRegStride + x];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
    if (lane == 0 && selw) s_red[warp] = sum;
    __syncthreads();
    const uint32_t tmem = *s_tmem;
    float mu = 0.f;
    for (int w = 0; w < kThreads / 32; w++) mu += s_red[w];
    mu /= (float)(vrows * vcols);
    float mx = 0.f;
    for (int e = tid; selw && e < vrows * vcols; e += kThreads) {
        const int y = e / vcols, x = e - y * vcols;
        mx = fmaxf(mx, fabsf(reg[y * kRegStride + x] - mu));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
    __syncthreads(); // every thread has read the sums
    if (lane == 0 && selw) s_red[warp] = mx;
    __syncthreads();
    float maxabs = 0.f;
    for (int w = 0; w < kThreads / 32; w++) maxabs = fmaxf(maxabs, s_red[w]);
    int ex = 0;
    frexpf(maxabs, &ex);
    // power-of-two scale: the largest tile-centred magnitude in [2^12, 2^13),
    // so block-centred values stay below 2^14, inside FP16 range
    const float sc = maxabs > 0.f ? ldexpf(1.f, 13 - ex) : 1.f;
    const float vt = maxabs * sc * 1.0001f; // bound on every tile-centred scaled value
    const bool bad = !tma_ok || !isfinite(mu) || !isfinite(maxabs) || ex > 100 || ex < -100 ||
                     !(fabsf(mu) * sc < 1e30f);
    const float nms = -mu * sc; // fma(x, sc, nms) = (x - mu) sc, rounded once

    // ---- this thread's reference (tensor-memory lane tid) and its window
    // warp w owns an 8-row x 4-column block of the tile (rows 8 (w >> 1) ..,
    // columns 4 (w & 1) ..), so that its references' windows cover about 30
    // of the tile's chunks and 48 of the 64 candidate columns of each
    const int m = tid;
    const int rr = 8 * (m >> 6) + ((m & 31) >> 2), rc = 4 * ((m >> 5) & 1) + (m & 3);
    const bool vref = rr < nP && rc < nQ;
    const int ri = vref ? grid_pos(p0 + rr, s, H, kPatch) : 0;
    const int rj = vref ? grid_pos(q0 + rc, s, W, kPatch) : 0;
    const int iy = ri - uy0, ix = rj - ux0;

    // One block (src: its top-left in the region) -> tile-centred scaled
    // values v = (x - mu) sc, their mean m, and the block-centred values
    // v - m, written as FP16 halves into row n of the operand tiles at
    // (off_hi, off_lo); returns their sum of squares and their sum.  The
    // distance splits exactly as |a - b|^2 = |a~ - b~|^2 + 2 (m_a - m_b)
    // (S_a - S_b) + 64 (m_a - m_b)^2 (a~ = a - m_a, S_a = sum of a~), so the
    // product only sees the small within-block parts.
    // src must address an in-bounds block even when valid is false.
    auto centre = [&](const float *src, bool valid, int off_hi, int off_lo, int n, float &n2, float &mean,
                      float &ssum) {
        const f2 sc2 = pack2(sc, sc), nms2 = valid ? pack2(nms, nms) : 0ull;
        const f2 scv = valid ? sc2 : 0ull; // an invalid block is all zeros
        // pass 1: row sums of v (two columns per packed operation)
        f2 acc = 0ull;
#pragma unroll
        for (int a = 0; a < kPatch; a++) {
            const float *r = src + a * kRegStride;
            f2 rs = fma2(pack2(r[0], r[1]), scv, nms2);
#pragma unroll
            for (int b = 2; b < kPatch; b += 2) rs = add2(rs, fma2(pack2(r[b], r[b + 1]), scv, nms2));
            acc = add2(acc, rs);
        }
        float s0, s1;
        unpack2(acc, s0, s1);
        mean = (s0 + s1) * (1.f / kKd);
        // pass 2: the same v again, centred, split, summed
        const f2 nm2 = pack2(-mean, -mean);
        f2 q2 = 0ull, sq = 0ull;
#pragma unroll
        for (int a = 0; a < kPatch; a++) {
            const float *r = src + a * kRegStride;
            float t[8];
#pragma unroll
            for (int b = 0; b < kPatch; b += 2) {
                const f2 tv = add2(fma2(pack2(r[b], r[b + 1]), scv, nms2), nm2);
                q2 = fma2(tv, tv, q2);
                sq = add2(sq, tv);
                unpack2(tv, t[b], t[b + 1]);
            }
            uint4 hi, lo;
            split8(t, hi, lo);
            *reinterpret_cast<uint4 *>(smem + off_hi + op_off(n, a)) = hi;
            *reinterpret_cast<uint4 *>(smem + off_lo + op_off(n, a)) = lo;
        }
        float q0, q1;
        unpack2(q2, q0, q1);
        n2 = q0 + q1;
        unpack2(sq, q0, q1);
        ssum = q0 + q1;
    };

    // ---- reference operand A (thread m builds reference m) and the chunk order
    float ra2 = 0.f, a8 = 0.f, ta = 0.f; // reference: centred norm, 8 m_a, 8 m_a + S_a / 4
    if (!bad && selw) {
        float mean, ssum;
        // a padding lane (no reference) reads the region's first block, which
        // is in bounds, and zeroes it
        centre(vref ? reg + iy * kRegStride + ix : reg, vref, lay.a_hi, lay.a_lo, m, ra2, mean, ssum);
        a8 = 8.f * mean;
        ta = a8 + 0.25f * ssum;
    }
    // chunk order: each chunk's rank is its distance (in chunks) to the
    // nearest warp's own reference rows, so that every warp meets the
    // candidates closest to its references first and its threshold tightens
    // early (the result does not depend on the order)
    if (tid < nch) {
        int cw[4];
#pragma unroll
        for (int w = 0; w < 4; w++) {
            const int r0 = min(8 * (w >> 1), nP - 1), r1 = min(8 * (w >> 1) + 7, nP - 1);
            const int mid = (grid_pos(p0 + r0, s, H, kPatch) + grid_pos(p0 + r1, s, H, kPatch)) / 2 - uy0;
            cw[w] = min(nch - 1, max(0, mid / kChunkRows));
        }
        auto key = [&](int u) {
            int k = INT_MAX;
#pragma unroll
            for (int w = 0; w < 4; w++) k = min(k, abs(u - cw[w]));
            return k;
        };
        const int kt = key(tid);
        int rank = 0;
        for (int u = 0; u < nch; u++) {
            const int ku = key(u);
            rank += (ku < kt || (ku == kt && u < tid)) ? 1 : 0;
        }
        s_order[rank] = tid;
    }
    __syncthreads();

    // builds the candidate operand rows of chunk ch (thread n = candidate n)
    // and their per-candidate terms into buffer par
    auto build = [&](int ch, int par) {
        const int n = tid;
        // columns past the union (never inside a window) repeat its last
        // column, so no read leaves the region's columns 0 .. UW + 6
        const int rowl = ch * kChunkRows + (n >> 6), col = min(n & (kChunkCols - 1), UW - 1);
        float n2, mean, ssum;
        centre(reg + rowl * kRegStride + col, true, lay.b_hi, lay.b_lo, n, n2, mean, ssum);
        nbs[par * kNc + n] = n2;
        nbm[par * kNc + n] = -8.f * mean;
        ntb[par * kNc + n] = -(8.f * mean + 0.25f * ssum);
    };
    // issues the twelve MMAs of one chunk into accumulator buffer b (thread 0)
    auto issue = [&](int b) {
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * kNc);
        const uint32_t ah = sbase + lay.a_hi, al = sbase + lay.a_lo;
        const uint32_t bh = sbase + lay.b_hi, bl = sbase + lay.b_lo;
#pragma unroll
        for (int t = 0; t < kKd / 16; t++) { // K = 16 FP16 per instruction = two K-chunks
            mma_f16(d, smem_desc(ah + t * 256), smem_desc(bh + t * 256), t > 0 ? 1u : 0u);
            mma_f16(d, smem_desc(ah + t * 256), smem_desc(bl + t * 256), 1u);
            mma_f16(d, smem_desc(al + t * 256), smem_desc(bh + t * 256), 1u);
        }
        mma_commit(smem_u32(&mbar[b]));
    };

    // ---- selection state: this lane's window in union coordinates
    int ky_lo = 1, ky_hi = 0;
    unsigned colm0 = 0, colm1 = 0;
    if (vref) {
        ky_lo = max(0, ri - R) - uy0;
        ky_hi = min(H - kPatch, ri + R) - uy0;
        const int kx_lo = max(0, rj - R) - ux0, kx_hi = min(W - kPatch, rj + R) - ux0;
        colm0 = range_mask(kx_lo, kx_hi);
        colm1 = range_mask(kx_lo - 32, kx_hi - 32);
    }
    const unsigned self0 = (ix >= 0 && ix < 32) ? ~(1u << ix) : kFull;
    const unsigned self1 = (ix >= 32 && ix < 64) ? ~(1u << (ix - 32)) : kFull;
    int wlo = vref ? ky_lo : INT_MAX, whi = vref ? ky_hi : -1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        wlo = min(wlo, __shfl_xor_sync(kFull, wlo, o));
        whi = max(whi, __shfl_xor_sync(kFull, whi, o));
    }
    const int wc_lo = whi >= 0 ? wlo / kChunkRows : 1, wc_hi = whi >= 0 ? whi / kChunkRows : 0;
    // the warp's candidate columns, in steps of 8: cs_lo .. cs_hi of the chunk row's 8
    int xlo = vref ? max(0, rj - R) - ux0 : INT_MAX, xhi = vref ? min(W - kPatch, rj + R) - ux0 : -1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        xlo = min(xlo, __shfl_xor_sync(kFull, xlo, o));
        xhi = max(xhi, __shfl_xor_sync(kFull, xhi, o));
    }
    const int cs_lo = xhi >= 0 ? xlo >> 3 : 0, ncs = xhi >= 0 ? (xhi >> 3) - cs_lo + 1 : 0;
    const float kInf = __int_as_float(0x7f800000);
    // this lane's LP best keys so far, ascending, in registers (static indices only)
    float lkr[LP];
    int lir[LP];
#pragma unroll
    for (int t = 0; t < LP; t++) {
        lkr[t] = kInf;
        lir[t] = 0;
    }
    // delta(x) bounds |key - (exact FP32 distance - |a~|^2)| for a key x
    // (scaled units): product rounding and accumulation, the centring and
    // mean roundings, the norm sums and the direct sum's own rounding, each
    // bounded through |a~|^2 and x + |a~|^2
    const float na = sqrtf(ra2);
    auto delta = [&](float x) {
        const float dd = fabsf(x) + ra2, r = sqrtf(dd + 1.f);
        return 1.2e-4f * ra2 + 7e-5f * dd + 4e-6f * vt * r + 3e-6f * (na + r) + 1e-30f;
    };
    float thr = kInf;   // the LT-th best key so far
    float thr_q = kInf; // keys below thr + 2.5 delta(thr) are queued: every key never
                        // queued is above the final one of these
    float x1 = kInf, x2 = kInf; // the two smallest keys merges have dropped
    int i1 = 0;                 // the candidate of x1
    int np = 0;         // pending keys of this lane (shared memory)

    // merges every lane's sixteen oldest pending keys into its list: once when
    // a lane's queue reached kFlushAt (at most 23 pending, at most 7 left, so
    // the queue of kPend = 24 never overflows and the next merge waits until
    // more lanes have keys), until every queue is empty when drain is set
    auto flush = [&](bool drain) {
        do {
            float pkr[16];
            int pir[16];
#pragma unroll
            for (int t = 0; t < 16; t++) {
                const bool h = t < np;
                pkr[t] = h ? pk[t * kM + m] : kInf;
                pir[t] = h ? (int)pi[t * kM + m] : 0;
            }
#pragma unroll
            for (int t = 16; t < kPend; t++)
                if (t < np) {
                    pk[(t - 16) * kM + m] = pk[t * kM + m];
                    pi[(t - 16) * kM + m] = pi[t * kM + m];
                }
            np = np > 16 ? np - 16 : 0;
            merge16<LP>(lkr, lir, pkr, pir, x1, i1, x2);
            thr = lkr[LT - 1];
            thr_q = thr < kInf ? thr + 2.5f * delta(thr) : kInf;
        } while (drain && __any_sync(kFull, np > 0));
    };

    // ---- pipeline: MMA(c + 1) runs while the warps select on chunk c
    const bool issuer = tid == kThreads; // lane 0 of the issuing warp
    int last_issued = -1;                // issuer only
    if (!bad) {
        if (selw) build(s_order[0], 0);
        fence_async_smem();
        __syncthreads();
        if (issuer) {
            issue(0);
            last_issued = 0;
        }
    }
    if (!bad && issuer) {
        // product c + 1 into buffer (c + 1) & 1: its operand rows are built
        // (phase c of mb_built) and chunk c - 1, which used that buffer, is read
        for (int c = 0; c + 1 < nch; c++) {
            if (!mbar_wait(smem_u32(mb_built), c & 1, s_err)) break;
            if (c >= 1 && !mbar_wait(smem_u32(&mb_used[(c + 1) & 1]), ((c - 1) >> 1) & 1, s_err)) break;
            issue((c + 1) & 1);
            last_issued = c + 1;
        }
    }
    for (int c = 0; c < (bad || !selw ? 0 : nch); c++) {
        const int b = c & 1;
        const bool ok = __all_sync(kFull, mbar_wait(smem_u32(&mbar[b]), (c >> 1) & 1, s_err));
        tc_fence_after();
        // the product of chunk c is done: its operand tile is free for chunk c + 1
        if (c + 1 < nch) {
            if (!*s_err) build(s_order[c + 1], (c + 1) % 3);
            fence_async_smem();
            mbar_arrive(smem_u32(mb_built));
        }
        // select on chunk c: 8 columns per step; the final step of the last
        // chunk only merges what is still pending (one copy of the merge code)
        const int ch = s_order[c];
        const int nsteps = (ok && ch >= wc_lo && ch <= wc_hi) ? kChunkRows * ncs : 0;
        const int nst = nsteps + (c == nch - 1 ? 1 : 0);
        const uint32_t tcol = tmem + (uint32_t)(b * kNc) + ((uint32_t)(warp * 32) << 16);
        const int pb = (c % 3) * kNc;
        const f2 a8x2 = pack2(a8, a8), tax2 = pack2(ta, ta), m2x2 = pack2(-2.f, -2.f);
#pragma unroll 1
        for (int st = 0; st < nst; st++) {
            if (st < nsteps) {
                // step st: chunk row st / ncs, columns 8 cs .. 8 cs + 7 of it
                const int r2 = st >= ncs ? 1 : 0, cs = cs_lo + st - r2 * ncs;
                const int col8 = r2 * kChunkCols + 8 * cs; // column of the chunk (accumulator, terms)
                const int j8 = (cs & 3) * 8;
                const int rowl = ch * kChunkRows + r2;
                const int h = cs >> 2;
                unsigned msk = 0u;
                if (rowl >= ky_lo && rowl <= ky_hi) {
                    msk = h ? colm1 : colm0;
                    if (rowl == iy) msk &= h ? self1 : self0;
                }
                msk >>= j8;
                uint32_t v[8];
                tmem_ld8(tcol + (uint32_t)col8, v);
                // e = |b~|^2 + d (d + (S_a - S_b) / 4) - 2 a~.b~ with d = 8 (m_a - m_b):
                // the block-centred key, two columns per packed FP32 operation
                const ulonglong2 *qn = reinterpret_cast<const ulonglong2 *>(nbs + pb + col8);
                const ulonglong2 *qm = reinterpret_cast<const ulonglong2 *>(nbm + pb + col8);
                const ulonglong2 *qt = reinterpret_cast<const ulonglong2 *>(ntb + pb + col8);
                const ulonglong2 n0 = qn[0], n1 = qn[1], m0 = qm[0], m1 = qm[1], t0 = qt[0], t1 = qt[1];
                const f2 nn[4] = {n0.x, n0.y, n1.x, n1.y}, mm[4] = {m0.x, m0.y, m1.x, m1.y};
                const f2 tt[4] = {t0.x, t0.y, t1.x, t1.y};
                float ev[8];
#pragma unroll
                for (int jp = 0; jp < 4; jp++) {
                    const f2 dd = add2(a8x2, mm[jp]);
                    const f2 bb = fma2(dd, add2(tax2, tt[jp]), nn[jp]);
                    const f2 ee = fma2(pack2(__uint_as_float(v[2 * jp]), __uint_as_float(v[2 * jp + 1])), m2x2, bb);
                    unpack2(ee, ev[2 * jp], ev[2 * jp + 1]);
                }
                const int cbase = rowl * kChunkCols + h * 32 + j8;
#pragma unroll
                for (int jj = 0; jj < 8; jj++) {
                    const float e = ev[jj];
                    if (((msk >> jj) & 1u) && e < thr_q) {
                        pk[np * kM + m] = e;
                        pi[np * kM + m] = (unsigned short)(cbase + jj);
                        np++;
                    }
                }
            }
            const bool fin = st == nsteps; // the last chunk's final step drains every queue
            if (__any_sync(kFull, np >= kFlushAt || (fin && np > 0))) flush(fin);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&mb_used[b]));
    }

    // ---- the lists move to shared memory (over the operand tiles, whose last
    // product has completed); after a timeout the last product may still be running: let it finish
    // before its operand tiles are overwritten and its accumulators released
    if (issuer && *s_err && last_issued >= 0)
        mbar_wait(smem_u32(&mbar[last_issued & 1]), (last_issued >> 1) & 1, nullptr);
    fence_async_smem();
    __syncthreads();
    const bool err = *s_err != 0;
    float *lk = reinterpret_cast<float *>(smem + lay.lk); // [LT][kM] keys, then exact distances
    int *li = reinterpret_cast<int *>(smem + lay.li);
    int cnt = 0;
    if (selw) { // (the issuing warp holds no list)
#pragma unroll
        for (int t = 0; t < LT; t++) {
            lk[t * kM + m] = lkr[t];
            li[t * kM + m] = lir[t];
            cnt += lkr[t] < kInf ? 1 : 0;
        }
        // the smallest dropped key joins the exact re-rank (slot LT; it is not
        // below any kept key: the list only ever takes smaller keys)
        if (x1 < kInf) {
            lk[LT * kM + m] = x1;
            li[LT * kM + m] = i1;
            cnt++;
        }
    }

    if (vref) {
        const size_t gq = ((size_t)(p0 + rr) * Bx + q0 + rc) * K;
        bool ovf = bad || err;
        if (!ovf && cnt >= L) {
            // certify: every key left out (dropped by a merge and not x1: >= x2;
            // never queued: >= thr_q, which only decreased) is provably above
            // the (K-1)-th kept one.  (A list that never filled left nothing out.)
            const float T = lk[(K - 2) * kM + m], X = fminf(x2, thr_q);
            ovf = !(X - delta(X) > T + delta(T));
        }
        if (ovf) {
            idx[gq] = -1; // re-matched by the direct kernel
            atomicAdd(&g_tc_rematched, 1ull);
        } else {
            // exact FP32 distances, in the direct kernel's operation order
            f2 nr[kPatch][kPatch / 2];
#pragma unroll
            for (int a = 0; a < kPatch; a++)
#pragma unroll
                for (int b = 0; b < kPatch / 2; b++)
                    nr[a][b] = pack2(-reg[(iy + a) * kRegStride + ix + 2 * b], -reg[(iy + a) * kRegStride + ix + 2 * b + 1]);
            for (int q = 0; q < cnt; q++) {
                const int ci = li[q * kM + m];
                const int ky = ci >> 6, kx = ci & (kChunkCols - 1);
                const float *xr = reg + ky * kRegStride + kx;
                f2 acc = 0ull;
#pragma unroll
                for (int a = 0; a < kPatch; a++)
#pragma unroll
                    for (int b = 0; b < kPatch / 2; b++)
                        acc = sqdiff_acc2(nr[a][b], pack2(xr[a * kRegStride + 2 * b], xr[a * kRegStride + 2 * b + 1]), acc);
                float e0, e1;
                unpack2(acc, e0, e1);
                lk[q * kM + m] = e0 + e1;
                li[q * kM + m] = (uy0 + ky) * W + ux0 + kx;
            }
            // sort by (distance, position); the keys were already nearly in order
            for (int a = 1; a < cnt; a++) {
                const float dv = lk[a * kM + m];
                const int iv = li[a * kM + m];
                int b = a;
                while (b > 0) {
                    const float pd = lk[(b - 1) * kM + m];
                    const int pv = li[(b - 1) * kM + m];
                    if (!key_less(dv, iv, pd, pv)) break;
                    lk[b * kM + m] = pd;
                    li[b * kM + m] = pv;
                    b--;
                }
                lk[b * kM + m] = dv;
                li[b * kM + m] = iv;
            }
            idx[gq] = ri * W + rj;
            if (dist) dist[gq] = 0.f;
            for (int t = 0; t < K - 1; t++) {
                const bool have = t < cnt;
                idx[gq + 1 + t] = have ? li[t * kM + m] : INT_MAX;
                if (dist) dist[gq + 1 + t] = have ? lk[t * kM + m] : kInf;
            }
        }
    }
    // a region load that never completed may still land: wait for it (again
    // bounded) before the shared memory is released
    if (use_tma && !tma_ok && tid == 0) mbar_wait(smem_u32(mb_tma), 0, nullptr);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

} // namespace

TcLayout tc_layout(int H, int s, int R, int K)
{
    TcLayout t{};
    int uh = (kTileY - 1) * s + 2 * R + 1;
    if (uh > H - kPatch + 1) uh = H - kPatch + 1;
    if (uh < 1) uh = 1;
    t.reg_rows = (uh + kChunkRows - 1) / kChunkRows * kChunkRows + kPatch - 1;
    t.L = K <= 16 ? 16 : 32; // kept keys (K - 1 of them are returned)
    int o = 0;
    t.a_hi = o;
    o += kOp;
    t.a_lo = o;
    o += kOp;
    t.b_hi = o;
    o += kOp;
    t.b_lo = o;
    o += kOp;
    t.reg = o;
    o += t.reg_rows * kRegStride * 4;
    o = (o + 15) / 16 * 16;
    t.nb = o;
    o += 3 * kNc * 4;
    t.nbm = o;
    o += 3 * kNc * 4;
    t.ntb = o;
    o += 3 * kNc * 4;
    t.pk = o;
    o += kPend * kM * 4;
    t.pi = o;
    o += kPend * kM * 2;
    o = (o + 15) / 16 * 16;
    t.misc = o; // mbarriers, tensor-memory address, flags, reductions, chunk order
    o += 128 + 4 * 128;
    t.bytes = o;
    t.lk = t.a_hi; // after the loop: lists (L kept + 1 dropped) over the operand tiles
    t.li = t.lk + (t.L + 1) * kM * 4;
    return t;
}

bool match_tc_supported(int H, int W, int N, int s, int R, int K)
{
    (void)W;
    if (N != kPatch || K < 2 || K > kMaxK) return false;
    if ((kTileX - 1) * s + 2 * R + 1 > kChunkCols) return false; // union width must fit one chunk row
    const TcLayout t = tc_layout(H, s, R, K);
    if ((t.reg_rows - kPatch + 1) / kChunkRows > 128) return false; // chunk order table
    return t.bytes <= 227 * 1024;
}

// cuTensorMapEncodeTiled from the driver (through the runtime, so the
// library needs no link to libcuda), looked up once.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

// Tensor map of the image for the region loads: 2-D FP32 (W columns, H rows,
// row pitch `pitch` floats), box kRegStride x reg_rows, zero fill outside.
// False where TMA does not apply: a base address not 16-byte aligned, a row
// pitch that is not a multiple of 16 bytes, a box past the 256 limit, or a
// union wider than the box holds after the up-to-3-column alignment shift.
static bool region_tensor_map(const float *img, int H, int W, int pitch, int s, int R, const TcLayout &lay,
                              CUtensorMap *map)
{
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || ((uintptr_t)img & 15) || (pitch & 3) || lay.reg_rows > 256) return false;
    if ((kTileX - 1) * s + 2 * R + 1 + (kPatch - 1) + 3 > kRegStride) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kRegStride, (cuuint32_t)lay.reg_rows};
    const cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(img), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_match_tc(const float *img, int H, int W, int pitch, int By, int Bx, int s, int R, int K,
                            int32_t *idx, float *dist, cudaStream_t st)
{
    const TcLayout lay = tc_layout(H, s, R, K);
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof tmap);
    const int use_tma = region_tensor_map(img, H, W, pitch, s, R, lay, &tmap) ? 1 : 0;
    // the operand tiles and pending keys alone take over a third of the SM's
    // shared memory: at most two CTAs per SM, 2 x 256 tensor-memory columns
    auto kern = lay.L == 16 ? k_match_tc<16, 16> : k_match_tc<32, 32>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, lay.bytes);
    if (e != cudaSuccess) return e;
    dim3 grid((Bx + kTileX - 1) / kTileX, (By + kTileY - 1) / kTileY);
    kern<<<grid, kCta, lay.bytes, st>>>(img, H, W, pitch, By, Bx, s, R, K, lay, idx, dist, tmap, use_tma);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_match_fix(img, H, W, pitch, By, Bx, s, R, K, idx, dist, st);
}

cudaError_t tc_stats(unsigned long long *timeouts, unsigned long long *rematched)
{
    cudaError_t e = cudaMemcpyFromSymbol(timeouts, g_tc_timeouts, sizeof *timeouts);
    if (e != cudaSuccess) return e;
    return cudaMemcpyFromSymbol(rematched, g_tc_rematched, sizeof *rematched);
}

} // namespace gbm3d
