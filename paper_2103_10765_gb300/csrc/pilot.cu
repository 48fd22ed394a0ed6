// pilot.cu -- learned pilot: a small convolutional network trained to imitate
// the method's stage-1 estimate (Sec. 3; Sec. 4 uses it as the pilot of the
// Wiener stage), with its own forward, backward and optimiser kernels.
//
// Network (per pixel, zero-padded 3 x 3 convolutions, NHWC activations):
//   x0 = (Z, sigma)  -> conv 2->32 + ReLU -> fourteen conv 32->32 + ReLU
//   -> conv 32->1 = r;  pilot = Z - r;  loss = mean (pilot - Y1)^2
// Weights W[l][tap][ci][co] (tap = 3 (dy+1) + (dx+1)), biases b[l][co], in
// one flat FP32 master vector; every convolution uses the weights rounded
// to BF16.  Activations x1 .. x15 are stored BF16 (NHWC, 64 bytes a pixel,
// rounded to nearest-even by the layer that writes them); accumulation is
// FP32 throughout.  The forward 32 -> 32 layers run on the
// 5th-generation tensor cores (tcgen05.mma, accumulators in tensor memory)
// as implicit GEMMs over 128-pixel row tiles, and so do their backward-data
// passes (the same kernel with the weights flipped and transposed, masked by
// the ReLU of the layer below) and their weight gradients (k_wgrad_tc:
// per-CTA partial sums, then a fixed-order reduction: deterministic).  The
// gradients between the 32-channel layers are stored BF16, like the
// activations.  The thin first and last layers and Adam are SIMT.
#include <cuda_bf16.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include "internal.cuh"

namespace gbm3d {
namespace {

constexpr int kC = 32;      // hidden channels
constexpr int kMid = 14;    // 32 -> 32 layers (receptive field 2 kMid + 5)
constexpr int kW1 = 9 * 2 * kC, kWm = 9 * kC * kC, kW8 = 9 * kC;
// offsets of the flat parameter vector (per layer: weights, then biases)
constexpr int kOffW1 = 0, kOffB1 = kW1;
__host__ __device__ constexpr int off_wm(int m) { return kW1 + kC + m * (kWm + kC); }
__host__ __device__ constexpr int off_bm(int m) { return off_wm(m) + kWm; }
constexpr int kOffW8 = kW1 + kC + kMid * (kWm + kC), kOffB8 = kOffW8 + kW8;
constexpr int kParams = kOffB8 + 1; // 130369

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// four BF16 channels (8 bytes) as FP32
__device__ __forceinline__ float4 ld_bf16x4(const __nv_bfloat16 *p)
{
    const uint2 u = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
    const float2 c = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
    return make_float4(a.x, a.y, c.x, c.y);
}

// ---- weights: BF16 copies in the layouts the kernels read -------------------
// wf[m][tap][co][ci] (forward, 32 -> 32), wb[m][tap][ci][co] = W[m][8 - tap][ci][co]
// (backward data), w1r / w8r: the first / last layer's weights rounded to BF16.
__global__ void k_pack(const float *__restrict__ theta, __nv_bfloat16 *__restrict__ wf,
                       __nv_bfloat16 *__restrict__ wb, float *__restrict__ w1r, float *__restrict__ w8r)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < kMid * kWm) {
        const int m = e / kWm, r = e - m * kWm;
        const int tap = r / (kC * kC), ci = (r / kC) % kC, co = r % kC; // source W[tap][ci][co]
        const __nv_bfloat16 v = __float2bfloat16_rn(theta[off_wm(m) + r]);
        wf[(size_t)m * kWm + (tap * kC + co) * kC + ci] = v;
        wb[(size_t)m * kWm + ((8 - tap) * kC + ci) * kC + co] = v;
    }
    if (e < kW1) w1r[e] = bf16r(theta[kOffW1 + e]);
    if (e < kW8) w8r[e] = bf16r(theta[kOffW8 + e]);
}

// x0[b][y][x] = (Z, sigma_b)
__global__ void k_input(const float *__restrict__ Z, int zpitch, long long zbatch, const float *__restrict__ sigma,
                        float2 *__restrict__ x0, int H, int W)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5), b = blockIdx.z;
    if (x >= W || y >= H) return;
    x0[((size_t)b * H + y) * W + x] = make_float2(Z[b * zbatch + (long long)y * zpitch + x], sigma[b]);
}

// First layer, 2 -> 32, + ReLU, straight from Z and sigma: a CTA of 256
// threads covers 16 pixels of kThinRows rows; it stages the two input
// channels of its tile with the 1-pixel halo in shared memory (zero outside
// the image, the zero padding of both channels), then sixteen lanes per pixel
// compute two output channels each from the 36 weights they hold in
// registers (the 64-byte BF16 output row of a pixel is one coalesced store).
constexpr int kThinRows = 8;

__global__ void __launch_bounds__(256) k_conv_first(const float *__restrict__ Z, int zpitch, long long zbatch,
                                                    const float *__restrict__ sigma, const float *__restrict__ w1r,
                                                    const float *__restrict__ theta, __nv_bfloat16 *__restrict__ x1,
                                                    int H, int W)
{
    __shared__ float2 sx[kThinRows + 2][16 + 2];
    const int b = blockIdx.z, xb = blockIdx.x * 16, yb = blockIdx.y * kThinRows;
    const float sg = sigma[b];
    for (int i = threadIdx.x; i < (kThinRows + 2) * 18; i += 256) {
        const int r = i / 18, c = i - r * 18, yy = yb + r - 1, xx = xb + c - 1;
        const bool inside = yy >= 0 && yy < H && xx >= 0 && xx < W;
        sx[r][c] = inside ? make_float2(Z[b * zbatch + (long long)yy * zpitch + xx], sg) : make_float2(0.f, 0.f);
    }
    const int cp = threadIdx.x & 15, px = threadIdx.x >> 4; // output channels 2 cp, 2 cp + 1 of pixel px
    float2 w[9][2];
#pragma unroll
    for (int tap = 0; tap < 9; tap++)
#pragma unroll
        for (int ci = 0; ci < 2; ci++) w[tap][ci] = reinterpret_cast<const float2 *>(w1r + (tap * 2 + ci) * kC)[cp];
    const float2 bq = reinterpret_cast<const float2 *>(theta + kOffB1)[cp];
    __syncthreads();
    const int x = xb + px;
    if (x >= W) return;
    const int rows = min(kThinRows, H - yb);
    for (int r = 0; r < rows; r++) {
        float2 a = bq;
#pragma unroll
        for (int tap = 0; tap < 9; tap++) {
            const float2 v = sx[r + tap / 3][px + tap % 3];
            a.x = fmaf(v.x, w[tap][0].x, fmaf(v.y, w[tap][1].x, a.x));
            a.y = fmaf(v.x, w[tap][0].y, fmaf(v.y, w[tap][1].y, a.y));
        }
        reinterpret_cast<__nv_bfloat162 *>(x1 + (((size_t)b * H + yb + r) * W + x) * kC)[cp] =
            __floats2bfloat162_rn(fmaxf(a.x, 0.f), fmaxf(a.y, 0.f));
    }
}

// ---- the forward 32 -> 32 convolution on the 5th-generation tensor cores ------
// tcgen05.mma kind::f16 (BF16 inputs, FP32 accumulators in tensor memory):
// per tile of 128 pixels of one image row, M = 128 pixels, N = 32 output
// channels, K = 16 input channels per instruction; 9 taps x 2 channel halves
// = 18 instructions accumulate the whole 3 x 3 x 32 contraction.  Input rows
// (BF16 NHWC in memory) are staged in shared memory as [channel group of
// 8][pixel][8] BF16 (130 pixels with the halo): a tap's shifted 128-pixel
// window is then a K-major operand without swizzle (16-byte core-matrix rows,
// 8-pixel groups 128 bytes apart, channel groups 2080 bytes apart) that
// starts at the tap's row and pixel.  The weights sit once per CTA in the
// same layout ([tap][channel group][output channel][8]).
// Each CTA walks a vertical run of tiles (one 128-pixel column strip, rows
// y0 .. y1) with a ring of 4 staged rows.  A run's first three rows arrive
// by cp.async; after that, each tile's step stores the row fetched into
// registers during the previous step (coalesced 16-byte loads; a cp.async
// here would scatter the two halves of every 32-byte sector to different
// channel groups, doubling the L2 traffic and the shared-memory wavefronts)
// and fetches the next.  Per tile the epilogue (tcgen05.ld, bias, ReLU, BF16
// store) drains one of two 32-column accumulator buffers while the next
// tile's product fills the other.  Every mbarrier wait is bounded; a wait that gives up
// counts in g_conv_timeouts and ends the CTA's work.
__device__ unsigned long long g_conv_timeouts = 0;

constexpr int kCT = 128;                        // pixels per tile (one row segment)
constexpr int kCPix = kCT + 2;                  // staged pixels per row
constexpr int kCGrp = kC / 8;                   // channel groups of 8
constexpr int kCRowBytes = kCGrp * kCPix * 16;  // one staged row (4 groups x 130 pixels x 16 bytes)
constexpr int kCRing = 4;                       // staged rows: 3 in use, 1 being stored
constexpr int kCWBytes = 9 * kCGrp * kC * 16;   // the weights
constexpr int kCTcSmem = kCRing * kCRowBytes + kCWBytes + 64;
constexpr int kCTcPerSm = 4;                    // CTAs per SM (shared memory: 4 x 51.8 KB)
constexpr int kCLd = (kCPix * kCGrp + 127) / 128; // 16-byte chunks of a row per thread (5)
constexpr uint32_t kConvIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kC >> 3) << 17) |
                                ((uint32_t)(kCT >> 4) << 24); // D FP32, A/B BF16, K-major, N 32, M 128
constexpr int kCSpin = 1 << 22;
static_assert(kCRing == 4, "ring slots are row & 3");

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t cdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ bool cbar_wait(uint32_t a, uint32_t parity)
{
    for (int i = 0; i < kCSpin; i++) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (ok) return true;
    }
    return false;
}

// Runs: (image b, strip sx, rows y0 .. y0 + run_len - 1); run j of the batch:
// b = j / (strips * runs_col), then strip, then run within the strip's column.
struct ConvRuns {
    int strips, runs_col, run_len, total;
};

// BWD = false: the forward layer, out = ReLU(conv(in, V) + bias).  BWD =
// true: its backward-data pass, out = conv(in, V) * (mask > 0) with in the
// BF16 gradient at the layer's output, V the flipped, transposed weights and
// mask the layer's input activation (the ReLU of the layer below); bias is
// unused.  Both write BF16.
template <bool BWD>
__global__ void __launch_bounds__(128, kCTcPerSm) k_conv_tc(const __nv_bfloat16 *__restrict__ in,
                                                            const __nv_bfloat16 *__restrict__ V,
                                                            const float *__restrict__ bias,
                                                            const __nv_bfloat16 *__restrict__ mask,
                                                            __nv_bfloat16 *__restrict__ out, int B, int H, int W,
                                                            ConvRuns RN)
{
    extern __shared__ __align__(1024) unsigned char ctsm[];
    unsigned char *s_ring = ctsm, *s_w = ctsm + kCRing * kCRowBytes;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(s_w + kCWBytes);
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(mbar + 2);
    volatile int *s_err = reinterpret_cast<volatile int *>(mbar + 3);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(s_tmem)), "r"(64)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < 2; b++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(mbar + b)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_err = 0;
    }
    // weights: V[tap][co][ci] -> [tap][ci group][co][8]
    for (int i = tid; i < 9 * kC * kCGrp; i += 128) {
        const int g = i & 3, co = (i >> 2) & (kC - 1), tap = i >> 7;
        *reinterpret_cast<uint4 *>(s_w + ((tap * kCGrp + g) * kC + co) * 16) =
            *reinterpret_cast<const uint4 *>(V + (tap * kC + co) * kC + g * 8);
    }
    float bv[kC];
#pragma unroll
    for (int c = 0; c < kC; c++) bv[c] = BWD ? 0.f : bias[c];
    // chunk i of a staged row: channel group i & 3 of pixel i >> 2 (x0 - 1 + i >> 2)
    auto src_of = [&](int b, int yy, int x0, int i, bool &inside) {
        const int xx = x0 + (i >> 2) - 1;
        inside = yy >= 0 && yy < H && xx >= 0 && xx < W;
        return inside ? in + (((size_t)b * H + yy) * W + xx) * kC + (i & 3) * 8 : in;
    };
    auto dst_of = [&](int yy, int i) { // [group][pixel][16 bytes] in ring slot yy & 3
        return s_ring + (yy & (kCRing - 1)) * kCRowBytes + ((i & 3) * kCPix + (i >> 2)) * 16;
    };
    // a run's first rows: cp.async (zero-filled outside the image)
    auto copy_row = [&](int b, int yy, int x0) {
        for (int i = tid; i < kCPix * kCGrp; i += 128) {
            bool inside;
            const __nv_bfloat16 *src = src_of(b, yy, x0, i, inside);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(su32(dst_of(yy, i))), "l"(src),
                         "r"(inside ? 16 : 0)
                         : "memory");
        }
    };
    // later rows: fetched into registers one step ahead, then stored
    uint4 pre[kCLd];
    auto fetch_row = [&](int b, int yy, int x0) {
#pragma unroll
        for (int j = 0; j < kCLd; j++) {
            const int i = tid + 128 * j;
            pre[j] = make_uint4(0, 0, 0, 0);
            bool inside = false;
            const __nv_bfloat16 *src = i < kCPix * kCGrp ? src_of(b, yy, x0, i, inside) : in;
            if (inside) pre[j] = __ldg(reinterpret_cast<const uint4 *>(src));
        }
    };
    auto put_row = [&](int yy) {
#pragma unroll
        for (int j = 0; j < kCLd; j++) {
            const int i = tid + 128 * j;
            if (i < kCPix * kCGrp) *reinterpret_cast<uint4 *>(dst_of(yy, i)) = pre[j];
        }
    };
    // the product of output row y (rows y-1 .. y+1 staged) into accumulator buf (thread 0)
    auto issue = [&](int y, int buf) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = *s_tmem + (uint32_t)(buf * kC);
        const uint32_t rb = su32(s_ring), wb = su32(s_w);
#pragma unroll 1
        for (int tap = 0; tap < 9; tap++) {
            const int dy = tap / 3, dx = tap % 3; // row y + dy - 1, pixel offset dx
            const uint32_t row = rb + ((y + dy - 1) & (kCRing - 1)) * kCRowBytes;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint64_t ad = cdesc(row + 2 * h * kCPix * 16 + dx * 16, kCPix * 16, 128);
                const uint64_t bd = cdesc(wb + ((tap * kCGrp + 2 * h) * kC) * 16, kC * 16, 128);
                const uint32_t acc = (tap | h) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                             "l"(ad), "l"(bd), "r"(kConvIdesc), "r"(acc)
                             : "memory");
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         su32(mbar + buf))
                     : "memory");
    };
    int issued = 0; // products issued by this CTA (thread 0's count; buffer = count & 1)
    int done = 0;   // products waited for
    for (int run = blockIdx.x; run < RN.total && !*s_err; run += gridDim.x) {
        const int b = run / (RN.strips * RN.runs_col), rem = run - b * RN.strips * RN.runs_col;
        const int sx = rem / RN.runs_col, ry = rem - sx * RN.runs_col;
        const int x0 = sx * kCT, y0 = ry * RN.run_len, y1 = min(H, y0 + RN.run_len);
        // input rows y0 - 1 .. y1 are needed: the first three by cp.async, row y0 + 2 into registers
        copy_row(b, y0 - 1, x0);
        copy_row(b, y0, x0);
        copy_row(b, y0 + 1, x0);
        asm volatile("cp.async.commit_group;" ::: "memory");
        if (y0 + 2 <= y1) fetch_row(b, y0 + 2, x0);
        asm volatile("cp.async.wait_all;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) issue(y0, issued & 1);
        issued++;
        for (int y = y0; y < y1; y++) {
            const int buf = done & 1;
            // row y + 2 (the next product's last) into the slot of row y - 2, whose last
            // product (y - 1) has completed; then row y + 3 into registers
            if (y + 1 < y1) {
                put_row(y + 2);
                if (y + 3 <= y1) fetch_row(b, y + 3, x0);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const bool ok = cbar_wait(su32(mbar + buf), (done >> 1) & 1);
            done++;
            if (!ok && lane == 0) {
                *s_err = 1;
                atomicAdd(&g_conv_timeouts, 1ull);
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            __syncthreads();
            if (*s_err) break;
            if (y + 1 < y1) {
                if (tid == 0) issue(y + 1, issued & 1);
                issued++;
            }
            uint32_t v[32];
            const uint32_t taddr = *s_tmem + (uint32_t)(buf * kC) + ((uint32_t)(warp * 32) << 16);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                         "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                         "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
                         "tcgen05.wait::ld.sync.aligned;"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                           "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
                           "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
                           "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                         : "r"(taddr)
                         : "memory");
            const int x = x0 + warp * 32 + lane;
            if (x < W) {
                const size_t pix = ((size_t)b * H + y) * W + x;
                uint4 *o = reinterpret_cast<uint4 *>(out + pix * kC);
#pragma unroll
                for (int q = 0; q < kC / 8; q++) {
                    uint32_t h[4];
                    uint4 mk = make_uint4(0, 0, 0, 0);
                    if (BWD) mk = __ldg(reinterpret_cast<const uint4 *>(mask + pix * kC) + q);
                    const uint32_t mw[4] = {mk.x, mk.y, mk.z, mk.w};
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const int c = 8 * q + 2 * j;
                        float v0, v1;
                        if (BWD) { // the ReLU's derivative: pass where the input activation is positive
                            const float2 m2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&mw[j]));
                            v0 = m2.x > 0.f ? __uint_as_float(v[c]) : 0.f;
                            v1 = m2.y > 0.f ? __uint_as_float(v[c + 1]) : 0.f;
                        } else {
                            v0 = fmaxf(__uint_as_float(v[c]) + bv[c], 0.f);
                            v1 = fmaxf(__uint_as_float(v[c + 1]) + bv[c + 1], 0.f);
                        }
                        __nv_bfloat162 t = __floats2bfloat162_rn(v0, v1);
                        h[j] = *reinterpret_cast<uint32_t *>(&t);
                    }
                    o[q] = make_uint4(h[0], h[1], h[2], h[3]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        }
        __syncthreads(); // the ring is restaged by the next run
    }
    // after a timeout a product may still run: let it finish before its
    // accumulators are released
    if (tid == 0 && *s_err && issued > done) cbar_wait(su32(mbar + ((issued - 1) & 1)), ((issued - 1) >> 1) & 1);
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*s_tmem), "r"(64) : "memory");
}

// Last layer, 32 -> 1: r = b + sum W_last x_last; pilot = Z - r.  A CTA of 256
// threads covers kLX pixels of kThinRows rows: it stages its x_last tile with
// the 1-pixel halo in shared memory (cp.async 16-byte copies, zero outside
// the image), then eight lanes per pixel each take four channels of every
// tap against the 36 weights they hold in registers, and a shuffle sums the
// eight.  With a target: the loss gradient g8 = dL/dr = -2 (pilot - Y1) / n
// and one partial sum of (pilot - Y1)^2 / n per kLX-pixel row segment
// (reduced later in a fixed order).
constexpr int kLX = 32;
constexpr int kLTile = (kThinRows + 2) * (kLX + 2) * kC * 2; // bytes of the staged x_last tile

__global__ void __launch_bounds__(256) k_conv_last(const __nv_bfloat16 *__restrict__ x7, const float *__restrict__ w8r,
                                                   const float *__restrict__ theta, const float *__restrict__ Z,
                                                   int zpitch, long long zbatch, const float *__restrict__ Y1,
                                                   float *__restrict__ pilot, int ppitch, long long pbatch,
                                                   float *__restrict__ g8, float *__restrict__ loss_part, float inv_n,
                                                   int H, int W)
{
    __shared__ __align__(16) unsigned char st[kLTile];
    __shared__ float red[kThinRows][8];
    const int tid = threadIdx.x, b = blockIdx.z, xb = blockIdx.x * kLX, yb = blockIdx.y * kThinRows;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(st);
    for (int i = tid; i < (kThinRows + 2) * (kLX + 2) * 4; i += 256) {
        const int q = i & 3, pr = i >> 2, r = pr / (kLX + 2), c = pr - r * (kLX + 2);
        const int yy = yb + r - 1, xx = xb + c - 1;
        const bool inside = yy >= 0 && yy < H && xx >= 0 && xx < W;
        const __nv_bfloat16 *src = inside ? x7 + (((size_t)b * H + yy) * W + xx) * kC + q * 8 : x7;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sbase + (uint32_t)i * 16), "l"(src),
                     "r"(inside ? 16 : 0)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    const int cq = tid & 7, px = tid >> 3; // channels 4 cq .. 4 cq + 3 of pixel px
    float4 w[9];
#pragma unroll
    for (int tap = 0; tap < 9; tap++) w[tap] = reinterpret_cast<const float4 *>(w8r + tap * kC)[cq];
    const float b8 = theta[kOffB8];
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    const int x = xb + px, rows = min(kThinRows, H - yb);
    for (int r = 0; r < rows; r++) {
        float part = 0.f;
#pragma unroll
        for (int tap = 0; tap < 9; tap++) {
            const float4 u = ld_bf16x4(reinterpret_cast<const __nv_bfloat16 *>(
                                           st + ((r + tap / 3) * (kLX + 2) + px + tap % 3) * kC * 2) +
                                       4 * cq);
            part = fmaf(u.x, w[tap].x, fmaf(u.y, w[tap].y, fmaf(u.z, w[tap].z, fmaf(u.w, w[tap].w, part))));
        }
        // sum over the pixel's eight lanes (fixed order)
        part += __shfl_xor_sync(0xffffffffu, part, 4);
        part += __shfl_xor_sync(0xffffffffu, part, 2);
        part += __shfl_xor_sync(0xffffffffu, part, 1);
        const int y = yb + r;
        float e2 = 0.f;
        if (x < W && cq == 0) {
            const float pv = Z[b * zbatch + (long long)y * zpitch + x] - (b8 + part);
            if (pilot) pilot[b * pbatch + (long long)y * ppitch + x] = pv;
            if (Y1) {
                const float d = pv - Y1[((size_t)b * H + y) * W + x];
                g8[((size_t)b * H + y) * W + x] = -2.f * d * inv_n;
                e2 = d * d * inv_n; // partial sums of the mean
            }
        }
        if (Y1) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
            if ((tid & 31) == 0) red[r][tid >> 5] = e2;
        }
    }
    if (!Y1) return;
    __syncthreads();
    if (tid < rows) {
        const float *q = red[tid];
        loss_part[((size_t)b * H + yb + tid) * gridDim.x + blockIdx.x] =
            ((q[0] + q[1]) + (q[2] + q[3])) + ((q[4] + q[5]) + (q[6] + q[7]));
    }
}

// Backward of the last layer (x7 here names its input x_last, g7 the gradient at
// that input's pre-activation): g7[p][ci] = (sum_tap g8[p - off(tap)] W8[tap][ci]) * (x7[p][ci] > 0);
// eight lanes per pixel, four channels each (coalesced rows), 16 pixels of
// kThinRows rows per CTA.
__global__ void __launch_bounds__(128) k_last_bwd(const float *__restrict__ g8, const float *__restrict__ w8r,
                                                  const __nv_bfloat16 *__restrict__ x7, __nv_bfloat16 *__restrict__ g7,
                                                  int H, int W)
{
    const int cq = threadIdx.x & 7;
    const int x = blockIdx.x * 16 + (threadIdx.x >> 3), b = blockIdx.z;
    if (x >= W) return;
    float4 w[9];
#pragma unroll
    for (int tap = 0; tap < 9; tap++) w[tap] = reinterpret_cast<const float4 *>(w8r + tap * kC)[cq];
    const int y1 = min(H, (blockIdx.y + 1) * kThinRows);
    for (int y = blockIdx.y * kThinRows; y < y1; y++) {
        float gv[9];
#pragma unroll
        for (int tap = 0; tap < 9; tap++) {
            const int yy = y - (tap / 3 - 1), xx = x - (tap % 3 - 1);
            gv[tap] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? g8[((size_t)b * H + yy) * W + xx] : 0.f;
        }
        const size_t p = ((size_t)b * H + y) * W + x;
        const float4 mk = ld_bf16x4(x7 + p * kC + 4 * cq);
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int tap = 0; tap < 9; tap++) {
            acc[0] = fmaf(gv[tap], w[tap].x, acc[0]);
            acc[1] = fmaf(gv[tap], w[tap].y, acc[1]);
            acc[2] = fmaf(gv[tap], w[tap].z, acc[2]);
            acc[3] = fmaf(gv[tap], w[tap].w, acc[3]);
        }
        // the gradient at x7's pre-activation, stored BF16 (the input of the
        // tensor-core backward passes)
        const __nv_bfloat162 lo = __floats2bfloat162_rn(mk.x > 0.f ? acc[0] : 0.f, mk.y > 0.f ? acc[1] : 0.f);
        const __nv_bfloat162 hi = __floats2bfloat162_rn(mk.z > 0.f ? acc[2] : 0.f, mk.w > 0.f ? acc[3] : 0.f);
        reinterpret_cast<uint2 *>(g7 + p * kC)[cq] =
            make_uint2(*reinterpret_cast<const uint32_t *>(&lo), *reinterpret_cast<const uint32_t *>(&hi));
    }
}

// ---- weight gradients of the thin first and last layers ------------------------
// dW[tap][ci][co] = sum_p x[p + off(tap)][ci] g[p][co] and db[co] = sum_p g[p][co].
// A CTA of 256 threads splits the 9 CI CO + CO outputs among its threads
// (each keeps its own few sums in registers) and walks row segments of 128
// pixels (64 for the 32-channel input, keeping the stage under 48 KB) (x with halo and g staged in shared memory) over a strided share
// of the batch, then writes its partial sums; k_reduce adds the CTAs'
// partials in a fixed order.  (The 32 -> 32
// layers use k_wgrad_tc on the tensor cores.)
constexpr int kWgThreads = 256; // threads of a thin-layer weight-gradient CTA

__device__ __forceinline__ float ldf(const float *p) { return *p; }
__device__ __forceinline__ float ldf(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

template <int CI, int CO, typename TX, typename TG>
__global__ void __launch_bounds__(kWgThreads) k_wgrad(const TX *__restrict__ x, const TG *__restrict__ g, int B,
                                                      int H, int W, float *__restrict__ part)
{
    constexpr int kGX = CI >= 16 ? 64 : 128;                   // pixels of a row segment (one unit)
    constexpr int NW = 9 * CI * CO, NO = NW + CO;              // weights, then biases
    constexpr int J = (NO + kWgThreads - 1) / kWgThreads;      // outputs per thread
    constexpr int NX = 3 * (kGX + 2) * CI, NG = kGX * CO;      // staged values
    __shared__ float sx[3][kGX + 2][CI];
    __shared__ float sg[kGX][CO];
    const int tid = threadIdx.x;
    // output o = tid + kWgThreads j: weight (tap, ci, co) or bias co; for
    // consecutive threads co (then ci) runs fastest, so their shared reads are
    // consecutive or broadcast
    int xo[J], go[J];
    bool has[J];
#pragma unroll
    for (int j = 0; j < J; j++) {
        const int o = tid + kWgThreads * j;
        has[j] = o < NO;
        if (o < NW) {
            const int tap = o / (CI * CO), rem = o - tap * CI * CO, ci = rem / CO, co = rem - ci * CO;
            xo[j] = ((tap / 3) * (kGX + 2) + tap % 3) * CI + ci; // + c * CI for pixel c
            go[j] = co;
        } else {
            xo[j] = -1; // bias: x = 1
            go[j] = has[j] ? o - NW : 0;
        }
    }
    float acc[J];
#pragma unroll
    for (int j = 0; j < J; j++) acc[j] = 0.f;
    const float *sxf = &sx[0][0][0];
    const int segs = (W + kGX - 1) / kGX;
    const long long units = (long long)B * H * segs;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const int seg = (int)(u % segs), y = (int)((u / segs) % H), b = (int)(u / ((long long)segs * H));
        const int xb = seg * kGX;
        __syncthreads();
        if constexpr (sizeof(TX) == 2 && CI % 8 == 0) {
            // BF16 activations: 16-byte loads of 8 channels, all of a thread's in flight first
            constexpr int NV = NX / 8, NL = (NV + kWgThreads - 1) / kWgThreads;
            uint4 v[NL];
#pragma unroll
            for (int q = 0; q < NL; q++) {
                const int i = tid + q * kWgThreads;
                const int r = i / ((kGX + 2) * (CI / 8)), rem = i - r * (kGX + 2) * (CI / 8);
                const int c = rem / (CI / 8), ch8 = rem - c * (CI / 8);
                const int yy = y + r - 1, xx = xb + c - 1;
                v[q] = make_uint4(0, 0, 0, 0);
                if (i < NV && yy >= 0 && yy < H && xx >= 0 && xx < W)
                    v[q] = __ldg(reinterpret_cast<const uint4 *>(x + (((size_t)b * H + yy) * W + xx) * CI) + ch8);
            }
#pragma unroll
            for (int q = 0; q < NL; q++) {
                const int i = tid + q * kWgThreads;
                if (i >= NV) continue;
                const uint32_t w4[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
                float *d = &sx[0][0][0] + 8 * i;
#pragma unroll
                for (int h = 0; h < 4; h++) {
                    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w4[h]));
                    d[2 * h] = f.x;
                    d[2 * h + 1] = f.y;
                }
            }
        } else
        // eight loads of a thread in flight before their stores
        for (int i0 = tid; i0 < NX; i0 += 8 * kWgThreads) {
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int i = i0 + q * kWgThreads;
                const int r = i / ((kGX + 2) * CI), rem = i - r * (kGX + 2) * CI, c = rem / CI, ch = rem - c * CI;
                const int yy = y + r - 1, xx = xb + c - 1;
                v[q] = (i < NX && yy >= 0 && yy < H && xx >= 0 && xx < W)
                           ? ldf(x + (((size_t)b * H + yy) * W + xx) * CI + ch)
                           : 0.f;
            }
#pragma unroll
            for (int q = 0; q < 8; q++)
                if (i0 + q * kWgThreads < NX) (&sx[0][0][0])[i0 + q * kWgThreads] = v[q];
        }
        for (int i0 = tid; i0 < NG; i0 += 8 * kWgThreads) {
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int i = i0 + q * kWgThreads, c = i / CO, co = i - c * CO, xx = xb + c;
                v[q] = (i < NG && xx < W) ? ldf(g + (((size_t)b * H + y) * W + xx) * CO + co) : 0.f;
            }
#pragma unroll
            for (int q = 0; q < 8; q++)
                if (i0 + q * kWgThreads < NG) (&sg[0][0])[i0 + q * kWgThreads] = v[q];
        }
        __syncthreads();
        for (int c = 0; c < kGX; c++) {
#pragma unroll
            for (int j = 0; j < J; j++) {
                const float xv = xo[j] >= 0 ? sxf[xo[j] + c * CI] : 1.f;
                acc[j] = fmaf(xv, sg[c][go[j]], acc[j]);
            }
        }
    }
    float *o = part + (size_t)blockIdx.x * NO;
#pragma unroll
    for (int j = 0; j < J; j++)
        if (has[j]) o[tid + kWgThreads * j] = acc[j];
}

// ---- weight gradient of a 32 -> 32 layer on the tensor cores ----------------------
// dW[tap][ci][co] = sum_p x[p + off(tap)][ci] g[p][co] as tcgen05.mma kind::f16
// (BF16 operands, FP32 accumulators in tensor memory), db[co] = sum_p g[p][co].
// A unit is one 128-pixel segment of an image row y (pixels x0 .. x0 + 127):
// the rows y - 1 .. y + 2 of x with a 1-pixel halo (the fourth row only pads
// the M = 128 operand) are staged as [row][channel group][pixel]
// [8 BF16], and the row y of g as [co group][pixel][8].  Both are MN-major
// operands without swizzle (core matrices of 8 channels x 8 pixels, 16-byte
// rows): x's 16 row-and-group blocks sit 130 x 16 bytes apart, so one
// operand of M = 128 rows = (row, ci) spans all three kernel rows; starting
// it dx + 1 pixels into the staged row applies the column offset.  For each
// dx the 8 instructions of K = 16 pixels add x[y + dy][x + dx][ci] g[y][x][co]
// into accumulator dx + 1 (tensor-memory lane 32 (dy + 1) + ci, column co;
// lane 96, whose operand row is a one, sums g: the bias gradient).  Units
// are staged by cp.async into two alternating stages: the next unit's copies
// are in flight while the products of the current one run.  Each CTA takes
// a strided share of the units, then writes one partial row (the layout of
// k_wgrad's), which k_reduce sums in a fixed order: deterministic.
constexpr int kWtPix = kCT + 2;                            // staged pixels of an x row
constexpr int kWtX = 4 * kCGrp * kWtPix * 16;              // staged x rows (33,280 bytes)
constexpr int kWtG = kCGrp * kCT * 16;                     // staged g row (8,192 bytes)
constexpr int kWtStage = kWtX + kWtG;
constexpr int kWtSmem = 2 * kWtStage + 64;
constexpr uint32_t kWtIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                              ((uint32_t)(kC >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
// D FP32; A, B BF16; both MN-major; N = 32; M = 128

__global__ void __launch_bounds__(128, 2) k_wgrad_tc(const __nv_bfloat16 *__restrict__ x,
                                                     const __nv_bfloat16 *__restrict__ g, int B, int H, int W,
                                                     float *__restrict__ part)
{
    extern __shared__ __align__(1024) unsigned char wsm[];
    uint64_t *ready = reinterpret_cast<uint64_t *>(wsm + 2 * kWtStage); // [2] stage staged (128 arrivals)
    uint64_t *done = ready + 2;                                          // [2] products of the stage complete
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(done + 2);
    volatile int *s_err = reinterpret_cast<volatile int *>(s_tmem + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int segs = (W + kCT - 1) / kCT;
    const long long units = (long long)B * H * segs;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(s_tmem)), "r"(128)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < 2; b++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(su32(ready + b)) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(done + b)) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_err = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_tmem;
    int n = 0;         // units of this CTA
    int issued = -1;   // thread 0: the last unit whose products were issued
    // stages unit u into stage st with cp.async (zero fill outside the image);
    // the padding row holds a one in channel 0 (lane 96 of every accumulator
    // then sums g over the unit: the bias gradient)
    auto stage_unit = [&](long long u, int st) {
        unsigned char *sx = wsm + st * kWtStage, *sg = sx + kWtX;
        const int seg = (int)(u % segs), y = (int)((u / segs) % H), b = (int)(u / ((long long)segs * H));
        const int x0 = seg * kCT;
        for (int i = tid; i < 4 * kWtPix * kCGrp; i += 128) { // x: 4 rows x 130 pixels x 4 groups of 16 bytes
            const int grp = i & 3, pix = (i >> 2) % kWtPix, r = (i >> 2) / kWtPix;
            unsigned char *dst = sx + ((r * kCGrp + grp) * kWtPix + pix) * 16;
            if (r == 3) {
                *reinterpret_cast<uint4 *>(dst) = make_uint4(grp == 0 ? 0x3F80u : 0u, 0, 0, 0); // BF16 1.0
                continue;
            }
            const int yy = y + r - 1, xx = x0 + pix - 1;
            const bool inside = yy >= 0 && yy < H && xx >= 0 && xx < W;
            const __nv_bfloat16 *src = inside ? x + (((size_t)b * H + yy) * W + xx) * kC + grp * 8 : x;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(su32(dst)), "l"(src),
                         "r"(inside ? 16 : 0)
                         : "memory");
        }
        for (int i = tid; i < kCT * kCGrp; i += 128) { // g: 128 pixels x 4 groups
            const int grp = i & 3, pix = i >> 2, xx = x0 + pix;
            const __nv_bfloat16 *src = xx < W ? g + (((size_t)b * H + y) * W + xx) * kC + grp * 8 : g;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(su32(sg + (grp * kCT + pix) * 16)),
                         "l"(src), "r"(xx < W ? 16 : 0)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if ((long long)blockIdx.x < units) stage_unit(blockIdx.x, 0);
    for (long long u = blockIdx.x; u < units; u += gridDim.x, n++) {
        const int st = n & 1;
        unsigned char *sx = wsm + st * kWtStage, *sg = sx + kWtX;
        // the next unit's copies go out before this one is consumed: into the
        // other stage, once the products of unit n - 1 have read it
        const long long un = u + gridDim.x;
        if (un < units) {
            if (n >= 1 && !*s_err && !cbar_wait(su32(done + (st ^ 1)), ((n - 1) >> 1) & 1)) {
                *s_err = 1;
                atomicAdd(&g_conv_timeouts, 1ull);
            }
            if (!*s_err) stage_unit(un, st ^ 1);
            else asm volatile("cp.async.commit_group;" ::: "memory"); // keeps the group count
            asm volatile("cp.async.wait_group 1;" ::: "memory");         // this unit's copies have landed
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(ready + st)) : "memory");
        if (tid == 0 && !*s_err) {
            if (!cbar_wait(su32(ready + st), (n >> 1) & 1)) {
                *s_err = 1;
                atomicAdd(&g_conv_timeouts, 1ull);
            } else {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t xb = su32(sx), gb = su32(sg);
#pragma unroll
                for (int d = 0; d < 3; d++)
#pragma unroll
                    for (int ks = 0; ks < kCT / 16; ks++) {
                        // A: MN stride (row-and-group blocks) 130 x 16 bytes, K stride (8 pixels) 128
                        const uint64_t ad = cdesc(xb + d * 16 + ks * 256, 128, kWtPix * 16);
                        const uint64_t bd = cdesc(gb + ks * 256, 128, kCT * 16);
                        const uint32_t acc = (n > 0 || ks > 0) ? 1u : 0u;
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                                         tmem + (uint32_t)(d * kC)),
                                     "l"(ad), "l"(bd), "r"(kWtIdesc), "r"(acc)
                                     : "memory");
                    }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 su32(done + st))
                             : "memory");
                issued = n;
            }
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory"); // no copy may land after the CTA ends
    if (tid == 0 && issued >= 0 && !cbar_wait(su32(done + (issued & 1)), (issued >> 1) & 1)) {
        *s_err = 1;
        atomicAdd(&g_conv_timeouts, 1ull);
    }
    if (tid == 0 && issued != n - 1) *s_err = 1; // a unit was not multiplied
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool ok = !*s_err;
    float *o = part + (size_t)blockIdx.x * (9 * kC * kC + kC);
    if (warp == 3) { // lane 96 (warp 3, lane 0) of accumulator 1: the bias gradient
        uint32_t v[32];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                     "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                     "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
                     "tcgen05.wait::ld.sync.aligned;"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                       "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                       "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
                       "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
                       "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                     : "r"(tmem + ((uint32_t)96 << 16) + (uint32_t)kC)
                     : "memory");
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < kC; c++)
                o[9 * kC * kC + c] = !ok ? __int_as_float(0x7fc00000) : (n == 0 ? 0.f : __uint_as_float(v[c]));
    }
    if (warp < 3) { // kernel row dy + 1 = warp, input channel = lane
#pragma unroll 1
        for (int d = 0; d < 3; d++) {
            uint32_t v[32];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                         "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                         "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
                         "tcgen05.wait::ld.sync.aligned;"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                           "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
                           "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
                           "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                         : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(d * kC))
                         : "memory");
            float *row = o + ((warp * 3 + d) * kC + lane) * kC; // tap 3 (dy + 1) + (dx + 1)
#pragma unroll
            for (int c = 0; c < kC; c += 4) {
                const float nan = __int_as_float(0x7fc00000);
                float4 w4 = n == 0 ? make_float4(0.f, 0.f, 0.f, 0.f)
                                   : make_float4(__uint_as_float(v[c]), __uint_as_float(v[c + 1]),
                                                 __uint_as_float(v[c + 2]), __uint_as_float(v[c + 3]));
                if (!ok) w4 = make_float4(nan, nan, nan, nan); // a product failed: visible in the gradient
                *reinterpret_cast<float4 *>(row + c) = w4;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128) : "memory");
    }
}

// dst[i] = sum over c < nparts of src[c][i] in a fixed order (deterministic):
// four lanes take a quarter of the c range each (ascending c), then the four
// sums are added in lane order.
__global__ void __launch_bounds__(128) k_reduce(const float *__restrict__ src, int nparts, int len,
                                                float *__restrict__ dst)
{
    const int i = blockIdx.x * 32 + (threadIdx.x >> 2), q = threadIdx.x & 3;
    const int per = (nparts + 3) / 4, c0 = q * per, c1 = min(nparts, c0 + per);
    float s = 0.f;
    if (i < len) {
#pragma unroll 8
        for (int c = c0; c < c1; c++) s += __ldg(src + (size_t)c * len + i);
    }
    const float s1 = __shfl_down_sync(0xffffffffu, s, 1), s2 = __shfl_down_sync(0xffffffffu, s, 2),
                s3 = __shfl_down_sync(0xffffffffu, s, 3);
    if (q == 0 && i < len) dst[i] = ((s + s1) + s2) + s3;
}

// Sum of n values in a fixed order by one CTA of 1024 threads: strided
// per-thread sums, then a fixed shared-memory tree (deterministic).
__global__ void __launch_bounds__(1024) k_sum(const float *__restrict__ src, int n, float *__restrict__ dst)
{
    __shared__ float red[1024];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += 1024) s += src[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = 512; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *dst = red[0];
}

// Adam on the flat parameter vector (step t >= 1, bias-corrected).
__global__ void k_adam(float *__restrict__ theta, const float *__restrict__ grad, float *__restrict__ m1,
                       float *__restrict__ m2, int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gv = grad[i];
    const float a = b1 * m1[i] + (1.f - b1) * gv, v = b2 * m2[i] + (1.f - b2) * gv * gv;
    m1[i] = a;
    m2[i] = v;
    theta[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

} // namespace
} // namespace gbm3d

// ---- host side ----------------------------------------------------------------
namespace gbm3d {
namespace {

constexpr int kWgMax = 512; // most CTAs of a weight-gradient launch (partial-sum rows)

struct PilotLayout {
    size_t wf, wb, w1r, w8r, x0, act, g8, ga, gb, part, grad, lpart, loss, bytes;
    size_t plane; // pixels of the batch
    int lparts;   // loss partial sums
};

PilotLayout pilot_layout(int B, int H, int W, bool train)
{
    PilotLayout L{};
    const size_t P = (size_t)B * H * W;
    L.plane = P;
    L.lparts = B * H * ((W + kLX - 1) / kLX);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align_up(bytes);
        return at;
    };
    L.wf = take((size_t)kMid * kWm * 2);
    L.wb = take((size_t)kMid * kWm * 2);
    L.w1r = take(kW1 * 4);
    L.w8r = take(kW8 * 4);
    L.x0 = train ? take(P * 2 * 4) : 0; // (Z, sigma) for the first layer's weight gradient
    // activations x1 .. x_{kMid+1} when training (kept for the backward pass), else two ping-pong buffers
    L.act = take(P * kC * 2 * (train ? kMid + 1 : 2)); // BF16
    if (train) {
        L.g8 = take(P * 4);
        L.ga = take(P * kC * 2); // BF16 gradients between the 32-channel layers
        L.gb = take(P * kC * 2);
        L.part = take((size_t)kWgMax * (kWm + kC) * 4);
        L.grad = take((size_t)kParams * 4);
        L.lpart = take((size_t)L.lparts * 4);
        L.loss = take(4);
    }
    L.bytes = o;
    return L;
}

// Grid of the tensor-core convolutions (forward and backward data): runs of
// rows of each 128-pixel strip, sized so that the runs fill kCTcPerSm CTAs per
// SM (shared memory) once, and one CTA per run.  Sets the shared-memory
// limits of the tensor-core kernels once.
int conv_tc_ctas(int B, int H, int W, ConvRuns &RN)
{
    static int per_dev = 0;
    if (!per_dev) {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            nsm = 148;
        cudaFuncSetAttribute(k_conv_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCTcSmem);
        cudaFuncSetAttribute(k_conv_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCTcSmem);
        cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kWtSmem);
        per_dev = kCTcPerSm * nsm;
    }
    RN.strips = (W + kCT - 1) / kCT;
    const long long cols = (long long)B * RN.strips; // strips in the batch
    // rows per run: the strips' rows spread over about per_dev runs (at least 4 rows)
    long long len = (cols * H + per_dev - 1) / per_dev;
    if (len < 4) len = 4;
    if (len > H) len = H;
    RN.run_len = (int)len;
    RN.runs_col = (H + RN.run_len - 1) / RN.run_len;
    RN.total = (int)(cols * RN.runs_col);
    return RN.total < per_dev ? RN.total : per_dev;
}

int wgrad_ctas()
{
    static int n = 0;
    if (!n) {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            nsm = 148;
        n = 2 * nsm < kWgMax ? 2 * nsm : kWgMax;
    }
    return n;
}

// Forward through the network; with Y1 also the loss pieces (training).
cudaError_t pilot_forward(const float *Z, int B, int H, int W, int zpitch, long long zbatch, const float *sigma,
                          const float *theta, const float *Y1, float *pilot, int ppitch, long long pbatch,
                          char *ws, const PilotLayout &L, bool train, cudaStream_t st)
{
    __nv_bfloat16 *wf = (__nv_bfloat16 *)(ws + L.wf), *wb = (__nv_bfloat16 *)(ws + L.wb);
    float *w1r = (float *)(ws + L.w1r), *w8r = (float *)(ws + L.w8r);
    k_pack<<<(kMid * kWm + 255) / 256, 256, 0, st>>>(theta, wf, wb, w1r, w8r);
    if (train) // x0 = (Z, sigma) for the first layer's weight gradient
        k_input<<<dim3((W + 31) / 32, (H + 7) / 8, B), 256, 0, st>>>(Z, zpitch, zbatch, sigma, (float2 *)(ws + L.x0),
                                                                    H, W);
    __nv_bfloat16 *act = (__nv_bfloat16 *)(ws + L.act);
    auto X = [&](int l) { // x_l, l = 1 .. kMid + 1
        return act + (size_t)(train ? l - 1 : (l - 1) & 1) * L.plane * kC;
    };
    k_conv_first<<<dim3((W + 15) / 16, (H + kThinRows - 1) / kThinRows, B), 256, 0, st>>>(
        Z, zpitch, zbatch, sigma, w1r, theta, X(1), H, W);
    ConvRuns RN;
    const int gtc = conv_tc_ctas(B, H, W, RN);
    for (int m = 0; m < kMid; m++)
        k_conv_tc<false><<<gtc, 128, kCTcSmem, st>>>(X(m + 1), wf + (size_t)m * kWm, theta + off_bm(m), nullptr,
                                                    X(m + 2), B, H, W, RN);
    const float inv_n = 1.f / (float)L.plane;
    k_conv_last<<<dim3((W + kLX - 1) / kLX, (H + kThinRows - 1) / kThinRows, B), 256, 0, st>>>(
        X(kMid + 1), w8r, theta, Z, zpitch, zbatch, Y1, pilot, ppitch, pbatch, train ? (float *)(ws + L.g8) : nullptr,
        train ? (float *)(ws + L.lpart) : nullptr, inv_n, H, W);
    return cudaGetLastError();
}

// Gradient of the loss (after pilot_forward with Y1) into ws grad, and the
// loss into ws loss.
cudaError_t pilot_backward(int B, int H, int W, char *ws, const PilotLayout &L, cudaStream_t st)
{
    const __nv_bfloat16 *act = (const __nv_bfloat16 *)(ws + L.act);
    float *grad = (float *)(ws + L.grad), *part = (float *)(ws + L.part);
    auto X = [&](int l) { return act + (size_t)(l - 1) * L.plane * kC; };
    const __nv_bfloat16 *wb = (const __nv_bfloat16 *)(ws + L.wb);
    const float *w8r = (const float *)(ws + L.w8r);
    float *g8 = (float *)(ws + L.g8);
    __nv_bfloat16 *ga = (__nv_bfloat16 *)(ws + L.ga), *gb = (__nv_bfloat16 *)(ws + L.gb);
    const int nc = wgrad_ctas();
    // loss = sum of the scaled partials (their rows hold (pilot - Y1)^2 / n)
    k_sum<<<1, 1024, 0, st>>>((const float *)(ws + L.lpart), L.lparts, (float *)(ws + L.loss));
    // last layer
    k_wgrad<32, 1, __nv_bfloat16, float><<<nc, kWgThreads, 0, st>>>(X(kMid + 1), g8, B, H, W, part);
    k_reduce<<<(kW8 + 1 + 31) / 32, 128, 0, st>>>(part, nc, kW8 + 1, grad + kOffW8);
    const dim3 g128((W + 15) / 16, (H + kThinRows - 1) / kThinRows, B); // 16 x kThinRows pixels per CTA
    ConvRuns RN;
    const int gtc = conv_tc_ctas(B, H, W, RN);
    k_last_bwd<<<g128, 128, 0, st>>>(g8, w8r, X(kMid + 1), ga, H, W);
    __nv_bfloat16 *gcur = ga, *gnext = gb;
    for (int m = kMid - 1; m >= 0; m--) { // layer m + 2: x_{m+1} -> x_{m+2}; gcur = dL/dpre_{m+2}
        k_wgrad_tc<<<nc, 128, kWtSmem, st>>>(X(m + 1), gcur, B, H, W, part);
        k_reduce<<<(kWm + kC + 31) / 32, 128, 0, st>>>(part, nc, kWm + kC, grad + off_wm(m));
        k_conv_tc<true><<<gtc, 128, kCTcSmem, st>>>(gcur, wb + (size_t)m * kWm, nullptr, X(m + 1), gnext, B, H, W,
                                                   RN);
        __nv_bfloat16 *t = gcur;
        gcur = gnext;
        gnext = t;
    }
    // first layer (gcur = dL/dpre_1)
    k_wgrad<2, 32, float, __nv_bfloat16><<<nc, kWgThreads, 0, st>>>((const float *)(ws + L.x0), gcur, B, H, W, part);
    k_reduce<<<(kW1 + kC + 31) / 32, 128, 0, st>>>(part, nc, kW1 + kC, grad + kOffW1);
    return cudaGetLastError();
}

int pilot_fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return set_error(code, buf);
}

int check_batch(int B, int H, int W)
{
    if (B < 1 || H < 1 || W < 1) return pilot_fail(GBM3D_EINVAL, "pilot: empty batch %d x %d x %d", B, H, W);
    if ((long long)B * H * W * kC >= (1ll << 40)) return pilot_fail(GBM3D_EINVAL, "pilot: batch too large");
    return GBM3D_OK;
}

} // namespace

namespace {
__global__ void k_set(float *d, float v) { *d = v; }
} // namespace

size_t pilot_infer_bytes(int H, int W) { return pilot_layout(1, H, W, false).bytes + 256; }

cudaError_t launch_pilot(const float *Z, int H, int W, int pitch, float sigma, const float *theta, float *pilot,
                         int ppitch, void *ws, cudaStream_t st)
{
    const PilotLayout L = pilot_layout(1, H, W, false);
    float *sdev = (float *)((char *)ws + L.bytes); // the noise level, in the slot after the layout
    k_set<<<1, 1, 0, st>>>(sdev, sigma);
    return pilot_forward(Z, 1, H, W, pitch, 0, sdev, theta, nullptr, pilot, ppitch, 0, (char *)ws, L, false, st);
}

} // namespace gbm3d

using namespace gbm3d;

extern "C" {

int gbm3d_pilot_param_count(void) { return kParams; }

int gbm3d_pilot_workspace_bytes(int B, int H, int W, int train, size_t *bytes)
{
    int s = check_batch(B, H, W);
    if (s) return s;
    if (!bytes) return pilot_fail(GBM3D_EINVAL, "pilot: bytes is NULL");
    *bytes = pilot_layout(B, H, W, train != 0).bytes + 256; // + a slot for the noise levels
    return GBM3D_OK;
}

int gbm3d_pilot_forward(const float *Z, int B, int H, int W, const float *sigma, const float *theta, float *pilot,
                        void *ws, gbm3d_stream_t stream)
{
    int s = check_batch(B, H, W);
    if (s) return s;
    if (!Z || !sigma || !theta || !pilot || !ws) return pilot_fail(GBM3D_EINVAL, "pilot: null pointer argument");
    if (((uintptr_t)ws) % kAlign) return pilot_fail(GBM3D_EINVAL, "pilot: ws must be 256-byte aligned");
    const PilotLayout L = pilot_layout(B, H, W, false);
    const long long n = (long long)H * W;
    cudaError_t e = pilot_forward(Z, B, H, W, W, n, sigma, theta, nullptr, pilot, W, n, (char *)ws, L, false,
                                  (cudaStream_t)stream);
    return e == cudaSuccess ? GBM3D_OK : pilot_fail(GBM3D_ECUDA, "pilot forward: %s", cudaGetErrorString(e));
}

int gbm3d_pilot_loss_grad(const float *Z, const float *Y1, int B, int H, int W, const float *sigma,
                          const float *theta, float *grad, float *loss, void *ws, gbm3d_stream_t stream)
{
    int s = check_batch(B, H, W);
    if (s) return s;
    if (!Z || !Y1 || !sigma || !theta || !ws) return pilot_fail(GBM3D_EINVAL, "pilot: null pointer argument");
    if (((uintptr_t)ws) % kAlign) return pilot_fail(GBM3D_EINVAL, "pilot: ws must be 256-byte aligned");
    const PilotLayout L = pilot_layout(B, H, W, true);
    cudaStream_t st = (cudaStream_t)stream;
    const long long n = (long long)H * W;
    char *base = (char *)ws;
    cudaError_t e = pilot_forward(Z, B, H, W, W, n, sigma, theta, Y1, nullptr, 0, 0, base, L, true, st);
    if (e == cudaSuccess) e = pilot_backward(B, H, W, base, L, st);
    if (e == cudaSuccess && grad)
        e = cudaMemcpyAsync(grad, base + L.grad, (size_t)kParams * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, base + L.loss, 4, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? GBM3D_OK : pilot_fail(GBM3D_ECUDA, "pilot gradient: %s", cudaGetErrorString(e));
}

int gbm3d_pilot_train_step(const float *Z, const float *Y1, int B, int H, int W, const float *sigma, float *theta,
                           float *adam_m, float *adam_v, int step, float lr, float *loss, void *ws,
                           gbm3d_stream_t stream)
{
    if (!adam_m || !adam_v || step < 1 || !(lr > 0.f)) return pilot_fail(GBM3D_EINVAL, "pilot: bad optimiser state");
    int s = gbm3d_pilot_loss_grad(Z, Y1, B, H, W, sigma, theta, nullptr, loss, ws, stream);
    if (s) return s;
    const PilotLayout L = pilot_layout(B, H, W, true);
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<(kParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(theta, (const float *)((char *)ws + L.grad),
                                                                     adam_m, adam_v, kParams, lr, b1, b2, 1e-8f, c1,
                                                                     c2);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBM3D_OK : pilot_fail(GBM3D_ECUDA, "pilot adam: %s", cudaGetErrorString(e));
}

} // extern "C"
