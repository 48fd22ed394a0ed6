// ht.cu -- stage-1 global volume hard thresholding (Sec. 3.1 eq. BM3DHT,
// cycle spinning U_h = S_{-h} T^-1 Upsilon T S_h V, TV weights w = 1/TV).
//
// The volume of matched blocks is never materialised: the level-1 analysis
// gathers each voxel V[pN+a, qN+b, r] = Z[k_r+a, l_r+b] straight from the
// image through the match list (the image and list stay in L2), with the
// cycle-spin shift folded into the index arithmetic.  Each level of the
// periodic 3-D transform (bior1.5 x bior1.5 x Haar, Mallat) is one kernel
// over tiles of output positions (analysis 8 x 64, synthesis 16 x 32) and one
// pair of slices along the group axis; rows and columns use the lifting form
// of bior1.5
//   d[n]  = (x[2n] - x[2n+1]) / sqrt2,  a0[n] = (x[2n] + x[2n+1]) / sqrt2,
//   a[n]  = a0[n] + (3 d[n-2] - 22 d[n-1] + 22 d[n+1] - 3 d[n+2]) / 128,
// and its exact inverse.  Each thread of a lifting pass slides along one line
// in registers (every pair's d and a0 computed once); shared-memory row
// strides are chosen so that the passes that read across rows are
// conflict-free.  Detail bands are hard-thresholded as they are written.
//
// The level-1 synthesis writes the filtered blocks into a group-major
// buffer (averaging the spins); one last pass per group (a warp) reads the
// group, computes its TV weight and, for the aggregation, copies its rows
// into the position-sorted planar layout.
#include "internal.cuh"

namespace gbm3d {
namespace {

constexpr float kS = 0.70710678118654752f; // 1/sqrt(2)
constexpr float kU1 = 0.171875f;           // 22/128
constexpr float kU2 = 0.0234375f;          // 3/128
constexpr int TY = 16, TX = 32;            // output positions per tile
constexpr int HY = TY + 4, HX = TX + 4;    // synthesis band tile with halo 2: 20 x 36
constexpr int SB = HX + 1;                 // its shared row stride (odd)
constexpr int SO = 2 * TX + 1;             // synthesis output row stride (odd)
// band tiles of the synthesis lie SBB floats apart: with the 14-float gap the
// two band rows that the lanes of one x-inverse warp read fall on distinct banks
constexpr int SBB = HY * SB + 14;
static_assert(2 * 2 * TY * SO <= 8 * SBB, "the y-pass output fits over the band tiles");

// Periodic index (eq. (1)).  Tile halos reach at most a few samples past
// either end, so one conditional add or subtract suffices unless the axis is
// shorter than the halo (coarse levels of tiny images): then the true modulo,
// kept out of line so that it is never executed speculatively.
__device__ __noinline__ int pwrap_slow(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

__device__ __forceinline__ int pwrap(int i, int n)
{
    if (i < 0) i += n;
    if (i >= n) i -= n;
    if ((unsigned)i >= (unsigned)n) i = pwrap_slow(i, n);
    return i;
}

// Pixel offset k*pitch + l of every match-list entry (once per call, so the
// gathers need no division).
__global__ void k_offsets(const int32_t *__restrict__ idx, int n, int H, int W, int N, int pitch,
                          int *__restrict__ ofs)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    int k, l;
    block_kl(idx[e], H, W, N, k, l);
    ofs[e] = k * pitch + l;
}

// Lifting update U(d)[n] from the four detail values d[n-2], d[n-1], d[n+1], d[n+2].
__device__ __forceinline__ float lift_u(float dm2, float dm1, float dp1, float dp2)
{
    return kU2 * (dm2 - dp2) + kU1 * (dp1 - dm1);
}

// Level analysis: input (Z, Y, X) -> 8 bands [band][Z/2][Y/2][X/2], band =
// 4 hz + 2 hy + hx, for one tile of ATY x ATX output positions and one slice
// pair.  GATHER: the input is the cycle-spun mosaic of blocks of side 2^LN
// read from the image through the pixel offsets of the match list (level 1);
// otherwise a [Z][Y][X] plane stack.  vec: X/2 is a multiple of 4 (float4
// stores).
//
// Thread xx < AIX holds input column xx of both slices in registers (its
// loads all in flight at once), applies the Haar step along z and the
// lifting along y there and writes the four (z band, y band) columns to
// shared memory; then the CTA's 256 x-pass jobs (row, chunk of 8 output
// columns) slide the x lifting along their rows (float4 reads, a row stride
// of 4 mod 8 floats so the eight rows of a quarter warp hit distinct banks),
// threshold and store.  A CTA has kAnaThreads = 160 threads: AIX = 136 of
// them gather, so few wait at the barrier while the gathers are in flight,
// and the small CTAs fit seven to an SM (each thread takes one or two x-pass
// jobs).
constexpr int ATY = 8, ATX = 64;                    // analysis output positions per tile
constexpr int AIY = 2 * ATY + 8, AIX = 2 * ATX + 8; // its input tile: 24 x 136
constexpr int ASX = AIX + 4;                        // y-pass output row stride (140)
constexpr int kAnaThreads = 160;                    // threads of an analysis CTA (AIX gather, all the x pass)
static_assert(AIX <= kAnaThreads && kAnaThreads <= 256 && (ASX & 7) == 4, "analysis tile");

// SHIFT (GATHER only): the cycle-spin shift.  Tiles start at multiples of 8
// output rows, i.e. of 16 input rows, so the first input row's place inside
// its mosaic block (N <= 16 rows) is (-4 - SHIFT) mod N for every tile: which
// block each input row falls in is known at compile time, and a thread keeps
// its column's block offsets in registers instead of looking one up per load.
template <bool GATHER, int LN, int SHIFT = 0>
__global__ void __launch_bounds__(kAnaThreads)
k_dwt_ana(const float *__restrict__ src, const float *__restrict__ img, int pitch, const int *__restrict__ ofs,
          int Bx, int shift, int Y, int X, int Z, float *__restrict__ dst, float tau, int vec)
{
    __shared__ __align__(16) float s_y[2][2][ATY][ASX]; // [z band][y band][output row][input col]
    const int m = blockIdx.z;                           // slice pair
    const int y0 = blockIdx.y * ATY, x0 = blockIdx.x * ATX;
    const int iy0 = 2 * y0 - 4, ix0 = 2 * x0 - 4;
    const int tid = threadIdx.x;

    // Gather: the tile's input rows and columns span at most OY x OX blocks
    // of the mosaic (4 x 18 for N = 8, 3 x 10 for N = 16; an N-aligned block
    // wraps as a whole), whose pixel offsets for the two slices are staged in
    // shared memory first; every voxel is then one image load.
    constexpr int NB = 1 << LN;
    constexpr int OY = ((NB + AIY - 2) >> LN) + 1, OX = ((NB + AIX - 2) >> LN) + 1;
    __shared__ int s_ofs[OY][OX][2];
    int z0 = 2 * m, z1 = 2 * m + 1;
    const int uy0 = iy0 - shift, ux0 = ix0 - shift;
    const int ybase = (uy0 >> LN) << LN, xbase = (ux0 >> LN) << LN; // floor to a block
    if (GATHER) {
        z0 = pwrap(z0 - shift, Z);
        z1 = pwrap(z1 - shift, Z);
        for (int e = tid; e < OY * OX * 2; e += blockDim.x) {
            const int ry = e / (2 * OX), rem = e - ry * (2 * OX), rx = rem >> 1, zz = rem & 1;
            const int gy = pwrap(ybase + NB * ry, Y) >> LN, gx = pwrap(xbase + NB * rx, X) >> LN;
            s_ofs[ry][rx][zz] = __ldg(ofs + (size_t)(gy * Bx + gx) * Z + (zz ? z1 : z0));
        }
        __syncthreads();
    }
    if (tid < AIX) { // z and y passes on input column xx
        const int xx = tid;
        float v0[AIY], v1[AIY];
        if (GATHER) {
            static_assert((2 * ATY) % NB == 0, "tile rows start on a block boundary of the mosaic");
            constexpr int kB0 = ((-4 - SHIFT) % NB + NB) % NB; // uy0 - ybase in every tile
            const int dx = ux0 + xx - xbase, rx = dx >> LN;
            const float *colimg = img + (dx & (NB - 1));
            int o0[OY], o1[OY]; // this column's block offsets, both slices
#pragma unroll
            for (int ry = 0; ry < OY; ry++) {
                o0[ry] = s_ofs[ry][rx][0];
                o1[ry] = s_ofs[ry][rx][1];
            }
#pragma unroll
            for (int yy = 0; yy < AIY; yy++) {
                const int dy = kB0 + yy, ry = dy >> LN; // both known at compile time
                const float *b = colimg + (size_t)(dy & (NB - 1)) * pitch;
                v0[yy] = __ldg(b + o0[ry]);
                v1[yy] = __ldg(b + o1[ry]);
            }
        } else {
            const int x = pwrap(ix0 + xx, X);
            const float *r0 = src + (size_t)z0 * Y * X + x, *r1 = src + (size_t)z1 * Y * X + x;
#pragma unroll
            for (int yy = 0; yy < AIY; yy++) {
                const size_t y = (size_t)pwrap(iy0 + yy, Y) * X;
                v0[yy] = __ldg(r0 + y);
                v1[yy] = __ldg(r1 + y);
            }
        }
        // Haar along z (band zb), then along y: output row o uses pairs o .. o+4
#pragma unroll
        for (int zb = 0; zb < 2; zb++) {
            float d[AIY / 2], a0[AIY / 2];
#pragma unroll
            for (int n = 0; n < AIY / 2; n++) {
                const float u = (zb ? v0[2 * n] - v1[2 * n] : v0[2 * n] + v1[2 * n]) * kS;
                const float v = (zb ? v0[2 * n + 1] - v1[2 * n + 1] : v0[2 * n + 1] + v1[2 * n + 1]) * kS;
                d[n] = (u - v) * kS;
                a0[n] = (u + v) * kS;
            }
#pragma unroll
            for (int o = 0; o < ATY; o++) {
                s_y[zb][0][o][xx] = a0[o + 2] + lift_u(d[o], d[o + 1], d[o + 3], d[o + 4]);
                s_y[zb][1][o][xx] = d[o + 2];
            }
        }
    }
    __syncthreads();

    // x pass: 256 jobs, job = 32 chunk + (z band, y band, output row); a job
    // slides over 12 pairs to make 8 output columns
    const int Zo = Z >> 1, Yo = Y >> 1, Xo = X >> 1;
    const size_t E = (size_t)Zo * Yo * Xo;
    for (int job = tid; job < 256; job += kAnaThreads) {
        const int row = job & 31, chunk = job >> 5;
        const int zb = row >> 4, yb = (row >> 3) & 1, o = row & 7;
        const float4 *sr = reinterpret_cast<const float4 *>(&s_y[zb][yb][o][16 * chunk]);
        float d[12], a0[12];
#pragma unroll
        for (int q = 0; q < 6; q++) {
            const float4 t = sr[q];
            d[2 * q] = (t.x - t.y) * kS;
            a0[2 * q] = (t.x + t.y) * kS;
            d[2 * q + 1] = (t.z - t.w) * kS;
            a0[2 * q + 1] = (t.z + t.w) * kS;
        }
        const int band = zb * 4 + yb * 2;
        float lo[8], hi[8];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const float a = a0[j + 2] + lift_u(d[j], d[j + 1], d[j + 3], d[j + 4]);
            const float h = d[j + 2];
            lo[j] = (band == 0 || fabsf(a) >= tau) ? a : 0.f;
            hi[j] = (fabsf(h) >= tau) ? h : 0.f;
        }
        const int yo = y0 + o, xo = x0 + 8 * chunk;
        if (yo >= Yo || xo >= Xo) continue;
        float *pl = dst + band * E + ((size_t)m * Yo + yo) * Xo + xo;
        float *ph = pl + E;
        if (vec && xo + 8 <= Xo) {
            reinterpret_cast<float4 *>(pl)[0] = make_float4(lo[0], lo[1], lo[2], lo[3]);
            reinterpret_cast<float4 *>(pl)[1] = make_float4(lo[4], lo[5], lo[6], lo[7]);
            reinterpret_cast<float4 *>(ph)[0] = make_float4(hi[0], hi[1], hi[2], hi[3]);
            reinterpret_cast<float4 *>(ph)[1] = make_float4(hi[4], hi[5], hi[6], hi[7]);
        } else {
#pragma unroll
            for (int j = 0; j < 8; j++)
                if (xo + j < Xo) {
                    pl[j] = lo[j];
                    ph[j] = hi[j];
                }
        }
    }
}

// Level synthesis: 8 bands [band][Zc][Yc][Xc] -> (2Zc, 2Yc, 2Xc) for one tile
// of 16 x 32 coefficient positions and one slice pair.  SCATTER (level 1):
// the voxel at spun position (z,y,x) belongs to mosaic position
// (z,y,x) - shift, i.e. block r = z of group (y/N, x/N) at (y%N, x%N), with
// N = 2^LN; it is written (or added) scaled into out, which is group-major
// (out.base[((g K + r) N + row) N + col]).
template <bool SCATTER, int LN>
__global__ void __launch_bounds__(256, 4) // four CTAs per SM: at most 64 registers a thread
k_dwt_syn(const float *__restrict__ coef, int Yc, int Xc, int Zc, float *__restrict__ dst, GroupOut out, int Bx,
          int shift, float scale, int accumulate)
{
    __shared__ float s_b[8 * SBB];       // band tiles with halo (band stride SBB); later the y-pass output
    __shared__ float s_x[2][2][HY][SO];  // after the x inverse: [z band][y band][coef row][output col]
    const int m = blockIdx.z;
    const int y0 = blockIdx.y * TY, x0 = blockIdx.x * TX;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t E = (size_t)Zc * Yc * Xc;

    { // warp w loads band w (eight warps, eight bands): its HY halo rows, all of a
      // thread's loads in flight before any store
        const int band = warp;
        const int xa = pwrap(x0 - 2 + lane, Xc), xb = pwrap(x0 - 2 + 32 + (lane & 3), Xc);
        const float *bsrc = coef + band * E + (size_t)m * Yc * Xc;
        float va[HY], vb[HY];
        if (y0 >= 2 && y0 - 2 + HY <= Yc) { // no row wraps: rows HY apart by a fixed stride
            const float *src = bsrc + (size_t)(y0 - 2) * Xc;
#pragma unroll
            for (int yy = 0; yy < HY; yy++) {
                va[yy] = __ldg(src + xa);
                vb[yy] = lane < HX - 32 ? __ldg(src + xb) : 0.f;
                src += Xc;
            }
        } else {
#pragma unroll
            for (int yy = 0; yy < HY; yy++) {
                const float *src = bsrc + (size_t)pwrap(y0 - 2 + yy, Yc) * Xc;
                va[yy] = __ldg(src + xa);
                vb[yy] = lane < HX - 32 ? __ldg(src + xb) : 0.f;
            }
        }
#pragma unroll
        for (int yy = 0; yy < HY; yy++) {
            s_b[band * SBB + yy * SB + lane] = va[yy];
            if (lane < HX - 32) s_b[band * SBB + yy * SB + 32 + lane] = vb[yy];
        }
    }
    __syncthreads();

    // inverse along x: job (halo row id 0..79 = (z band, y band, row), chunk of
    // 4 output pairs); pair n of the tile needs low n and highs n-2 .. n+2
    for (int job = tid; job < 4 * HY * 8; job += 256) {
        const int rid = job % (4 * HY), chunk = job / (4 * HY);
        const int zy = rid / HY, rw = rid - zy * HY;
        const float *lo = &s_b[2 * zy * SBB + rw * SB + 4 * chunk + 2];
        const float *hi = &s_b[(2 * zy + 1) * SBB + rw * SB + 4 * chunk];
        float h[8];
#pragma unroll
        for (int i = 0; i < 8; i++) h[i] = hi[i];
        float *dst_x = &s_x[zy >> 1][zy & 1][rw][8 * chunk];
#pragma unroll
        for (int p = 0; p < 4; p++) {
            const float a0 = lo[p] - lift_u(h[p], h[p + 1], h[p + 3], h[p + 4]);
            dst_x[2 * p] = (a0 + h[p + 2]) * kS;
            dst_x[2 * p + 1] = (a0 - h[p + 2]) * kS;
        }
    }
    __syncthreads();

    // inverse along y: thread (z band, half of the 16 pairs, output column)
    float(*s_o)[2 * TY][SO] = reinterpret_cast<float(*)[2 * TY][SO]>(&s_b[0]); // [z band][row][col]
    {
        const int zb = tid >> 7, half = (tid >> 6) & 1, col = tid & 63;
        float h[12];
#pragma unroll
        for (int i = 0; i < 12; i++) h[i] = s_x[zb][1][8 * half + i][col];
#pragma unroll
        for (int p = 0; p < 8; p++) {
            const float a0 = s_x[zb][0][8 * half + 2 + p][col] - lift_u(h[p], h[p + 1], h[p + 3], h[p + 4]);
            s_o[zb][16 * half + 2 * p][col] = (a0 + h[p + 2]) * kS;
            s_o[zb][16 * half + 2 * p + 1][col] = (a0 - h[p + 2]) * kS;
        }
    }
    __syncthreads();

    // inverse along z, store: each thread owns one output column (x index
    // math once) and every fourth output row
    const int Yo = 2 * Yc, Xo = 2 * Xc, Zo = 2 * Zc;
    const int col = tid & 63, xo = 2 * x0 + col;
    if (xo >= Xo) return;
    int bx = 0, z0 = 0, z1 = 0;
    long long gx = 0;
    if (SCATTER) {
        const int x = pwrap(xo - shift, Xo);
        gx = x >> LN;
        bx = x & ((1 << LN) - 1);
        z0 = pwrap(2 * m - shift, Zo);
        z1 = pwrap(2 * m + 1 - shift, Zo);
    }
    if (SCATTER) {
        // this thread's 8 output rows: every destination and, when averaging
        // spins, every previous value first (16 loads in flight), then the stores
        constexpr int NRO = 2 * TY / 4;
        constexpr int PER = (1 << LN) / 4; // rows i and i + PER of a thread lie one block row of groups apart
        float *p0[NRO], *p1[NRO];
        float o0[NRO], o1[NRO];
        // the level-1 output is group-major ([group][block][row][col], strides
        // N^2 and N: compile-time shifts)
        auto rowp = [&](int ys) {
            const int y = pwrap(ys - shift, Yo);
            const long long g = (long long)(y >> LN) * Bx + gx;
            return out.base + (g * Zo << (2 * LN)) + ((y & ((1 << LN) - 1)) << LN) + bx;
        };
        const long long dz = (long long)(z1 - z0) * (1 << (2 * LN));
        if (2 * y0 - shift >= 0 && 2 * y0 + 2 * TY - 1 < Yo) {
            // no row of the tile wraps: the first PER rows in full, the others
            // one group row (Bx Zo N^2 floats) further per PER rows
            const long long gstride = ((long long)Bx * Zo) << (2 * LN);
#pragma unroll
            for (int i = 0; i < NRO; i++) {
                p0[i] = i < PER ? rowp(2 * y0 + (tid >> 6) + 4 * i) + ((long long)z0 << (2 * LN))
                                : p0[i - PER] + gstride;
                p1[i] = p0[i] + dz;
                o0[i] = o1[i] = 0.f;
            }
        } else {
#pragma unroll
            for (int i = 0; i < NRO; i++) {
                const int orow = (tid >> 6) + 4 * i, ys = 2 * y0 + orow;
                p0[i] = p1[i] = nullptr;
                if (ys < Yo) {
                    p0[i] = rowp(ys) + ((long long)z0 << (2 * LN));
                    p1[i] = p0[i] + dz;
                }
                o0[i] = o1[i] = 0.f;
            }
        }
        if (accumulate) {
#pragma unroll
            for (int i = 0; i < NRO; i++)
                if (p0[i]) {
                    o0[i] = *p0[i];
                    o1[i] = *p1[i];
                }
        }
#pragma unroll
        for (int i = 0; i < NRO; i++)
            if (p0[i]) {
                const int orow = (tid >> 6) + 4 * i;
                const float L = s_o[0][orow][col], Hh = s_o[1][orow][col];
                *p0[i] = o0[i] + scale * ((L + Hh) * kS);
                *p1[i] = o1[i] + scale * ((L - Hh) * kS);
            }
    } else {
        for (int orow = tid >> 6; orow < 2 * TY; orow += 4) {
            const int ys = 2 * y0 + orow;
            if (ys >= Yo) break;
            const float L = s_o[0][orow][col], Hh = s_o[1][orow][col];
            dst[((size_t)(2 * m) * Yo + ys) * Xo + xo] = (L + Hh) * kS;
            dst[((size_t)(2 * m + 1) * Yo + ys) * Xo + xo] = (L - Hh) * kS;
        }
    }
}

// Stage-1 weights: w = 1 / max(TV(u), eps) with TV the sum of absolute
// forward differences along rows, columns and the group axis inside the
// N x N x K block (no wrap).  One warp per group reads the group-major block
// gm[g][r][a][b] (contiguous, float4), stages it in shared memory, sums the
// differences and writes w; with permute it also copies each block row to
// out.row(g*K + r, a) and w to each of the group's slots.  Warps per CTA:
// as many as keep the staged blocks within 32 KB of shared memory (<= 4).
template <int K, int NB>
__host__ __device__ constexpr int tv_warps()
{
    return 8192 / (K * NB * NB) >= 4 ? 4 : (8192 / (K * NB * NB) >= 1 ? 8192 / (K * NB * NB) : 1);
}

template <int K, int NB>
__global__ void __launch_bounds__(tv_warps<K, NB>() * 32)
k_tv(const float *__restrict__ gm, int G, float eps, GroupOut out, int permute)
{
    constexpr int NW = tv_warps<K, NB>(), E = K * NB * NB; // floats per group
    constexpr int NV = E / 4 / 32;                         // float4 per lane
    constexpr int NL = NB == 8 ? 3 : 4;                    // log2 NB
    __shared__ __align__(16) float su[NW][E];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * NW + warp;
    if (g >= G) return;
    float *u = su[warp];
    const float4 *src = reinterpret_cast<const float4 *>(gm + (size_t)g * E);
    constexpr int CH = NV < 8 ? NV : 8; // float4 loads in flight per lane
#pragma unroll 1
    for (int i0 = 0; i0 < NV; i0 += CH) {
        float4 v[CH];
#pragma unroll
        for (int i = 0; i < CH; i++) v[i] = __ldg(src + lane + 32 * (i0 + i));
#pragma unroll
        for (int i = 0; i < CH; i++) reinterpret_cast<float4 *>(u)[lane + 32 * (i0 + i)] = v[i];
    }
    __syncwarp();
    float tv = 0.f;
#pragma unroll 4
    for (int e = lane; e < E; e += 32) {
        const int r = e >> (2 * NL), a = (e >> NL) & (NB - 1), b = e & (NB - 1);
        const float c = u[e];
        if (a < NB - 1) tv += fabsf(u[e + NB] - c);
        if (b < NB - 1) tv += fabsf(u[e + 1] - c);
        if (r < K - 1) tv += fabsf(u[e + NB * NB] - c);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tv += __shfl_xor_sync(0xffffffffu, tv, o);
    const float wv = 1.f / fmaxf(tv, eps);
    if (!permute) {
        if (lane == 0) out.w[g] = wv;
        return;
    }
    // NB / 4 lanes per block row q = NB r + a, one float4 each: every row
    // (32 or 64 bytes, whole sectors) is written by one instruction
    constexpr int LPR = NB / 4, RPI = 32 / LPR; // lanes per row, rows per instruction
    const int h = lane % LPR;
#pragma unroll 8
    for (int i = 0; i < K * NB / RPI; i++) {
        const int q = lane / LPR + RPI * i;
        const float4 *s = reinterpret_cast<const float4 *>(u + q * NB);
        reinterpret_cast<float4 *>(out.row((long long)g * K + (q >> NL), q & (NB - 1)))[h] = s[h];
    }
    if (lane < K) out.w[out.slot((long long)g * K + lane)] = wv;
}

// The same weights for 8 x 8 blocks without shared memory.  Lane l of a
// group's warp holds the half row (bc = l & 1, row a = (l >> 1) & 7) of the
// blocks r = (l >> 4) K/2 .. (l >> 4) K/2 + K/2 - 1 as float4 registers (one
// coalesced 512-byte load per step: two whole block slices).  Differences
// along the group axis are taken in registers (one shuffle from lane l + 16
// where the two halves meet), along the row inside the float4 and, across
// its two halves, by one shuffle from lane l + 1, and between rows by
// shuffles from lane l + 2.  Each lane sums its terms; the warp adds the
// lanes.  With permute the rows go to the planar layout straight from the
// registers (32-byte rows, whole sectors).
template <int K>
__global__ void __launch_bounds__(128)
k_tv8(const float *__restrict__ gm, int G, float eps, GroupOut out, int permute)
{
    constexpr int NR = K / 2; // blocks a lane holds
    constexpr unsigned kFull = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * 4 + warp;
    if (g >= G) return;
    const int bc = lane & 1, a = (lane >> 1) & 7, rg = lane >> 4;
    const float4 *src = reinterpret_cast<const float4 *>(gm + (size_t)g * K * 64) + (rg * NR) * 16 + a * 2 + bc;
    float4 v[NR];
#pragma unroll
    for (int j = 0; j < NR; j++) v[j] = __ldg(src + 16 * j);
    float tv = 0.f;
#pragma unroll
    for (int j = 0; j < NR; j++) {
        // along the row: inside the half row, then to the next half
        tv += fabsf(v[j].y - v[j].x) + fabsf(v[j].z - v[j].y) + fabsf(v[j].w - v[j].z);
        const float nx = __shfl_down_sync(kFull, v[j].x, 1);
        if (bc == 0) tv += fabsf(nx - v[j].w);
        // to the next row of the block (lane l + 2: same half, row a + 1)
        const float4 d = make_float4(__shfl_down_sync(kFull, v[j].x, 2), __shfl_down_sync(kFull, v[j].y, 2),
                                     __shfl_down_sync(kFull, v[j].z, 2), __shfl_down_sync(kFull, v[j].w, 2));
        if (a < 7) tv += fabsf(d.x - v[j].x) + fabsf(d.y - v[j].y) + fabsf(d.z - v[j].z) + fabsf(d.w - v[j].w);
        // to the next block of the group
        if (j + 1 < NR)
            tv += fabsf(v[j + 1].x - v[j].x) + fabsf(v[j + 1].y - v[j].y) + fabsf(v[j + 1].z - v[j].z) +
                  fabsf(v[j + 1].w - v[j].w);
    }
    { // block K/2 - 1 (first half, lanes 0..15) to block K/2 (lane l + 16's first)
        const float4 n = make_float4(__shfl_down_sync(kFull, v[0].x, 16), __shfl_down_sync(kFull, v[0].y, 16),
                                     __shfl_down_sync(kFull, v[0].z, 16), __shfl_down_sync(kFull, v[0].w, 16));
        const float4 &c = v[NR - 1];
        if (rg == 0) tv += fabsf(n.x - c.x) + fabsf(n.y - c.y) + fabsf(n.z - c.z) + fabsf(n.w - c.w);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tv += __shfl_xor_sync(kFull, tv, o);
    const float wv = 1.f / fmaxf(tv, eps);
    if (!permute) {
        if (lane == 0) out.w[g] = wv;
        return;
    }
#pragma unroll
    for (int j = 0; j < NR; j++)
        reinterpret_cast<float4 *>(out.row((long long)g * K + rg * NR + j, a))[bc] = v[j];
    if (lane < K) out.w[out.slot((long long)g * K + lane)] = wv;
}

template <int K, int NB>
void launch_tv(const float *gm, int G, float eps, const GroupOut &out, int permute, cudaStream_t st)
{
    if constexpr (NB == 8) {
        k_tv8<K><<<(G + 3) / 4, 128, 0, st>>>(gm, G, eps, out, permute);
    } else {
        constexpr int NW = tv_warps<K, NB>();
        k_tv<K, NB><<<(G + NW - 1) / NW, NW * 32, 0, st>>>(gm, G, eps, out, permute);
    }
}

template <int LN>
void launch_levels(const HtGeom &g, const float *img, int pitch, const int *ofs, float *const C[4], float sigma,
                   float tau_a, float tau_b, int cycle_spins, const GroupOut &gm_out, cudaStream_t st)
{
    const float inv_c = 1.f / (float)cycle_spins;
    for (int c = 0; c < cycle_spins; c++) {
        for (int l = 1; l <= g.levels; l++) { // analysis
            const int Y = g.Yd >> (l - 1), X = g.Xd >> (l - 1), Z = g.K >> (l - 1);
            const float tau = sigma * (tau_a - tau_b * (float)l);
            const int vec = ((X >> 1) % 4) == 0;
            dim3 grid((X / 2 + ATX - 1) / ATX, (Y / 2 + ATY - 1) / ATY, Z / 2);
            if (l == 1) {
                auto kern = c == 0 ? k_dwt_ana<true, LN, 0>
                                   : c == 1 ? k_dwt_ana<true, LN, 1> : c == 2 ? k_dwt_ana<true, LN, 2> : k_dwt_ana<true, LN, 3>;
                kern<<<grid, kAnaThreads, 0, st>>>(nullptr, img, pitch, ofs, g.Bx, c, Y, X, Z, C[1], tau, vec);
            }
            else
                k_dwt_ana<false, 3><<<grid, kAnaThreads, 0, st>>>(C[l - 1], nullptr, 0, nullptr, 0, 0, Y, X, Z, C[l], tau,
                                                          vec);
        }
        // synthesis, levels L..1; level l writes the approximation of level
        // l-1, i.e. band 0 of C[l-1] (or the blocks for l = 1)
        for (int l = g.levels; l >= 1; l--) {
            const int Yc = g.Yd >> l, Xc = g.Xd >> l, Zc = g.K >> l;
            dim3 grid((Xc + TX - 1) / TX, (Yc + TY - 1) / TY, Zc);
            if (l == 1)
                k_dwt_syn<true, LN><<<grid, 256, 0, st>>>(C[1], Yc, Xc, Zc, nullptr, gm_out, g.Bx, c, inv_c, c > 0);
            else
                k_dwt_syn<false, 3><<<grid, 256, 0, st>>>(C[l], Yc, Xc, Zc, C[l - 1], gm_out, 0, 0, 0.f, 0);
        }
    }
}

} // namespace

HtGeom ht_geom(int By, int Bx, int K, int levels, int N)
{
    HtGeom g{};
    g.N = N;
    g.By = By;
    g.Bx = Bx;
    g.K = K;
    g.Yd = By * N;
    g.Xd = Bx * N;
    g.levels = levels;
    size_t off = 0;
    for (int l = 1; l <= levels; l++) {
        // level-l coefficients: 8 bands of (K, Yd, Xd) >> l each
        g.level_elems[l] = ((size_t)g.Yd * g.Xd * K) >> (3 * (l - 1));
        g.level_off[l] = off;
        off += align_up(g.level_elems[l] * sizeof(float));
    }
    g.ofs_off = off;
    off += align_up((size_t)By * Bx * K * sizeof(int));
    g.gm_off = off;
    off += align_up((size_t)By * Bx * K * N * N * sizeof(float));
    g.bytes = off;
    return g;
}

cudaError_t launch_ht_transforms(const float *img, int H, int W, int pitch, const int32_t *idx, const HtGeom &g,
                                 float sigma, float tau_a, float tau_b, int cycle_spins, const GroupOut &out,
                                 void *ht_ws, cudaStream_t st)
{
    if (g.N != 8 && g.N != 16) return cudaErrorInvalidValue;
    char *base = (char *)ht_ws;
    int *ofs = (int *)(base + g.ofs_off);
    const int nent = g.By * g.Bx * g.K;
    k_offsets<<<(nent + 255) / 256, 256, 0, st>>>(idx, nent, H, W, g.N, pitch, ofs);
    float *C[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int l = 1; l <= g.levels; l++) C[l] = (float *)(base + g.level_off[l]);
    // the level-1 synthesis writes group-major: the output itself, or a
    // scratch that the TV pass permutes into the output's layout
    const bool permute = out.slot_of != nullptr;
    float *gm = permute ? (float *)(base + g.gm_off) : out.base;
    const GroupOut gm_out = group_major(gm, nullptr, g.N); // the layout k_dwt_syn<true> assumes
    if (g.N == 8)
        launch_levels<3>(g, img, pitch, ofs, C, sigma, tau_a, tau_b, cycle_spins, gm_out, st);
    else
        launch_levels<4>(g, img, pitch, ofs, C, sigma, tau_a, tau_b, cycle_spins, gm_out, st);
    return cudaGetLastError();
}

cudaError_t launch_ht_weights(const HtGeom &g, float eps_w, const GroupOut &out, void *ht_ws, cudaStream_t st)
{
    char *base = (char *)ht_ws;
    const bool permute = out.slot_of != nullptr;
    float *gm = permute ? (float *)(base + g.gm_off) : out.base;
    const int G = g.By * g.Bx;
    if (g.N == 8) {
        switch (g.K) {
        case 8: launch_tv<8, 8>(gm, G, eps_w, out, permute, st); break;
        case 16: launch_tv<16, 8>(gm, G, eps_w, out, permute, st); break;
        default: launch_tv<32, 8>(gm, G, eps_w, out, permute, st); break;
        }
    } else {
        switch (g.K) {
        case 8: launch_tv<8, 16>(gm, G, eps_w, out, permute, st); break;
        case 16: launch_tv<16, 16>(gm, G, eps_w, out, permute, st); break;
        default: launch_tv<32, 16>(gm, G, eps_w, out, permute, st); break;
        }
    }
    return cudaGetLastError();
}

} // namespace gbm3d

namespace gbm3d {

cudaError_t launch_filter_ht(const float *img, int H, int W, int pitch, const int32_t *idx, const HtGeom &g,
                             float sigma, float tau_a, float tau_b, int cycle_spins, float eps_w, const GroupOut &out,
                             void *ht_ws, cudaStream_t st)
{
    cudaError_t e = launch_ht_transforms(img, H, W, pitch, idx, g, sigma, tau_a, tau_b, cycle_spins, out, ht_ws, st);
    return e == cudaSuccess ? launch_ht_weights(g, eps_w, out, ht_ws, st) : e;
}

} // namespace gbm3d
