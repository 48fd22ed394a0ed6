// ht.cu -- stage-1 global volume hard thresholding (Sec. 3.1 eq. BM3DHT,
// cycle spinning U_h = S_{-h} T^-1 Upsilon T S_h V, TV weights w = 1/TV).
//
// The volume of matched blocks is never materialised: the level-1 analysis
// gathers each voxel V[pN+a, qN+b, r] = Z[k_r+a, l_r+b] straight from the
// image through the match list (the image and list stay in L2), with the
// cycle-spin shift folded into the index arithmetic.  Each level of the
// periodic 3-D transform (bior1.5 x bior1.5 x Haar, Mallat) is one kernel
// over tiles of 16 x 32 output positions and one pair of slices along the
// group axis; rows and columns use the lifting form of bior1.5
//   d[n]  = (x[2n] - x[2n+1]) / sqrt2,  a0[n] = (x[2n] + x[2n+1]) / sqrt2,
//   a[n]  = a0[n] + (3 d[n-2] - 22 d[n-1] + 22 d[n+1] - 3 d[n+2]) / 128,
// and its exact inverse.  Detail bands are hard-thresholded as they are
// written.  The level-1 synthesis writes the filtered blocks straight into
// the group-major output (undoing the spin shift), averaging the spins.
#include "internal.cuh"

namespace gbm3d {
namespace {

constexpr float kS = 0.70710678118654752f; // 1/sqrt(2)
constexpr float kU1 = 0.171875f;           // 22/128
constexpr float kU2 = 0.0234375f;          // 3/128
constexpr int TY = 16, TX = 32;            // output positions per tile
constexpr int IY = 2 * TY + 8, IX = 2 * TX + 8; // analysis input tile (halo 4 / 4 after the pair)
constexpr int HY = TY + 4, HX = TX + 4;    // synthesis band tile (halo 2 each side)

// Periodic index (eq. (1)).  Tile halos reach at most a few samples past
// either end, so one conditional add or subtract suffices unless the axis is
// shorter than the halo (coarse levels of tiny images): then the true modulo.
__device__ __forceinline__ int pwrap(int i, int n)
{
    if (i < 0) i += n;
    if (i >= n) i -= n;
    if ((unsigned)i >= (unsigned)n) {
        i %= n;
        if (i < 0) i += n;
    }
    return i;
}

// Pixel offset k*pitch + l of every match-list entry (once per call, so the
// gathers need no division).
__global__ void k_offsets(const int32_t *__restrict__ idx, int n, int H, int W, int pitch, int *__restrict__ ofs)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    int k, l;
    block_kl(idx[e], H, W, k, l);
    ofs[e] = k * pitch + l;
}

// Lifting update U(d)[n] from the five detail values d[n-2..n+2].
__device__ __forceinline__ float lift_u(float dm2, float dm1, float dp1, float dp2)
{
    return kU2 * (dm2 - dp2) + kU1 * (dp1 - dm1);
}

// One analysis step on ten consecutive samples v[0..9] = x[2n-4 .. 2n+5]:
// returns the low-pass a[n] and the high-pass d[n].
__device__ __forceinline__ void ana10(const float *v, int stride, float &lo, float &hi)
{
    float d[5];
#pragma unroll
    for (int m = 0; m < 5; m++) d[m] = (v[(2 * m) * stride] - v[(2 * m + 1) * stride]) * kS;
    const float a0 = (v[4 * stride] + v[5 * stride]) * kS;
    lo = a0 + lift_u(d[0], d[1], d[3], d[4]);
    hi = d[2];
}

// Level analysis: input (Z, Y, X) -> 8 bands [band][Z/2][Y/2][X/2], band =
// 4 hz + 2 hy + hx.  GATHER: the input is the cycle-spun mosaic read from the
// image through idx (level 1); otherwise a [Z][Y][X] plane stack.
template <bool GATHER>
__global__ void __launch_bounds__(256)
k_dwt_ana(const float *__restrict__ src, const float *__restrict__ img, int pitch, const int *__restrict__ ofs,
          int Bx, int shift, int Y, int X, int Z, float *__restrict__ dst, float tau)
{
    __shared__ float s_in[2][IY][IX];
    __shared__ float s_y[2][2][TY][IX]; // [z band][y band][row][col]
    const int m = blockIdx.z;            // slice pair
    const int y0 = blockIdx.y * TY, x0 = blockIdx.x * TX;
    const int iy0 = 2 * y0 - 4, ix0 = 2 * x0 - 4;
    for (int e = threadIdx.x; e < 2 * IY * IX; e += blockDim.x) {
        const int zz = e / (IY * IX), rem = e - zz * (IY * IX);
        const int yy = rem / IX, xx = rem - yy * IX;
        float v;
        if (GATHER) {
            const int z = pwrap(2 * m + zz - shift, Z);
            const int y = pwrap(iy0 + yy - shift, Y), x = pwrap(ix0 + xx - shift, X);
            const int g = (y >> 3) * Bx + (x >> 3);
            const int o = __ldg(ofs + (size_t)g * Z + z);
            v = __ldg(img + o + (size_t)(y & 7) * pitch + (x & 7));
        } else {
            const int y = pwrap(iy0 + yy, Y), x = pwrap(ix0 + xx, X);
            v = __ldg(src + ((size_t)(2 * m + zz) * Y + y) * X + x);
        }
        s_in[zz][yy][xx] = v;
    }
    __syncthreads();
    // Haar along z (slice pair) in place: [0] = low, [1] = high.
    for (int e = threadIdx.x; e < IY * IX; e += blockDim.x) {
        const int yy = e / IX, xx = e - yy * IX;
        const float a = s_in[0][yy][xx], b = s_in[1][yy][xx];
        s_in[0][yy][xx] = (a + b) * kS;
        s_in[1][yy][xx] = (a - b) * kS;
    }
    __syncthreads();
    // bior1.5 along y: output row o uses input rows 2o .. 2o+9 of the tile.
    for (int e = threadIdx.x; e < 2 * TY * IX; e += blockDim.x) {
        const int zb = e / (TY * IX), rem = e - zb * (TY * IX);
        const int o = rem / IX, xx = rem - o * IX;
        float lo, hi;
        ana10(&s_in[zb][2 * o][xx], IX, lo, hi);
        s_y[zb][0][o][xx] = lo;
        s_y[zb][1][o][xx] = hi;
    }
    __syncthreads();
    // bior1.5 along x, threshold, store.
    const int Zo = Z >> 1, Yo = Y >> 1, Xo = X >> 1;
    const size_t band_elems = (size_t)Zo * Yo * Xo;
    for (int e = threadIdx.x; e < 4 * TY * TX; e += blockDim.x) {
        const int zy = e / (TY * TX), rem = e - zy * (TY * TX);
        const int o = rem / TX, ox = rem - o * TX;
        const int zb = zy >> 1, yb = zy & 1;
        const int yo = y0 + o, xo = x0 + ox;
        if (yo >= Yo || xo >= Xo) continue;
        float lo, hi;
        ana10(&s_y[zb][yb][o][2 * ox], 1, lo, hi);
        const int band = zb * 4 + yb * 2;
        const size_t off = ((size_t)m * Yo + yo) * Xo + xo;
        dst[(size_t)band * band_elems + off] = (band == 0 || fabsf(lo) >= tau) ? lo : 0.f;
        dst[(size_t)(band + 1) * band_elems + off] = (fabsf(hi) >= tau) ? hi : 0.f;
    }
}

// Inverse lifting for one output pair from the low value at n and the five
// high values h[n-2..n+2]; writes x[2n], x[2n+1].
__device__ __forceinline__ void syn_pair(float lo, const float *h, int stride, float &x0, float &x1)
{
    const float hm2 = h[0], hm1 = h[stride], hc = h[2 * stride], hp1 = h[3 * stride], hp2 = h[4 * stride];
    const float a0 = lo - lift_u(hm2, hm1, hp1, hp2);
    x0 = (a0 + hc) * kS;
    x1 = (a0 - hc) * kS;
}

// Level synthesis: 8 bands [band][Zc][Yc][Xc] -> (2Zc, 2Yc, 2Xc).  SCATTER
// (level 1): the voxel at spun position (z,y,x) belongs to mosaic position
// (z,y,x) - shift, i.e. block r = z of group (y/8, x/8) at (y%8, x%8); it is
// written (or added) scaled into the output blocks.
template <bool SCATTER>
__global__ void __launch_bounds__(256)
k_dwt_syn(const float *__restrict__ coef, int Yc, int Xc, int Zc, float *__restrict__ dst, GroupOut out, int Bx,
          int shift, float scale, int accumulate)
{
    __shared__ float s_b[8][HY][HX];
    __shared__ float s_x[2][2][HY][2 * TX]; // [z band][y band][coef row][output col]
    const int m = blockIdx.z;
    const int y0 = blockIdx.y * TY, x0 = blockIdx.x * TX;
    const size_t band_elems = (size_t)Zc * Yc * Xc;
    for (int e = threadIdx.x; e < 8 * HY * HX; e += blockDim.x) {
        const int band = e / (HY * HX), rem = e - band * (HY * HX);
        const int yy = rem / HX, xx = rem - yy * HX;
        const int y = pwrap(y0 - 2 + yy, Yc), x = pwrap(x0 - 2 + xx, Xc);
        s_b[band][yy][xx] = __ldg(coef + (size_t)band * band_elems + ((size_t)m * Yc + y) * Xc + x);
    }
    __syncthreads();
    // inverse along x for every (z band, y band) and coefficient row
    for (int e = threadIdx.x; e < 4 * HY * TX; e += blockDim.x) {
        const int zy = e / (HY * TX), rem = e - zy * (HY * TX);
        const int row = rem / TX, o = rem - row * TX;
        const int lo_band = zy * 2; // (hz, hy, hx = 0); high band is lo_band + 1
        float v0, v1;
        syn_pair(s_b[lo_band][row][o + 2], &s_b[lo_band + 1][row][o], 1, v0, v1);
        s_x[zy >> 1][zy & 1][row][2 * o] = v0;
        s_x[zy >> 1][zy & 1][row][2 * o + 1] = v1;
    }
    __syncthreads();
    // inverse along y, then Haar along z; store
    const int Yo = 2 * Yc, Xo = 2 * Xc, Zo = 2 * Zc;
    for (int e = threadIdx.x; e < TY * 2 * TX; e += blockDim.x) {
        const int o = e / (2 * TX), col = e - o * (2 * TX);
        float a0, a1, b0, b1;
        syn_pair(s_x[0][0][o + 2][col], &s_x[0][1][o][col], 2 * TX, a0, a1);
        syn_pair(s_x[1][0][o + 2][col], &s_x[1][1][o][col], 2 * TX, b0, b1);
        const float vz[2][2] = {{(a0 + b0) * kS, (a1 + b1) * kS}, {(a0 - b0) * kS, (a1 - b1) * kS}};
        const int yb = 2 * (y0 + o), xo = 2 * x0 + col;
        if (xo >= Xo || yb >= Yo) continue;
#pragma unroll
        for (int zz = 0; zz < 2; zz++)
#pragma unroll
            for (int yy = 0; yy < 2; yy++) {
                const int zs = 2 * m + zz, ys = yb + yy;
                const float v = vz[zz][yy];
                if (SCATTER) {
                    const int z = pwrap(zs - shift, Zo), y = pwrap(ys - shift, Yo), x = pwrap(xo - shift, Xo);
                    const long long g = (long long)(y >> 3) * Bx + (x >> 3);
                    float *o_ = out.row(g * Zo + z, y & 7) + (x & 7);
                    *o_ = accumulate ? (*o_ + scale * v) : scale * v;
                } else {
                    dst[((size_t)zs * Yo + ys) * Xo + xo] = v;
                }
            }
    }
}

// Stage-1 weights: w = 1 / max(TV(u), eps) with TV the sum of absolute
// forward differences along rows, columns and the group axis inside the
// N x N x K block (no wrap).  One warp per group; lane = 4 a + bh owns the
// two columns 2bh, 2bh+1 of row a of every block.
__global__ void k_tv(GroupOut out, int G, int K, float eps)
{
    const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= G) return;
    const int a = lane >> 2, bh = lane & 3;
    float tv = 0.f;
    for (int r = 0; r < K; r++) {
        const long long e = (long long)g * K + r;
        const float *row = out.row(e, a);
        const float v0 = row[2 * bh], v1 = row[2 * bh + 1];
        tv += fabsf(v1 - v0);
        if (bh < 3) tv += fabsf(row[2 * bh + 2] - v1);
        if (a < 7) {
            const float *nxt = out.row(e, a + 1);
            tv += fabsf(nxt[2 * bh] - v0) + fabsf(nxt[2 * bh + 1] - v1);
        }
        if (r < K - 1) {
            const float *nz = out.row(e + 1, a);
            tv += fabsf(nz[2 * bh] - v0) + fabsf(nz[2 * bh + 1] - v1);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tv += __shfl_xor_sync(0xffffffffu, tv, o);
    const float wv = 1.f / fmaxf(tv, eps);
    if (out.per_slot) {
        for (int r = lane; r < K; r += 32) out.w[out.slot((long long)g * K + r)] = wv;
    } else if (lane == 0) {
        out.w[g] = wv;
    }
}

} // namespace

HtGeom ht_geom(int By, int Bx, int K, int levels)
{
    HtGeom g{};
    g.By = By;
    g.Bx = Bx;
    g.K = K;
    g.Yd = By * kPatch;
    g.Xd = Bx * kPatch;
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
    g.bytes = off;
    return g;
}

cudaError_t launch_filter_ht(const float *img, int H, int W, int pitch, const int32_t *idx, const HtGeom &g,
                             float sigma, float tau_a, float tau_b, int cycle_spins, float eps_w, const GroupOut &out,
                             void *ht_ws, cudaStream_t st)
{
    char *base = (char *)ht_ws;
    int *ofs = (int *)(base + g.ofs_off);
    const int nent = g.By * g.Bx * g.K;
    k_offsets<<<(nent + 255) / 256, 256, 0, st>>>(idx, nent, H, W, pitch, ofs);
    float *C[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int l = 1; l <= g.levels; l++) C[l] = (float *)(base + g.level_off[l]);
    const float inv_c = 1.f / (float)cycle_spins;
    for (int c = 0; c < cycle_spins; c++) {
        // analysis, levels 1..L
        for (int l = 1; l <= g.levels; l++) {
            const int Y = g.Yd >> (l - 1), X = g.Xd >> (l - 1), Z = g.K >> (l - 1);
            const float tau = sigma * (tau_a - tau_b * (float)l);
            dim3 grid((X / 2 + TX - 1) / TX, (Y / 2 + TY - 1) / TY, Z / 2);
            if (l == 1)
                k_dwt_ana<true><<<grid, 256, 0, st>>>(nullptr, img, pitch, ofs, g.Bx, c, Y, X, Z, C[1], tau);
            else
                k_dwt_ana<false><<<grid, 256, 0, st>>>(C[l - 1], nullptr, 0, nullptr, 0, 0, Y, X, Z, C[l], tau);
        }
        // synthesis, levels L..1; level l writes the approximation of level
        // l-1, i.e. band 0 of C[l-1] (or the groups for l = 1)
        for (int l = g.levels; l >= 1; l--) {
            const int Yc = g.Yd >> l, Xc = g.Xd >> l, Zc = g.K >> l;
            dim3 grid((Xc + TX - 1) / TX, (Yc + TY - 1) / TY, Zc);
            if (l == 1)
                k_dwt_syn<true><<<grid, 256, 0, st>>>(C[1], Yc, Xc, Zc, nullptr, out, g.Bx, c, inv_c, c > 0);
            else
                k_dwt_syn<false><<<grid, 256, 0, st>>>(C[l], Yc, Xc, Zc, C[l - 1], out, 0, 0, 0.f, 0);
        }
    }
    const int G = g.By * g.Bx;
    k_tv<<<(G + 7) / 8, 256, 0, st>>>(out, G, g.K, eps_w);
    return cudaGetLastError();
}

} // namespace gbm3d
