// wiener.cu -- stage-2 empirical Wiener filtering of every group (Sec. 4:
// 2-D DCT on the blocks, 1-D Haar along the group, Wiener shrinkage against
// the pilot, inverse, group weight).
//
// One CTA per group, K*8 threads.  Thread (r, c) reads column c of block r of
// both groups (noisy and pilot) straight from the images -- 8 lanes cover one
// 32-byte block row per load -- and runs the column DCT in registers (even/odd
// butterfly of the orthonormal DCT-II; the noisy and pilot columns as packed
// f32x2 pairs, and likewise the row DCTs); the row DCTs go through a
// bank-conflict-free shared layout, one thread per coefficient position runs
// the full-depth Haar along the K blocks in registers, and the inverse ends
// with the column pass writing the filtered group straight out, again 8 lanes
// per block row.
#include "internal.cuh"

namespace gbm3d {
namespace {

constexpr float kS = 0.70710678118654752f;
constexpr float kR8 = 0.35355339059327376f; // 1/sqrt(8)
// cos(k pi / 16)
constexpr float c1 = 0.98078528040323043f, c2 = 0.92387953251128674f, c3 = 0.83146961230254524f;
constexpr float c5 = 0.55557023301960218f, c6 = 0.38268343236508977f, c7 = 0.19509032201612825f;

// Orthonormal 8-point DCT-II, even/odd split (dct8x2 below), and its inverse.
// Two transforms at once: the noisy and the pilot values of one column (or
// row) travel as packed pairs, one f32x2 operation per step of dct8.
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk2(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void upk2(f2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f2 mul2(f2 a, float c)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(pk2(c, c)));
    return r;
}

__device__ __forceinline__ f2 fma2(f2 a, float c, f2 b) // a c + b
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(pk2(c, c)), "l"(b));
    return r;
}

__device__ __forceinline__ void dct8x2(f2 *x)
{
    const f2 s0 = add2(x[0], x[7]), s1 = add2(x[1], x[6]), s2 = add2(x[2], x[5]), s3 = add2(x[3], x[4]);
    const f2 d0 = sub2(x[0], x[7]), d1 = sub2(x[1], x[6]), d2 = sub2(x[2], x[5]), d3 = sub2(x[3], x[4]);
    const f2 e0 = add2(s0, s3), e1 = add2(s1, s2), f0 = sub2(s0, s3), f1 = sub2(s1, s2);
    x[0] = mul2(add2(e0, e1), kR8);
    x[4] = mul2(sub2(e0, e1), kR8);
    x[2] = mul2(fma2(f0, c2, mul2(f1, c6)), 0.5f);
    x[6] = mul2(fma2(f0, c6, mul2(f1, -c2)), 0.5f);
    x[1] = mul2(fma2(d0, c1, fma2(d1, c3, fma2(d2, c5, mul2(d3, c7)))), 0.5f);
    x[3] = mul2(fma2(d0, c3, fma2(d1, -c7, fma2(d2, -c1, mul2(d3, -c5)))), 0.5f);
    x[5] = mul2(fma2(d0, c5, fma2(d1, -c1, fma2(d2, c7, mul2(d3, c3)))), 0.5f);
    x[7] = mul2(fma2(d0, c7, fma2(d1, -c5, fma2(d2, c3, mul2(d3, -c1)))), 0.5f);
}

// Its inverse (DCT-III, the transpose).
__device__ __forceinline__ void idct8(float *X)
{
    const float p = (X[0] + X[4]) * kR8, m = (X[0] - X[4]) * kR8;
    const float u = 0.5f * (c2 * X[2] + c6 * X[6]), v = 0.5f * (c6 * X[2] - c2 * X[6]);
    const float e0 = p + u, e3 = p - u, e1 = m + v, e2 = m - v;
    const float o0 = 0.5f * (c1 * X[1] + c3 * X[3] + c5 * X[5] + c7 * X[7]);
    const float o1 = 0.5f * (c3 * X[1] - c7 * X[3] - c1 * X[5] - c5 * X[7]);
    const float o2 = 0.5f * (c5 * X[1] - c1 * X[3] + c7 * X[5] + c3 * X[7]);
    const float o3 = 0.5f * (c7 * X[1] - c5 * X[3] + c3 * X[5] - c1 * X[7]);
    X[0] = e0 + o0;
    X[7] = e0 - o0;
    X[1] = e1 + o1;
    X[6] = e1 - o1;
    X[2] = e2 + o2;
    X[5] = e2 - o2;
    X[3] = e3 + o3;
    X[4] = e3 - o3;
}

// Shared-memory address of coefficient (block r, row a, column b):
//   r*72 + (r/8)*8 + a*9 + b.
// Row pass (thread (r,a), 8 columns), column pass (thread (r,b), 8 rows) and
// group pass (thread (8 blocks of one quarter, position a*8+b), lanes = 4
// quarters x 8 columns) all hit 32 distinct banks.
__device__ __forceinline__ int sidx(int r, int a, int b) { return r * 72 + (r >> 3) * 8 + a * 9 + b; }

// Haar along the group, K = 2^L blocks, for one coefficient position: the
// position's K values are spread over Q = K/8 neighbouring lanes (lane bits
// 0..log2(Q)-1 = quarter q), 8 consecutive blocks each.  Levels 1..3 run in
// registers on each lane's 8 values (Mallat order: approximation in v[0]);
// levels 4..L combine the lanes' approximations by shuffles: at level 3+m
// lanes whose quarter index is a multiple of 2^(m-1) pair with q ^ 2^(m-1),
// the lower keeps the low-pass, the upper the high-pass.  These are exactly
// the pairings of the full-depth Mallat transform; every coefficient is held
// once, so the elementwise shrinkage needs no reordering.
template <int LEN>
__device__ __forceinline__ void haar_inv(float *h)
{
    if constexpr (LEN > 2) haar_inv<LEN / 2>(h);
    float t[LEN];
#pragma unroll
    for (int m = 0; m < LEN / 2; m++) {
        t[2 * m] = (h[m] + h[LEN / 2 + m]) * kS;
        t[2 * m + 1] = (h[m] - h[LEN / 2 + m]) * kS;
    }
#pragma unroll
    for (int m = 0; m < LEN; m++) h[m] = t[m];
}

// The forward transform on packed (pilot, noisy) pairs: one f32x2 operation
// for both groups, the pairings as described above.
template <int LEN>
__device__ __forceinline__ void haar_fwd2(f2 *h)
{
    f2 t[LEN];
#pragma unroll
    for (int m = 0; m < LEN / 2; m++) {
        t[m] = mul2(add2(h[2 * m], h[2 * m + 1]), kS);
        t[LEN / 2 + m] = mul2(sub2(h[2 * m], h[2 * m + 1]), kS);
    }
#pragma unroll
    for (int m = 0; m < LEN; m++) h[m] = t[m];
    if constexpr (LEN > 2) haar_fwd2<LEN / 2>(h);
}

template <int Q>
__device__ __forceinline__ void haar_fwd_lanes2(f2 *v, int q)
{
    haar_fwd2<8>(v);
#pragma unroll
    for (int st = 1; st < Q; st <<= 1) {
        const f2 o = __shfl_xor_sync(0xffffffffu, v[0], st);
        if ((q & (2 * st - 1)) == 0) v[0] = mul2(add2(v[0], o), kS);       // lower lane: low-pass
        else if ((q & (2 * st - 1)) == st) v[0] = mul2(sub2(o, v[0]), kS);  // upper lane: high-pass
    }
}

template <int Q>
__device__ __forceinline__ void haar_inv_lanes(float *v, int q)
{
#pragma unroll
    for (int st = Q >> 1; st >= 1; st >>= 1) {
        const float o = __shfl_xor_sync(0xffffffffu, v[0], st);
        if ((q & (2 * st - 1)) == 0) v[0] = (v[0] + o) * kS;       // low + high
        else if ((q & (2 * st - 1)) == st) v[0] = (o - v[0]) * kS;  // low - high
    }
    haar_inv<8>(v);
}

template <int K>
__global__ void __launch_bounds__(K * 8)
k_wiener(const float *__restrict__ noisy, int npitch, const float *__restrict__ pilot, int ppitch, int H, int W,
         const int32_t *__restrict__ idx, float sigma2, float eps_w, GroupOut out)
{
    constexpr int NT = K * 8, Q = K / 8, SZ = K * 72 + K;
    __shared__ float sp[SZ];
    __shared__ float sq[SZ];
    __shared__ float red[NT / 32];
    __shared__ long long s_zoff[K], s_poff[K]; // block r's top-left in the noisy and the pilot image
    __shared__ long long s_slot[K];      // block r's slot in the output
    const int g = blockIdx.x, t = threadIdx.x;
    const int r = t >> 3, a = t & 7; // row and column passes: (block r, row/column a)
    if (t < K) {
        int k, l;
        block_kl(__ldg(idx + (size_t)g * K + t), H, W, kPatch, k, l);
        s_zoff[t] = (long long)k * npitch + l;
        s_poff[t] = (long long)k * ppitch + l;
        s_slot[t] = out.slot((long long)g * K + t);
    }
    __syncthreads();
    const int cb = a; // in the column phases thread (r, a) owns column a of block r
    { // columns first, straight from global: 8 lanes read one 32-byte block row
        // per load; the column DCT runs in registers
        const float *zc = noisy + s_zoff[r] + cb, *pc = pilot + s_poff[r] + cb;
        f2 x[8];
#pragma unroll
        for (int u = 0; u < 8; u++) x[u] = pk2(__ldg(zc + (long long)u * npitch), __ldg(pc + (long long)u * ppitch));
        dct8x2(x);
#pragma unroll
        for (int u = 0; u < 8; u++) upk2(x[u], sq[sidx(r, u, cb)], sp[sidx(r, u, cb)]);
    }
    __syncthreads();
    { // rows: thread (r, a)
        f2 x[8];
#pragma unroll
        for (int b = 0; b < 8; b++) x[b] = pk2(sq[sidx(r, a, b)], sp[sidx(r, a, b)]);
        dct8x2(x);
#pragma unroll
        for (int b = 0; b < 8; b++) upk2(x[b], sq[sidx(r, a, b)], sp[sidx(r, a, b)]);
    }
    __syncthreads();
    float acc = 0.f;
    { // group axis: thread (position e, quarter q); Haar, shrink, inverse Haar
        const int q = t & (Q - 1), e = t / Q;
        const int ea = e >> 3, eb = e & 7;
        float vp[8], vq[8];
        f2 v2[8];
#pragma unroll
        for (int i = 0; i < 8; i++) v2[i] = pk2(sp[sidx(8 * q + i, ea, eb)], sq[sidx(8 * q + i, ea, eb)]);
        haar_fwd_lanes2<Q>(v2, q);
#pragma unroll
        for (int i = 0; i < 8; i++) upk2(v2[i], vp[i], vq[i]);
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const float p2 = vp[i] * vp[i];
            const float den = p2 + sigma2;
            const float om = den > 0.f ? __fdividef(p2, den) : 0.f; // ~2 ulp; den << 2^126
            vq[i] *= om;
            acc = fmaf(om, om, acc);
        }
        haar_inv_lanes<Q>(vq, q);
#pragma unroll
        for (int i = 0; i < 8; i++) sq[sidx(8 * q + i, ea, eb)] = vq[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((t & 31) == 0) red[t >> 5] = acc;
    __syncthreads();
    if (t < K) {
        float s = 0.f;
        for (int i = 0; i < NT / 32; i++) s += red[i];
        const float wv = 1.f / fmaxf(sigma2 * s, eps_w);
        if (out.per_slot) out.w[s_slot[t]] = wv;
        else if (t == 0) out.w[g] = wv;
    }
    { // inverse rows
        float x[8];
#pragma unroll
        for (int b = 0; b < 8; b++) x[b] = sq[sidx(r, a, b)];
        idct8(x);
#pragma unroll
        for (int b = 0; b < 8; b++) sq[sidx(r, a, b)] = x[b];
    }
    __syncthreads();
    { // inverse columns, written straight out: 8 lanes per 32-byte block row
        float x[8];
#pragma unroll
        for (int u = 0; u < 8; u++) x[u] = sq[sidx(r, u, cb)];
        idct8(x);
        float *o = out.base + s_slot[r] * out.s_slot + cb;
#pragma unroll
        for (int u = 0; u < 8; u++) o[u * out.s_row] = x[u];
    }
}

} // namespace

template <int K>
static void wiener_k(int G, const float *noisy, int npitch, const float *pilot, int ppitch, int H, int W,
                     const int32_t *idx, float s2, float eps_w, const GroupOut &out, cudaStream_t st)
{
    k_wiener<K><<<G, K * 8, 0, st>>>(noisy, npitch, pilot, ppitch, H, W, idx, s2, eps_w, out);
}

cudaError_t launch_filter_wiener(const float *noisy, int npitch, const float *pilot, int ppitch, int H, int W,
                                 const int32_t *idx, int G, int K, float sigma, float eps_w, const GroupOut &out,
                                 cudaStream_t st)
{
    const float s2 = sigma * sigma;
    switch (K) {
    case 8: wiener_k<8>(G, noisy, npitch, pilot, ppitch, H, W, idx, s2, eps_w, out, st); break;
    case 16: wiener_k<16>(G, noisy, npitch, pilot, ppitch, H, W, idx, s2, eps_w, out, st); break;
    case 32: wiener_k<32>(G, noisy, npitch, pilot, ppitch, H, W, idx, s2, eps_w, out, st); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

} // namespace gbm3d
