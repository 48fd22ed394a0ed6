// wiener.cu -- stage-2 empirical Wiener filtering of every group (Sec. 4:
// 2-D DCT on the blocks, 1-D Haar along the group, Wiener shrinkage against
// the pilot, inverse, group weight).
//
// One CTA per group, K*8 threads: thread (r, a) owns row a of block r while
// the 8-point DCTs run (even/odd butterfly of the orthonormal DCT-II), then
// one thread per coefficient position runs the full-depth Haar along the K
// blocks in registers.  Both groups (noisy and pilot) are gathered straight
// from the images; the filtered group is written once, coalesced, in the
// group-major layout [g][r][a][b].
#include "internal.cuh"

namespace gbm3d {
namespace {

constexpr float kS = 0.70710678118654752f;
constexpr float kR8 = 0.35355339059327376f; // 1/sqrt(8)
// cos(k pi / 16)
constexpr float c1 = 0.98078528040323043f, c2 = 0.92387953251128674f, c3 = 0.83146961230254524f;
constexpr float c5 = 0.55557023301960218f, c6 = 0.38268343236508977f, c7 = 0.19509032201612825f;
constexpr int PS = 72; // smem block stride (64 + 8 pad: column passes are conflict-free)

// Orthonormal 8-point DCT-II, even/odd split.
__device__ __forceinline__ void dct8(float *x)
{
    const float s0 = x[0] + x[7], s1 = x[1] + x[6], s2 = x[2] + x[5], s3 = x[3] + x[4];
    const float d0 = x[0] - x[7], d1 = x[1] - x[6], d2 = x[2] - x[5], d3 = x[3] - x[4];
    const float e0 = s0 + s3, e1 = s1 + s2, f0 = s0 - s3, f1 = s1 - s2;
    x[0] = (e0 + e1) * kR8;
    x[4] = (e0 - e1) * kR8;
    x[2] = 0.5f * (c2 * f0 + c6 * f1);
    x[6] = 0.5f * (c6 * f0 - c2 * f1);
    x[1] = 0.5f * (c1 * d0 + c3 * d1 + c5 * d2 + c7 * d3);
    x[3] = 0.5f * (c3 * d0 - c7 * d1 - c1 * d2 - c5 * d3);
    x[5] = 0.5f * (c5 * d0 - c1 * d1 + c7 * d2 + c3 * d3);
    x[7] = 0.5f * (c7 * d0 - c5 * d1 + c3 * d2 - c1 * d3);
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

// Full-depth orthonormal Haar along the group, in registers: one level on
// the first LEN entries, then recurse on the LEN/2 low-pass entries.
template <int LEN>
__device__ __forceinline__ void haar_fwd(float *h)
{
    float t[LEN];
#pragma unroll
    for (int m = 0; m < LEN / 2; m++) {
        t[m] = (h[2 * m] + h[2 * m + 1]) * kS;
        t[LEN / 2 + m] = (h[2 * m] - h[2 * m + 1]) * kS;
    }
#pragma unroll
    for (int m = 0; m < LEN; m++) h[m] = t[m];
    if constexpr (LEN > 2) haar_fwd<LEN / 2>(h);
}

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

template <int K>
__global__ void __launch_bounds__(K * 8)
k_wiener(const float *__restrict__ noisy, int npitch, const float *__restrict__ pilot, int ppitch, int H, int W,
         const int32_t *__restrict__ idx, float sigma2, float eps_w, GroupOut out)
{
    constexpr int NT = K * 8;
    __shared__ __align__(16) float sp[K * PS];
    __shared__ __align__(16) float sq[K * PS];
    __shared__ float red[NT / 32];
    const int g = blockIdx.x, t = threadIdx.x;
    const int r = t >> 3, a = t & 7;
    {
        int k, l;
        block_kl(__ldg(idx + (size_t)g * K + r), H, W, k, l);
        const float *pz = noisy + (size_t)(k + a) * npitch + l;
        const float *py = pilot + (size_t)(k + a) * ppitch + l;
        float xz[8], xy[8];
#pragma unroll
        for (int b = 0; b < 8; b++) {
            xz[b] = __ldg(pz + b);
            xy[b] = __ldg(py + b);
        }
        dct8(xz);
        dct8(xy);
#pragma unroll
        for (int b = 0; b < 8; b++) {
            sq[r * PS + a * 8 + b] = xz[b];
            sp[r * PS + a * 8 + b] = xy[b];
        }
    }
    __syncthreads();
    { // columns: thread (r, b = a)
        const int b = a;
        float xz[8], xy[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            xz[u] = sq[r * PS + u * 8 + b];
            xy[u] = sp[r * PS + u * 8 + b];
        }
        dct8(xz);
        dct8(xy);
#pragma unroll
        for (int u = 0; u < 8; u++) {
            sq[r * PS + u * 8 + b] = xz[u];
            sp[r * PS + u * 8 + b] = xy[u];
        }
    }
    __syncthreads();
    for (int job = t; job < 128; job += NT) { // Haar along the group, both arrays
        float *arr = job < 64 ? sp : sq;
        const int e = job & 63;
        float h[K];
#pragma unroll
        for (int rr = 0; rr < K; rr++) h[rr] = arr[rr * PS + e];
        haar_fwd<K>(h);
#pragma unroll
        for (int rr = 0; rr < K; rr++) arr[rr * PS + e] = h[rr];
    }
    __syncthreads();
    float acc = 0.f;
    for (int e = t; e < K * 64; e += NT) {
        const int o = (e >> 6) * PS + (e & 63);
        const float P = sp[o];
        const float p2 = P * P;
        const float den = p2 + sigma2;
        const float om = den > 0.f ? p2 / den : 0.f;
        sq[o] *= om;
        acc = fmaf(om, om, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((t & 31) == 0) red[t >> 5] = acc;
    __syncthreads();
    for (int e = t; e < 64; e += NT) {
        float h[K];
#pragma unroll
        for (int rr = 0; rr < K; rr++) h[rr] = sq[rr * PS + e];
        haar_inv<K>(h);
#pragma unroll
        for (int rr = 0; rr < K; rr++) sq[rr * PS + e] = h[rr];
    }
    if (t < K) {
        float s = 0.f;
        for (int i = 0; i < NT / 32; i++) s += red[i];
        const float wv = 1.f / fmaxf(sigma2 * s, eps_w);
        if (out.per_slot) out.w[out.slot((long long)g * K + t)] = wv;
        else if (t == 0) out.w[g] = wv;
    }
    __syncthreads();
    {
        const int b = a;
        float x[8];
#pragma unroll
        for (int u = 0; u < 8; u++) x[u] = sq[r * PS + u * 8 + b];
        idct8(x);
#pragma unroll
        for (int u = 0; u < 8; u++) sq[r * PS + u * 8 + b] = x[u];
    }
    __syncthreads();
    {
        float x[8];
#pragma unroll
        for (int b = 0; b < 8; b++) x[b] = sq[r * PS + a * 8 + b];
        idct8(x);
        float4 *o = reinterpret_cast<float4 *>(out.row((long long)g * K + r, a));
        o[0] = make_float4(x[0], x[1], x[2], x[3]);
        o[1] = make_float4(x[4], x[5], x[6], x[7]);
    }
}

} // namespace

cudaError_t launch_filter_wiener(const float *noisy, int npitch, const float *pilot, int ppitch, int H, int W,
                                 const int32_t *idx, int G, int K, float sigma, float eps_w, const GroupOut &out,
                                 cudaStream_t st)
{
    const float s2 = sigma * sigma;
    switch (K) {
    case 8: k_wiener<8><<<G, 64, 0, st>>>(noisy, npitch, pilot, ppitch, H, W, idx, s2, eps_w, out); break;
    case 16: k_wiener<16><<<G, 128, 0, st>>>(noisy, npitch, pilot, ppitch, H, W, idx, s2, eps_w, out); break;
    case 32: k_wiener<32><<<G, 256, 0, st>>>(noisy, npitch, pilot, ppitch, H, W, idx, s2, eps_w, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

} // namespace gbm3d
