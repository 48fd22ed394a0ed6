// peak.cu -- measured FP32 FMA throughput of the current device: the
// denominator of the ALU roofline that the block matcher and the transforms
// are reported against (a measured figure instead of one derived from unit
// counts and the nominal clock).
#include "internal.cuh"

namespace gbm3d {
namespace {

constexpr int kChains = 8;     // independent FMA chains per thread
constexpr int kPeakThreads = 256;

// Where a thread would store its sum if it ever equalled the sentinel (it
// never does: the chains converge to 1); keeps the chains from being removed.
__device__ float g_peak_sink[kPeakThreads];

// Every thread runs kChains dependent chains x <- x a + b for `iters` steps:
// 2 kChains iters FLOP per thread.  The chains are independent, so the
// latency of one FMA is hidden by the others and by the other warps.
__global__ void __launch_bounds__(kPeakThreads) k_fma(float *out, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; j++) x[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (int it = 0; it < iters; it++)
#pragma unroll
        for (int j = 0; j < kChains; j++) x[j] = fmaf(x[j], a, b);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; j++) s += x[j];
    if (s == 12345.f) out[threadIdx.x] = s; // keeps the chains live, never true in practice
}

// The same with packed pairs (fma.rn.f32x2): 4 FLOP per instruction.
__global__ void __launch_bounds__(kPeakThreads) k_fma2(float *out, int iters, float a, float b)
{
    unsigned long long x[kChains / 2], av, bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
    for (int j = 0; j < kChains / 2; j++) {
        const float lo = (float)(threadIdx.x + 2 * j) * 1e-3f, hi = lo + 1e-3f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[j]) : "f"(lo), "f"(hi));
    }
    for (int it = 0; it < iters; it++)
#pragma unroll
        for (int j = 0; j < kChains / 2; j++) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[j]) : "l"(av), "l"(bv));
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains / 2; j++) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[j]));
        s += lo + hi;
    }
    if (s == 12345.f) out[threadIdx.x] = s;
}

} // namespace
} // namespace gbm3d

using namespace gbm3d;

extern "C" int gbm3d_measure_fp32_peak(double *scalar_tflops, double *packed_tflops, gbm3d_stream_t stream)
{
    if (!scalar_tflops || !packed_tflops) return set_error(GBM3D_EINVAL, "null pointer argument");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_error(GBM3D_ECUDA, cudaGetErrorString(e));
    float *sink = nullptr;
    e = cudaGetSymbolAddress((void **)&sink, g_peak_sink);
    if (e != cudaSuccess) return set_error(GBM3D_ECUDA, cudaGetErrorString(e));
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int blocks = sms * 8, iters = 1 << 15; // 8 CTAs of 256 threads per SM: 16 warps per scheduler
    const double flop = 2.0 * kChains * (double)iters * blocks * kPeakThreads;
    double best[2] = {0.0, 0.0};
    for (int kind = 0; kind < 2 && e == cudaSuccess; kind++)
        for (int rep = 0; rep < 4 && e == cudaSuccess; rep++) { // the first run warms up
            e = cudaEventRecord(t0, st);
            if (e != cudaSuccess) break;
            if (kind == 0)
                k_fma<<<blocks, kPeakThreads, 0, st>>>(sink, iters, 0.9999f, 1e-4f);
            else
                k_fma2<<<blocks, kPeakThreads, 0, st>>>(sink, iters, 0.9999f, 1e-4f);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(t1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
            if (e == cudaSuccess && rep > 0 && ms > 0.f) {
                const double tf = flop / (ms * 1e-3) / 1e12;
                if (tf > best[kind]) best[kind] = tf;
            }
        }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (e != cudaSuccess) return set_error(GBM3D_ECUDA, cudaGetErrorString(e));
    *scalar_tflops = best[0];
    *packed_tflops = best[1];
    return GBM3D_OK;
}
