// api.cu -- the extern "C" entry points of libgbm3d: argument validation
// (host only, before any launch), workspace layout and the two-stage driver
// (Sec. 1.1 BM3D1 / BM3D2, translation averaging of eq. firstEst).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "internal.cuh"

namespace gbm3d {

static thread_local char g_err[512] = "";
// Measurement hook (gbm3d_set_match_events): events recorded around the
// matching launch of each stage, or null.
static thread_local cudaEvent_t *g_match_events = nullptr;

static int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

static int cuda_fail(cudaError_t e, const char *where)
{
    return fail(GBM3D_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

int set_error(int code, const char *msg)
{
    return fail(code, "%s", msg);
}

cudaEvent_t *swap_match_events(cudaEvent_t *events)
{
    cudaEvent_t *old = g_match_events;
    g_match_events = events;
    return old;
}

static bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Block side and grid stride of a stage (stage 2: patch2 / step2 where set).
static int stage_patch(const gbm3d_params *p, int stage)
{
    return (stage == 2 && p->patch2 > 0) ? p->patch2 : p->patch;
}

static int stage_step(const gbm3d_params *p, int stage)
{
    return (stage == 2 && p->step2 > 0) ? p->step2 : p->step;
}

// Reference grid and group size of one stage.
struct StageGeom {
    int N, s, By, Bx, G, K;
};

static StageGeom stage_geom(int H, int W, const gbm3d_params *p, int stage)
{
    StageGeom g;
    g.N = stage_patch(p, stage);
    g.s = stage_step(p, stage);
    g.By = grid_count(H, g.N, g.s);
    g.Bx = grid_count(W, g.N, g.s);
    g.G = g.By * g.Bx;
    g.K = stage == 2 ? p->k2 : p->k1;
    return g;
}

static int check_params(const gbm3d_params *p)
{
    if (!p) return fail(GBM3D_EINVAL, "params is NULL");
    if (p->patch != 8 && p->patch != 16) return fail(GBM3D_EUNSUPPORTED, "patch %d: supported 8, 16", p->patch);
    if (p->patch2 != 0 && p->patch2 != 8 && p->patch2 != 16)
        return fail(GBM3D_EUNSUPPORTED, "patch2 %d: supported 0 (= patch), 8, 16", p->patch2);
    if (p->step < 1) return fail(GBM3D_EINVAL, "step %d < 1", p->step);
    if (p->step2 < 0) return fail(GBM3D_EINVAL, "step2 %d < 0", p->step2);
    if (p->search_radius < 0) return fail(GBM3D_EINVAL, "search_radius %d < 0", p->search_radius);
    if (p->levels < 1 || p->levels > 3) return fail(GBM3D_EUNSUPPORTED, "levels %d: supported 1..3", p->levels);
    for (int k : {p->k1, p->k2})
        if (!pow2(k) || k < 8 || k > kMaxK) return fail(GBM3D_EUNSUPPORTED, "group size %d: supported 8, 16, 32", k);
    if (p->k1 % (1 << p->levels)) return fail(GBM3D_EINVAL, "k1 %d not divisible by 2^levels", p->k1);
    if (p->cycle_spins < 1 || p->cycle_spins > 4)
        return fail(GBM3D_EUNSUPPORTED, "cycle_spins %d: supported 1..4", p->cycle_spins);
    if (p->translations < 1 || p->translations > 3)
        return fail(GBM3D_EUNSUPPORTED, "translations %d: supported 1..3", p->translations);
    if (p->stages < 1 || p->stages > 2) return fail(GBM3D_EINVAL, "stages %d: 1 or 2", p->stages);
    if (!(p->eps_w > 0.f) || !isfinite(p->eps_w)) return fail(GBM3D_EINVAL, "eps_w must be positive");
    if (!isfinite(p->tau_a) || !isfinite(p->tau_b) || !isfinite(p->kaiser_beta) || p->kaiser_beta < 0.f)
        return fail(GBM3D_EINVAL, "tau_a, tau_b, kaiser_beta must be finite (beta >= 0)");
    if (p->match_engine < 0 || p->match_engine > 3)
        return fail(GBM3D_EINVAL, "match_engine %d: 0 auto, 1 direct, 2 tensor cores, 3 box sums", p->match_engine);
    for (int sg = 1; sg <= 2; sg++)
        if (match_smem_bytes(stage_step(p, sg), p->search_radius, stage_patch(p, sg)) > 227 * 1024)
            return fail(GBM3D_EUNSUPPORTED, "search region of R=%d, s=%d, N=%d exceeds shared memory",
                        p->search_radius, stage_step(p, sg), stage_patch(p, sg));
    return GBM3D_OK;
}

// The whole method: stage 2's Wiener filter is built for 8 x 8 blocks.
static int check_denoise_params(const gbm3d_params *p)
{
    if (p->stages == 2 && stage_patch(p, 2) != kPatch)
        return fail(GBM3D_EUNSUPPORTED, "stage-2 block side %d: the Wiener filter supports N = 8 (set patch2 = 8)",
                    stage_patch(p, 2));
    return GBM3D_OK;
}

// Largest block side the calls on these params use.
static int max_patch(const gbm3d_params *p)
{
    const int n2 = stage_patch(p, 2);
    return p->patch > n2 ? p->patch : n2;
}

static int check_image(int H, int W, int pitch, int N)
{
    if (H < N || W < N) return fail(GBM3D_EINVAL, "image %dx%d smaller than the %d-pixel block", H, W, N);
    if (pitch < W) return fail(GBM3D_EINVAL, "pitch %d < W %d", pitch, W);
    if ((long long)H * W >= (1ll << 31) - 1 || (long long)H * pitch >= (1ll << 40))
        return fail(GBM3D_EINVAL, "image %dx%d too large for int32 block indices", H, W);
    return GBM3D_OK;
}

static int check_window(int H, int W, int N, int R, int K)
{
    const long long wy = (H - N < R ? H - N : R) + 1, wx = (W - N < R ? W - N : R) + 1;
    if (wy * wx < K)
        return fail(GBM3D_EINVAL, "search window holds %lld blocks, fewer than K = %d", wy * wx, K);
    return GBM3D_OK;
}

// The tensor-core engine where the parameters allow it (and it is not
// switched off), else the direct one; engine 2 where unsupported is refused.
static int check_engine(int H, int W, const gbm3d_params *p, const StageGeom &g, int K)
{
    if (p->match_engine == 3 && !match_box_supported(g.N, g.s, p->search_radius, K))
        return fail(GBM3D_EUNSUPPORTED, "box-sum matching needs N = 8, s <= 3 and K <= 32 (N=%d s=%d K=%d)", g.N, g.s,
                    K);
    if (p->match_engine == 2 && !match_tc_supported(H, W, g.N, g.s, p->search_radius, K))
        return fail(GBM3D_EUNSUPPORTED,
                    "tensor-core matching needs N = 8, 7 s + 2 R + 1 <= 64 and K <= 32 (N=%d s=%d R=%d K=%d)", g.N,
                    g.s, p->search_radius, K);
    return GBM3D_OK;
}

// Checks of the whole method on an H x W image (both stages' windows and engines).
static int check_stages(int H, int W, const gbm3d_params *p)
{
    int st;
    for (int sg = 1; sg <= p->stages; sg++) {
        const StageGeom g = stage_geom(H, W, p, sg);
        if ((st = check_window(H, W, g.N, p->search_radius, g.K))) return st;
        if ((st = check_engine(H, W, p, g, g.K))) return st;
    }
    return GBM3D_OK;
}

static cudaError_t match_any(const float *img, int H, int W, int pitch, const StageGeom &g, const gbm3d_params *p,
                             int K, int32_t *idx, float *dist, cudaStream_t st)
{
    if (p->match_engine == 3)
        return launch_match_box(img, H, W, pitch, g.By, g.Bx, g.s, p->search_radius, K, idx, dist, st);
    if (p->match_engine != 1 && match_tc_supported(H, W, g.N, g.s, p->search_radius, K))
        return launch_match_tc(img, H, W, pitch, g.By, g.Bx, g.s, p->search_radius, K, idx, dist, st);
    return launch_match(img, H, W, pitch, g.By, g.Bx, g.N, g.s, p->search_radius, K, idx, dist, st);
}

// Kaiser window kappa[n] = I0(beta sqrt(1 - (2n/(N-1) - 1)^2)) / I0(beta), with
// I0 summed from its power series in double precision.
static double bessel_i0(double x)
{
    double s = 1.0, t = 1.0;
    for (int k = 1; k < 100; k++) {
        t *= 0.5 * x / k;
        s += t * t;
    }
    return s;
}

static void kaiser(int N, float beta, float *out)
{
    for (int n = 0; n < N; n++) {
        if (beta <= 0.f) {
            out[n] = 1.f;
            continue;
        }
        const double r = 2.0 * n / (N - 1) - 1.0;
        out[n] = (float)(bessel_i0(beta * sqrt(fmax(0.0, 1.0 - r * r))) / bessel_i0(beta));
    }
}

// One workspace layout serves every call (offsets in bytes):
//   csr    inverted match lists of the current stage (+ slot_of)
//   ht     stage-1 wavelet pyramid and pixel-offset table
//   planes filtered blocks, position-planar (aggregation order): the larger
//          stage's G K N^2 floats
//   wslot  per-slot weights;  idx  match lists (entries: max over stages of G,
//          times max(k1, k2))
//   y1     stage-1 estimate (pitch W); zs, ys, y1s translation buffers
struct Sizes {
    StageGeom st[2]; // stage 1, stage 2
    long long nent;  // entries the csr, wslot and idx areas hold
    HtGeom ht;
    size_t csr, ht_off, planes, wslot, idx, y1, zs, ys, y1s, total;
};

static Sizes sizes(int H, int W, const gbm3d_params *p)
{
    Sizes z{};
    z.st[0] = stage_geom(H, W, p, 1);
    z.st[1] = stage_geom(H, W, p, 2);
    const int Gmax = z.st[0].G > z.st[1].G ? z.st[0].G : z.st[1].G;
    const int Kmax = p->k1 > p->k2 ? p->k1 : p->k2;
    z.nent = (long long)Gmax * Kmax;
    z.ht = ht_geom(z.st[0].By, z.st[0].Bx, p->k1, p->levels, z.st[0].N);
    size_t vox = 0; // floats of one stage's filtered blocks
    for (const StageGeom &g : z.st) {
        const size_t v = (size_t)g.G * g.K * g.N * g.N;
        if (v > vox) vox = v;
    }
    const size_t img = align_up((size_t)H * W * sizeof(float));
    size_t o = 0;
    z.csr = o;
    o += align_up(agg_layout(H, W, (int)z.nent, 1, true).bytes);
    z.ht_off = o;
    o += align_up(z.ht.bytes);
    z.planes = o;
    o += align_up(vox * sizeof(float));
    z.wslot = o;
    o += align_up((size_t)z.nent * sizeof(float));
    z.idx = o;
    o += align_up((size_t)z.nent * sizeof(int32_t));
    z.y1 = o;
    o += img;
    if (p->translations > 1) {
        z.zs = o;
        o += img;
        z.ys = o;
        o += img;
        z.y1s = o;
        o += img;
    }
    z.total = o;
    return z;
}

static bool aligned(const void *ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

// Position-planar output descriptor over the workspace for a stage.
static GroupOut planar_out(const Sizes &S, char *ws, int H, int W, const StageGeom &g)
{
    const AggLayout L = agg_layout(H, W, g.G, g.K, true);
    return position_planar((float *)(ws + S.planes), (const int *)(ws + S.csr + L.slot_of), (long long)g.G * g.K,
                           (float *)(ws + S.wslot), g.N);
}

// A second stream per host thread and device, with two events, on which
// stage 1 builds its inverted lists while the wavelet transforms run (they
// need only the match lists; the TV pass that permutes into the planar
// layout waits for the lists).  Not used while the caller's stream is being
// captured into a graph (every capture branch would share this stream).
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t ready = nullptr, done = nullptr;
};

static bool side_stream(cudaStream_t st, SideStream **out)
{
    constexpr int kMaxDev = 64;
    static thread_local SideStream side[kMaxDev];
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return false;
    SideStream &ss = side[dev];
    if (!ss.s) {
        if (cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking) != cudaSuccess) {
            ss.s = nullptr;
            return false;
        }
        if (cudaEventCreateWithFlags(&ss.ready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ss.done, cudaEventDisableTiming) != cudaSuccess) {
            // back to the empty state, so that a later call retries from scratch
            // and this one takes the path without overlap
            if (ss.ready) cudaEventDestroy(ss.ready);
            if (ss.done) cudaEventDestroy(ss.done);
            cudaStreamDestroy(ss.s);
            ss = SideStream{};
            return false;
        }
    }
    *out = &ss;
    return true;
}

// ---- one stage on (possibly shifted) images ------------------------------
static int run_stage1(const float *z, int zp, int H, int W, float sigma, const gbm3d_params *p, const Sizes &S,
                      char *ws, float *out, int op, cudaStream_t st)
{
    const StageGeom &g = S.st[0];
    const int K = g.K;
    int32_t *idx = (int32_t *)(ws + S.idx);
    if (g_match_events) cudaEventRecord(g_match_events[0], st);
    cudaError_t e = match_any(z, H, W, zp, g, p, K, idx, nullptr, st);
    if (e != cudaSuccess) return cuda_fail(e, "match (stage 1)");
    if (g_match_events) cudaEventRecord(g_match_events[1], st);
    SideStream *side = nullptr;
    const bool overlap = side_stream(st, &side);
    if (overlap) { // inverted lists on the side stream, overlapping the transforms
        e = cudaEventRecord(side->ready, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side->s, side->ready, 0);
        if (e == cudaSuccess) e = build_csr(idx, g.G, K, H, W, g.N, ws + S.csr, true, side->s);
        if (e == cudaSuccess) e = cudaEventRecord(side->done, side->s);
    } else {
        e = build_csr(idx, g.G, K, H, W, g.N, ws + S.csr, true, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "inverted lists (stage 1)");
    const GroupOut go = planar_out(S, ws, H, W, g);
    e = launch_ht_transforms(z, H, W, zp, idx, S.ht, sigma, p->tau_a, p->tau_b, p->cycle_spins, go, ws + S.ht_off,
                             st);
    if (e == cudaSuccess && overlap) e = cudaStreamWaitEvent(st, side->done, 0);
    if (e == cudaSuccess) e = launch_ht_weights(S.ht, p->eps_w, go, ws + S.ht_off, st);
    if (e != cudaSuccess) return cuda_fail(e, "filter_ht");
    float win[kMaxPatch];
    kaiser(g.N, 0.f, win);
    e = launch_aggregate_planar(go.base, go.w, g.G * K, H, W, g.N, op, win, out, ws + S.csr, st);
    if (e != cudaSuccess) return cuda_fail(e, "aggregate (stage 1)");
    return GBM3D_OK;
}

static int run_stage2(const float *z, int zp, const float *y1, int yp, int H, int W, float sigma,
                      const gbm3d_params *p, const Sizes &S, char *ws, float *out, int op, cudaStream_t st)
{
    const StageGeom &g = S.st[1];
    const int K = g.K;
    int32_t *idx = (int32_t *)(ws + S.idx);
    if (g_match_events) cudaEventRecord(g_match_events[2], st);
    cudaError_t e = match_any(y1, H, W, yp, g, p, K, idx, nullptr, st);
    if (e != cudaSuccess) return cuda_fail(e, "match (stage 2)");
    if (g_match_events) cudaEventRecord(g_match_events[3], st);
    e = build_csr(idx, g.G, K, H, W, g.N, ws + S.csr, true, st);
    if (e != cudaSuccess) return cuda_fail(e, "inverted lists (stage 2)");
    const GroupOut go = planar_out(S, ws, H, W, g);
    e = launch_filter_wiener(z, zp, y1, yp, H, W, idx, g.G, K, sigma, p->eps_w, go, st);
    if (e != cudaSuccess) return cuda_fail(e, "filter_wiener");
    float win[kMaxPatch];
    kaiser(g.N, p->kaiser_beta, win);
    e = launch_aggregate_planar(go.base, go.w, g.G * K, H, W, g.N, op, win, out, ws + S.csr, st);
    if (e != cudaSuccess) return cuda_fail(e, "aggregate (stage 2)");
    return GBM3D_OK;
}

// Circular 2-D shift: dst[y][x] (+)= scale * src[y - h][x - h] (periodic).
__global__ void k_shift(const float *__restrict__ src, int sp, float *__restrict__ dst, int dp, int H, int W, int h,
                        float scale, int acc)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= W || y >= H) return;
    int ys = (y - h) % H, xs = (x - h) % W;
    if (ys < 0) ys += H;
    if (xs < 0) xs += W;
    const float v = scale * src[(size_t)ys * sp + xs];
    float *o = dst + (size_t)y * dp + x;
    *o = acc ? *o + v : v;
}

cudaError_t launch_shift(const float *src, int spitch, float *dst, int dpitch, int H, int W, int h, float scale,
                         int accumulate, cudaStream_t st)
{
    dim3 grid((W + 31) / 32, (H + 7) / 8);
    k_shift<<<grid, 256, 0, st>>>(src, spitch, dst, dpitch, H, W, h, scale, accumulate);
    return cudaGetLastError();
}

// ---- colour (an extension: the paper is grayscale) --------------------------
// Opponent transform per pixel, src planes -> dst planes (inverse: back to RGB):
//   Y = (R+G+B)/3, U = (R-B)/2, V = (R-2G+B)/4;  R = Y+U+2V/3, G = Y-4V/3, B = Y-U+2V/3.
__global__ void k_opp(const float *__restrict__ src, int sp, long long splane, float *dst, int dp, long long dplane,
                      int H, int W, int inverse)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= W || y >= H) return;
    const size_t si = (size_t)y * sp + x, di = (size_t)y * dp + x;
    const float a = src[si], b = src[si + splane], c = src[si + 2 * splane];
    float o0, o1, o2;
    if (!inverse) {
        o0 = (a + b + c) * (1.f / 3.f);
        o1 = (a - c) * 0.5f;
        o2 = (a - 2.f * b + c) * 0.25f;
    } else {
        o0 = a + b + c * (2.f / 3.f);
        o1 = a - c * (4.f / 3.f);
        o2 = a - b + c * (2.f / 3.f);
    }
    dst[di] = o0;
    dst[di + dplane] = o1;
    dst[di + 2 * dplane] = o2;
}

static cudaError_t launch_opp(const float *src, int sp, long long splane, float *dst, int dp, long long dplane, int H,
                              int W, int inverse, cudaStream_t st)
{
    dim3 grid((W + 31) / 32, (H + 7) / 8);
    k_opp<<<grid, 256, 0, st>>>(src, sp, splane, dst, dp, dplane, H, W, inverse);
    return cudaGetLastError();
}

// Noise deviation of opponent channel c per unit deviation in R, G, B: the
// norm of row c of the forward transform (the rows are orthogonal).
static double opp_scale(int c)
{
    static const double sq[3] = {1.0 / 3.0, 0.5, 3.0 / 8.0};
    return sqrt(sq[c]);
}

// One colour stage on opponent planes zo (pitch W, plane stride n): match
// once on the guide plane (zo[0] in stage 1, y1o[0] in stage 2), build the
// inverted lists once, then filter and aggregate each channel with its own
// sigma into out plane c (pitch op, plane stride oplane).
static int run_stage_color(const float *zo, const float *y1o, long long n, int H, int W, float sigma,
                           const gbm3d_params *p, const Sizes &S, char *ws, float *out, int op, long long oplane,
                           cudaStream_t st)
{
    const bool s2 = y1o != nullptr;
    const StageGeom &g = S.st[s2 ? 1 : 0];
    const int K = g.K;
    int32_t *idx = (int32_t *)(ws + S.idx);
    if (g_match_events) cudaEventRecord(g_match_events[s2 ? 2 : 0], st);
    cudaError_t e = match_any(s2 ? y1o : zo, H, W, W, g, p, K, idx, nullptr, st);
    if (e != cudaSuccess) return cuda_fail(e, s2 ? "match (stage 2)" : "match (stage 1)");
    if (g_match_events) cudaEventRecord(g_match_events[s2 ? 3 : 1], st);
    e = build_csr(idx, g.G, K, H, W, g.N, ws + S.csr, true, st);
    if (e != cudaSuccess) return cuda_fail(e, "inverted lists");
    const GroupOut go = planar_out(S, ws, H, W, g);
    float win[kMaxPatch];
    kaiser(g.N, s2 ? p->kaiser_beta : 0.f, win);
    for (int c = 0; c < 3; c++) {
        const float sc = (float)((double)sigma * opp_scale(c));
        if (s2)
            e = launch_filter_wiener(zo + c * n, W, y1o + c * n, W, H, W, idx, g.G, K, sc, p->eps_w, go, st);
        else
            e = launch_filter_ht(zo + c * n, H, W, W, idx, S.ht, sc, p->tau_a, p->tau_b, p->cycle_spins, p->eps_w, go,
                                 ws + S.ht_off, st);
        if (e != cudaSuccess) return cuda_fail(e, s2 ? "filter_wiener" : "filter_ht");
        e = launch_aggregate_planar(go.base, go.w, g.G * K, H, W, g.N, op, win, out + c * oplane, ws + S.csr, st);
        if (e != cudaSuccess) return cuda_fail(e, "aggregate");
    }
    return GBM3D_OK;
}

} // namespace gbm3d

using namespace gbm3d;

extern "C" {

const char *gbm3d_last_error_string(void) { return g_err; }

const char *gbm3d_version(void) { return "gbm3d 0.3 (sm_103a)"; }

int gbm3d_set_match_events(void *events)
{
    g_match_events = (cudaEvent_t *)events;
    return GBM3D_OK;
}

int gbm3d_match_stats(unsigned long long *timeouts, unsigned long long *rematched)
{
    if (!timeouts || !rematched) return fail(GBM3D_EINVAL, "timeouts/rematched is NULL");
    const cudaError_t e = tc_stats(timeouts, rematched);
    return e == cudaSuccess ? GBM3D_OK : cuda_fail(e, "match_stats");
}

int gbm3d_params_default(gbm3d_params *p, int preset)
{
    if (!p) return fail(GBM3D_EINVAL, "params is NULL");
    if (preset != 0 && preset != 1) return fail(GBM3D_EINVAL, "unknown preset %d", preset);
    p->patch = 8;
    p->levels = 3;
    p->cycle_spins = 2;
    p->stages = 2;
    p->tau_a = 3.6f;
    p->tau_b = 0.3f;
    p->kaiser_beta = 2.0f;
    p->eps_w = 1e-8f;
    p->match_engine = 0;
    if (preset == 0) {
        p->step = 3;
        p->search_radius = 19;
        p->k1 = 16;
        p->k2 = 32;
        p->translations = 1;
        p->patch2 = 8;
        p->step2 = 3;
    } else { // Sec. 5: 16 x 16 tiling blocks in stage 1, 8 x 8 in stage 2
        p->patch = 16;
        p->step = 16;
        p->search_radius = 16;
        p->k1 = 16;
        p->k2 = 16;
        p->translations = 2;
        p->patch2 = 8;
        p->step2 = 8;
    }
    g_err[0] = 0;
    return GBM3D_OK;
}

int gbm3d_params_stage(const gbm3d_params *p, int stage, gbm3d_params *out)
{
    if (!p || !out) return fail(GBM3D_EINVAL, "params is NULL");
    if (stage != 1 && stage != 2) return fail(GBM3D_EINVAL, "stage %d: 1 or 2", stage);
    gbm3d_params q = *p;
    q.patch = stage_patch(p, stage);
    q.step = stage_step(p, stage);
    q.patch2 = 0;
    q.step2 = 0;
    *out = q;
    return GBM3D_OK;
}

// Colour workspace: the grayscale layout, then the opponent planes of the
// input and of the stage-1 estimate (3 + 3 images, pitch W).
static size_t color_extra(int H, int W) { return 6 * align_up((size_t)H * W * sizeof(float)); }

int gbm3d_workspace_bytes_color(int H, int W, const gbm3d_params *p, size_t *bytes)
{
    int st = check_params(p);
    if (st) return st;
    if (!bytes) return fail(GBM3D_EINVAL, "bytes is NULL");
    if ((st = check_image(H, W, W, max_patch(p)))) return st;
    if (p->translations != 1) return fail(GBM3D_EUNSUPPORTED, "colour: translations must be 1");
    *bytes = sizes(H, W, p).total + color_extra(H, W);
    return GBM3D_OK;
}

int gbm3d_grid_dims(int H, int W, const gbm3d_params *p, int *By, int *Bx)
{
    int st = check_params(p);
    if (st) return st;
    if (!By || !Bx) return fail(GBM3D_EINVAL, "By/Bx is NULL");
    if ((st = check_image(H, W, W, p->patch))) return st;
    *By = grid_count(H, p->patch, p->step);
    *Bx = grid_count(W, p->patch, p->step);
    return GBM3D_OK;
}

int gbm3d_workspace_bytes(int H, int W, const gbm3d_params *p, size_t *bytes)
{
    int st = check_params(p);
    if (st) return st;
    if (!bytes) return fail(GBM3D_EINVAL, "bytes is NULL");
    if ((st = check_image(H, W, W, max_patch(p)))) return st;
    *bytes = sizes(H, W, p).total;
    return GBM3D_OK;
}

int gbm3d_match(const float *img, int H, int W, int pitch, const gbm3d_params *p, int K, int32_t *idx, float *dist,
                void *ws, gbm3d_stream_t stream)
{
    (void)ws;
    int st = check_params(p);
    if (st) return st;
    if ((st = check_image(H, W, pitch, p->patch))) return st;
    if (!img || !idx) return fail(GBM3D_EINVAL, "img/idx is NULL");
    if (K < 2 || K > kMaxK) return fail(GBM3D_EUNSUPPORTED, "K = %d: supported 2..32", K);
    const StageGeom g = stage_geom(H, W, p, 1);
    if ((st = check_window(H, W, g.N, p->search_radius, K))) return st;
    if ((st = check_engine(H, W, p, g, K))) return st;
    cudaError_t e = match_any(img, H, W, pitch, g, p, K, idx, dist, (cudaStream_t)stream);
    return e == cudaSuccess ? GBM3D_OK : cuda_fail(e, "match");
}

int gbm3d_filter_ht(const float *noisy, int H, int W, int pitch, const int32_t *idx, float sigma,
                    const gbm3d_params *p, float *groups, float *w, void *ws, gbm3d_stream_t stream)
{
    int st = check_params(p);
    if (st) return st;
    if ((st = check_image(H, W, pitch, max_patch(p)))) return st;
    if (!noisy || !idx || !groups || !w || !ws) return fail(GBM3D_EINVAL, "null pointer argument");
    if (!(sigma >= 0.f) || !isfinite(sigma)) return fail(GBM3D_EINVAL, "sigma must be finite and >= 0");
    if (!aligned(ws, kAlign) || !aligned(groups, 16)) return fail(GBM3D_EINVAL, "ws must be 256-byte aligned");
    const Sizes S = sizes(H, W, p);
    cudaError_t e = launch_filter_ht(noisy, H, W, pitch, idx, S.ht, sigma, p->tau_a, p->tau_b, p->cycle_spins,
                                     p->eps_w, group_major(groups, w, p->patch), (char *)ws + S.ht_off,
                                     (cudaStream_t)stream);
    return e == cudaSuccess ? GBM3D_OK : cuda_fail(e, "filter_ht");
}

int gbm3d_filter_wiener(const float *noisy, const float *pilot, int H, int W, int pitch, const int32_t *idx,
                        float sigma, const gbm3d_params *p, float *groups, float *w, void *ws, gbm3d_stream_t stream)
{
    (void)ws;
    int st = check_params(p);
    if (st) return st;
    if (p->patch != kPatch)
        return fail(GBM3D_EUNSUPPORTED, "patch %d: the Wiener filter supports N = 8", p->patch);
    if ((st = check_image(H, W, pitch, p->patch))) return st;
    if (!noisy || !pilot || !idx || !groups || !w) return fail(GBM3D_EINVAL, "null pointer argument");
    if (!(sigma >= 0.f) || !isfinite(sigma)) return fail(GBM3D_EINVAL, "sigma must be finite and >= 0");
    if (!aligned(groups, 16)) return fail(GBM3D_EINVAL, "groups must be 16-byte aligned");
    const int G = grid_count(H, kPatch, p->step) * grid_count(W, kPatch, p->step);
    cudaError_t e = launch_filter_wiener(noisy, pitch, pilot, pitch, H, W, idx, G, p->k2, sigma, p->eps_w,
                                         group_major(groups, w, kPatch), (cudaStream_t)stream);
    return e == cudaSuccess ? GBM3D_OK : cuda_fail(e, "filter_wiener");
}

int gbm3d_aggregate(const float *groups, const float *w, const int32_t *idx, int K, int H, int W, int pitch,
                    const gbm3d_params *p, float window_beta, float *out, void *ws, gbm3d_stream_t stream)
{
    int st = check_params(p);
    if (st) return st;
    if ((st = check_image(H, W, pitch, max_patch(p)))) return st;
    if (!groups || !w || !idx || !out || !ws) return fail(GBM3D_EINVAL, "null pointer argument");
    if (!pow2(K) || K > kMaxK) return fail(GBM3D_EUNSUPPORTED, "K = %d: supported powers of two up to 32", K);
    if (K > (p->k1 > p->k2 ? p->k1 : p->k2))
        return fail(GBM3D_EINVAL, "K = %d exceeds max(k1, k2): the workspace is sized by the params", K);
    if (!(window_beta >= 0.f) || !isfinite(window_beta)) return fail(GBM3D_EINVAL, "window_beta must be >= 0");
    if (!aligned(ws, kAlign)) return fail(GBM3D_EINVAL, "ws must be 256-byte aligned");
    const int N = p->patch;
    const int G = grid_count(H, N, p->step) * grid_count(W, N, p->step);
    float win[kMaxPatch];
    kaiser(N, window_beta, win);
    const Sizes S = sizes(H, W, p);
    cudaError_t e =
        launch_aggregate(groups, w, idx, G, K, H, W, N, pitch, win, out, (char *)ws + S.csr, (cudaStream_t)stream);
    return e == cudaSuccess ? GBM3D_OK : cuda_fail(e, "aggregate");
}

int gbm3d_aggregate_noalloc(const float *groups, const float *w, const int32_t *idx, int K, int H, int W,
                            int pitch, const gbm3d_params *p, float window_beta, float *out, gbm3d_stream_t stream)
{
    int st = check_params(p);
    if (st) return st;
    if ((st = check_image(H, W, pitch, p->patch))) return st;
    if (!groups || !w || !idx || !out) return fail(GBM3D_EINVAL, "null pointer argument");
    if (!pow2(K) || K > kMaxK) return fail(GBM3D_EUNSUPPORTED, "K = %d: supported powers of two up to 32", K);
    if (!(window_beta >= 0.f) || !isfinite(window_beta)) return fail(GBM3D_EINVAL, "window_beta must be >= 0");
    const int N = p->patch;
    const int G = grid_count(H, N, p->step) * grid_count(W, N, p->step);
    const AggLayout L = agg_layout(H, W, G, K);
    if (L.bytes > kFixedScratchBytes)
        return fail(GBM3D_ENOMEM, "aggregation of a %dx%d image with K = %d needs %zu bytes of scratch, more than "
                    "the fixed %zu bytes of gbm3d_aggregate_noalloc", H, W, K, L.bytes, kFixedScratchBytes);
    void *scratch = nullptr;
    cudaError_t e = fixed_scratch(&scratch);
    if (e != cudaSuccess) return cuda_fail(e, "fixed scratch address");
    float win[kMaxPatch];
    kaiser(N, window_beta, win);
    e = launch_aggregate(groups, w, idx, G, K, H, W, N, pitch, win, out, scratch, (cudaStream_t)stream);
    return e == cudaSuccess ? GBM3D_OK : cuda_fail(e, "aggregate_noalloc");
}

int gbm3d_denoise(const float *noisy, int H, int W, int pitch, float sigma, const gbm3d_params *p, float *out,
                  void *ws, gbm3d_stream_t stream)
{
    int st = check_params(p);
    if (st) return st;
    if ((st = check_denoise_params(p))) return st;
    if ((st = check_image(H, W, pitch, max_patch(p)))) return st;
    if (!noisy || !out || !ws) return fail(GBM3D_EINVAL, "null pointer argument");
    if (noisy == out) return fail(GBM3D_EINVAL, "out must not alias noisy");
    if (!(sigma >= 0.f) || !isfinite(sigma)) return fail(GBM3D_EINVAL, "sigma must be finite and >= 0");
    if (!aligned(ws, kAlign)) return fail(GBM3D_EINVAL, "ws must be 256-byte aligned");
    if ((st = check_stages(H, W, p))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const Sizes S = sizes(H, W, p);
    char *base = (char *)ws;
    float *y1 = (float *)(base + S.y1);
    const int T = p->translations;
    // translations h in {0, N/4, N/2} with each stage's own block side N
    const int N1 = S.st[0].N, N2 = S.st[1].N;
    const int hs[3] = {0, N1 / 4, N1 / 2}, hs2[3] = {0, N2 / 4, N2 / 2};
    float *final_out = p->stages == 1 ? out : nullptr;
    // stage 1: Y1 = (1/T) sum_h S_{-h} phi1(S_h Z)
    if (T == 1) {
        st = run_stage1(noisy, pitch, H, W, sigma, p, S, base, final_out ? out : y1, final_out ? pitch : W, s);
        if (st) return st;
    } else {
        float *zs = (float *)(base + S.zs), *ys = (float *)(base + S.ys);
        float *acc = final_out ? out : y1;
        const int ap = final_out ? pitch : W;
        for (int t = 0; t < T; t++) {
            cudaError_t e = launch_shift(noisy, pitch, zs, W, H, W, hs[t], 1.f, 0, s);
            if (e != cudaSuccess) return cuda_fail(e, "shift");
            if ((st = run_stage1(zs, W, H, W, sigma, p, S, base, ys, W, s))) return st;
            e = launch_shift(ys, W, acc, ap, H, W, -hs[t], 1.f / T, t > 0, s);
            if (e != cudaSuccess) return cuda_fail(e, "shift");
        }
    }
    if (p->stages == 1) return GBM3D_OK;
    // stage 2: Y2 = (1/T) sum_h S_{-h} phi2(S_h Z, S_h Y1)
    if (T == 1) return run_stage2(noisy, pitch, y1, W, H, W, sigma, p, S, base, out, pitch, s);
    float *zs = (float *)(base + S.zs), *ys = (float *)(base + S.ys), *y1s = (float *)(base + S.y1s);
    for (int t = 0; t < T; t++) {
        cudaError_t e = launch_shift(noisy, pitch, zs, W, H, W, hs2[t], 1.f, 0, s);
        if (e == cudaSuccess) e = launch_shift(y1, W, y1s, W, H, W, hs2[t], 1.f, 0, s);
        if (e != cudaSuccess) return cuda_fail(e, "shift");
        if ((st = run_stage2(zs, W, y1s, W, H, W, sigma, p, S, base, ys, W, s))) return st;
        e = launch_shift(ys, W, out, pitch, H, W, -hs2[t], 1.f / T, t > 0, s);
        if (e != cudaSuccess) return cuda_fail(e, "shift");
    }
    return GBM3D_OK;
}

int gbm3d_workspace_bytes_learned(int H, int W, const gbm3d_params *p, size_t *bytes)
{
    int st = check_params(p);
    if (st) return st;
    if (!bytes) return fail(GBM3D_EINVAL, "bytes is NULL");
    if ((st = check_image(H, W, W, max_patch(p)))) return st;
    *bytes = sizes(H, W, p).total + align_up(pilot_infer_bytes(H, W));
    return GBM3D_OK;
}

int gbm3d_denoise_learned(const float *noisy, int H, int W, int pitch, float sigma, const gbm3d_params *p,
                          const float *theta, float *out, void *ws, gbm3d_stream_t stream)
{
    int st = check_params(p);
    if (st) return st;
    if (p->stages != 2 || p->translations != 1 || stage_patch(p, 2) != kPatch)
        return fail(GBM3D_EUNSUPPORTED, "learned pilot: stages 2, translations 1 and an 8 x 8 stage 2 required");
    if ((st = check_image(H, W, pitch, max_patch(p)))) return st;
    if (!noisy || !out || !ws || !theta) return fail(GBM3D_EINVAL, "null pointer argument");
    if (noisy == out) return fail(GBM3D_EINVAL, "out must not alias noisy");
    if (!(sigma >= 0.f) || !isfinite(sigma)) return fail(GBM3D_EINVAL, "sigma must be finite and >= 0");
    if (!aligned(ws, kAlign)) return fail(GBM3D_EINVAL, "ws must be 256-byte aligned");
    const StageGeom g2 = stage_geom(H, W, p, 2);
    if ((st = check_window(H, W, g2.N, p->search_radius, g2.K))) return st;
    if ((st = check_engine(H, W, p, g2, g2.K))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const Sizes S = sizes(H, W, p);
    char *base = (char *)ws;
    float *y1 = (float *)(base + S.y1);
    cudaError_t e = launch_pilot(noisy, H, W, pitch, sigma, theta, y1, W, base + S.total, s);
    if (e != cudaSuccess) return cuda_fail(e, "learned pilot");
    return run_stage2(noisy, pitch, y1, W, H, W, sigma, p, S, base, out, pitch, s);
}

int gbm3d_denoise_color(const float *noisy, int H, int W, int pitch, long long plane_stride, float sigma,
                        const gbm3d_params *p, float *out, void *ws, gbm3d_stream_t stream)
{
    int st = check_params(p);
    if (st) return st;
    if ((st = check_denoise_params(p))) return st;
    if ((st = check_image(H, W, pitch, max_patch(p)))) return st;
    if (!noisy || !out || !ws) return fail(GBM3D_EINVAL, "null pointer argument");
    if (plane_stride < (long long)(H - 1) * pitch + W)
        return fail(GBM3D_EINVAL, "plane_stride %lld: planes would overlap", plane_stride);
    const long long span = 2 * plane_stride + (long long)(H - 1) * pitch + W; // elements of the 3 planes
    if (out < noisy + span && noisy < out + span) return fail(GBM3D_EINVAL, "out must not overlap noisy");
    if (!(sigma >= 0.f) || !isfinite(sigma)) return fail(GBM3D_EINVAL, "sigma must be finite and >= 0");
    if (!aligned(ws, kAlign)) return fail(GBM3D_EINVAL, "ws must be 256-byte aligned");
    if (p->translations != 1) return fail(GBM3D_EUNSUPPORTED, "colour: translations must be 1");
    if ((st = check_stages(H, W, p))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const Sizes S = sizes(H, W, p);
    char *base = (char *)ws;
    const long long n = (long long)(align_up((size_t)H * W * sizeof(float)) / sizeof(float));
    float *zo = (float *)(base + S.total), *y1o = zo + 3 * n;
    cudaError_t e = launch_opp(noisy, pitch, plane_stride, zo, W, n, H, W, 0, s);
    if (e != cudaSuccess) return cuda_fail(e, "opponent transform");
    if ((st = run_stage_color(zo, nullptr, n, H, W, sigma, p, S, base, y1o, W, n, s))) return st;
    if (p->stages == 2) {
        // stage 2 writes the opponent planes of the result into out, then back to RGB in place
        if ((st = run_stage_color(zo, y1o, n, H, W, sigma, p, S, base, out, pitch, plane_stride, s))) return st;
        e = launch_opp(out, pitch, plane_stride, out, pitch, plane_stride, H, W, 1, s);
    } else {
        e = launch_opp(y1o, W, n, out, pitch, plane_stride, H, W, 1, s);
    }
    return e == cudaSuccess ? GBM3D_OK : cuda_fail(e, "inverse opponent transform");
}

} // extern "C"
