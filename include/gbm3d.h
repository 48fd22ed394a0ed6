/*
 * gbm3d.h -- C ABI of the GB300 (sm_103a) G-BM3D denoising hot path.
 *
 * Method: T. Sanders and S. Larkin, "New Computational Techniques for a Faster
 * Variation of BM3D Image Denoising", arXiv 2103.10765.  Stage 1 is fast block
 * matching (Sec. 2) followed by global 3-D wavelet hard thresholding of the
 * volume of matched blocks with cycle spinning and aggregation (Sec. 3,
 * Sec. 3.1); stage 2 matches again on the stage-1 estimate and applies the
 * per-group 2-D DCT + 1-D Haar empirical Wiener filter (Sec. 4).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Images are float32, row-major, H rows by W columns, with a row pitch in
 *    ELEMENTS (pitch >= W).  Internal images (pilots, outputs of
 *    gbm3d_denoise) use the caller's pitch for `out`.
 *  - Every pointer argument except `params` is a DEVICE pointer owned by the
 *    caller, unless stated otherwise.  `params` is a host pointer.
 *  - Block indices are int32 linear top-left positions k*W + l (never use the
 *    pitch for these).
 *  - Reference blocks sit on the grid G_y x G_x, G = {0, s, 2s, ...} with the
 *    last position clamped to M - N (covers the image without padding;
 *    Sec. 3.1 tiling, generalised to a stride s).  Reference g = p*Bx + q sits
 *    at (G_y[p], G_x[q]).
 *  - All calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *    default stream).  They validate every argument on the host before any
 *    launch and return a status code; on failure nothing has been launched
 *    unless the code is GBM3D_ECUDA.  gbm3d_last_error_string() describes the
 *    last failure of the calling host thread.
 *  - `ws` is caller-owned device scratch of at least gbm3d_workspace_bytes()
 *    bytes, 256-byte aligned.  No call allocates device memory (no cudaMalloc
 *    or allocating library routine).  Calls that share one `ws` must be
 *    ordered on one stream.
 *  - Supported now: patch N = 8, K1, K2 in {8, 16, 32}, levels in 1..3,
 *    cycle_spins in 1..4, translations in 1..3.  Other values return
 *    GBM3D_EUNSUPPORTED.
 */
#ifndef GBM3D_H
#define GBM3D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *gbm3d_stream_t; /* same type as cudaStream_t */

enum {
    GBM3D_OK = 0,
    GBM3D_EINVAL = 1,       /* bad argument (null pointer, size, parameter) */
    GBM3D_ENOMEM = 2,       /* scratch too small for the request */
    GBM3D_ECUDA = 3,        /* a CUDA launch or runtime call failed */
    GBM3D_ETIMEOUT = 4,     /* reserved: a bounded device-side wait gave up */
    GBM3D_EUNSUPPORTED = 5  /* valid, but not supported by the library */
};

/* Method parameters (Sec. 5 parameter list; see gbm3d_params_default). */
typedef struct {
    int patch;          /* N: block side (stage 1; both stages if patch2 = 0): */
                        /* 8 or 16                                            */
    int step;           /* s: reference-grid stride (stage 1; see step2)      */
    int search_radius;  /* R: candidates with |k-i| <= R and |l-j| <= R       */
    int k1;             /* K: blocks per group, stage 1 (Sec. 3: K = 16)      */
    int k2;             /* K: blocks per group, stage 2                       */
    int levels;         /* wavelet levels of the 3-D transform (3)            */
    int cycle_spins;    /* number of cycle spins h = 0..C-1 (2)               */
    int translations;   /* image translations h in {0, N/4, N/2}[:T]          */
    int stages;         /* 1 = stage 1 only (BM3D1), 2 = both (BM3D2)         */
    float tau_a;        /* tau_l = sigma (tau_a - tau_b l), l = 1 finest (3.6) */
    float tau_b;        /* (0.3)                                              */
    float kaiser_beta;  /* stage-2 aggregation window, 0 = no window (2.0)    */
    float eps_w;        /* lower guard on TV and Wiener weight denominators   */
    int match_engine;   /* block matching: 0 = tensor cores where supported,   */
                        /* else direct; 1 = direct FP32 SSD; 2 = tensor cores */
                        /* (EUNSUPPORTED where not).  Engines 1 and 2 give     */
                        /* the same results, bit for bit: the tensor-core     */
                        /* engine ranks with the norm expansion of Theorem 1  */
                        /* and re-ranks its certified survivors with the      */
                        /* exact direct sum.  3 = box sums shared by          */
                        /* neighbouring references (N = 8, s <= 3): exact     */
                        /* selection on FP32 distances summed in another      */
                        /* order (equal to the others up to FP32 rounding).   */
    int patch2;         /* stage-2 block side; 0 = patch.  The Wiener filter  */
                        /* is built for 8 (Sec. 5: N = 16 in stage 1, 8 in 2) */
    int step2;          /* stage-2 grid stride; 0 = step                      */
} gbm3d_params;

/* Fill *p with a preset.  preset 0: N=8, s=3 in both stages, R=19 (39x39
 * candidate offsets), K1=16, K2=32, 3 levels, 2 cycle spins, 1 translation,
 * 2 stages, tau = sigma (3.6 - 0.3 l), Kaiser beta 2, eps_w 1e-8.  preset 1
 * (the Sec. 5 parameter list): stage 1 with 16 x 16 blocks tiling the image
 * (N = s = 16), stage 2 with 8 x 8 blocks tiling it (N = s = 8), R = 16 (the
 * 32-pixel search window), K1 = K2 = 16, 3 levels, 2 cycle spins,
 * 2 translations.  Translations shift by h in {0, N/4, N/2}, N the block side
 * of the stage being averaged.  Returns GBM3D_EINVAL for other presets or
 * p == NULL. */
int gbm3d_params_default(gbm3d_params *p, int preset);

/* The parameters that the block-level calls below (grid_dims, match,
 * filter_ht, filter_wiener, aggregate) take for stage `stage` (1 or 2) of the
 * whole method: a copy of *p whose patch / step are that stage's block side
 * and stride (patch2 / step2 for stage 2 where set) and whose patch2 / step2
 * are 0.  Host-only.  EINVAL for a NULL pointer or another stage. */
int gbm3d_params_stage(const gbm3d_params *p, int stage, gbm3d_params *out);

/* Reference-grid size for an H x W image with block side p->patch and stride
 * p->step: By = |G_y|, Bx = |G_x|.  Host-only, launches nothing. */
int gbm3d_grid_dims(int H, int W, const gbm3d_params *p, int *By, int *Bx);

/* Bytes of device scratch `ws` needed by any call below for an H x W image
 * with these parameters (the maximum over the calls; gbm3d_denoise needs the
 * most).  Host-only. */
int gbm3d_workspace_bytes(int H, int W, const gbm3d_params *p, size_t *bytes);

/* Block matching (Sec. 2 eq. dfg, Theorem 1, Algorithm 1; Sec. 3.1 S^K_pq).
 * For every reference block (i,j) of the grid: exact squared distances
 * ||z^{ij} - z^{kl}||^2 (FP32, direct sum of squared differences) to every
 * candidate top-left (k,l) with |k-i| <= R, |l-j| <= R inside [0,H-N]x[0,W-N];
 * slot 0 = the reference itself, slots 1..K-1 = the K-1 nearest other blocks
 * ordered by (distance, k, l).  Blocks are N x N with N = p->patch (8 or 16)
 * on the grid of stride p->step; the tensor-core engine serves N = 8.
 *   img  : H x W image, pitch elements per row.
 *   idx  : out, int32 [By*Bx][K].
 *   dist : out, float [By*Bx][K] (nullable); slot 0 holds 0.
 *   ws   : unused (may be NULL).
 * EINVAL if the smallest search window holds fewer than K blocks. */
int gbm3d_match(const float *img, int H, int W, int pitch, const gbm3d_params *p, int K,
                int32_t *idx, float *dist, void *ws, gbm3d_stream_t stream);

/* Stage-1 global hard thresholding (Sec. 3.1 eq. BM3DHT with cycle spinning,
 * TV weights).  The volume V[pN+a, qN+b, r] = Z[k_r+a, l_r+b] (mosaic of all
 * groups, (By N) x (Bx N) x K1) is transformed as a whole by a `levels`-level
 * 3-D wavelet (bior1.5 along rows and columns, Haar along the group axis,
 * periodic, Mallat), every detail coefficient of level l is hard-thresholded
 * at sigma (tau_a - tau_b l), the transform is inverted; this is repeated for
 * cycle spins h = 0..C-1 (circular shift by h along all three axes) and
 * averaged.  N = p->patch (8 or 16), grid of stride p->step.
 *   noisy  : H x W noisy image Z, pitch elements per row.
 *   idx    : int32 [By*Bx][K1] from gbm3d_match with K = k1.
 *   groups : out, float [By*Bx][K1][N][N] = filtered blocks U.
 *   w      : out, float [By*Bx]: 1 / max(TV(u^{pq}), eps_w).
 *   ws     : scratch, gbm3d_workspace_bytes. */
int gbm3d_filter_ht(const float *noisy, int H, int W, int pitch, const int32_t *idx, float sigma,
                    const gbm3d_params *p, float *groups, float *w, void *ws, gbm3d_stream_t stream);

/* Stage-2 empirical Wiener filtering (Sec. 4).  Per group: G_z (noisy) and
 * G_y (pilot) blocks, transform T = orthonormal 8x8 DCT-II per block then
 * full-depth orthonormal Haar along the K2 blocks; omega = P^2/(P^2+sigma^2)
 * with P = T(G_y); filtered group T^-1(omega . T(G_z)); weight
 * 1 / max(sigma^2 sum omega^2, eps_w).  p->patch must be 8 (else
 * GBM3D_EUNSUPPORTED); grid of stride p->step.
 *   noisy, pilot : H x W images sharing `pitch`.
 *   idx    : int32 [By*Bx][K2] (matching done on the pilot).
 *   groups : out, float [By*Bx][K2][N][N];  w : out, float [By*Bx].
 *   ws     : unused (may be NULL). */
int gbm3d_filter_wiener(const float *noisy, const float *pilot, int H, int W, int pitch,
                        const int32_t *idx, float sigma, const gbm3d_params *p, float *groups, float *w,
                        void *ws, gbm3d_stream_t stream);

/* Aggregation (Sec. 3.1 weighted average Y = sum w U / sum w chi).  Every
 * block of every group goes back to its own position k*W + l with weight
 * w[g] (times kappa[a] kappa[b], the Kaiser window of parameter window_beta,
 * when window_beta > 0).  Each output pixel sums its contributions in a fixed
 * order with Kahan-compensated FP32 numerator and denominator, so the result
 * is deterministic.
 *   groups : float [G][K][N][N];  w : float [G];  idx : int32 [G][K], with
 *            N = p->patch and G = By*Bx of its grid (stride p->step) for H x W.
 *   out    : out, H x W, pitch elements per row.
 *   ws     : scratch, gbm3d_workspace_bytes.
 * Every pixel must be covered by some block (true for grid-reference slot 0). */
int gbm3d_aggregate(const float *groups, const float *w, const int32_t *idx, int K, int H, int W,
                    int pitch, const gbm3d_params *p, float window_beta, float *out, void *ws,
                    gbm3d_stream_t stream);

/* Aggregation exactly as gbm3d_aggregate, for callers that cannot allocate
 * device memory -- for example code running inside a host framework that owns
 * every device allocation and hands plugins a fixed budget, or a real-time
 * loop that must not allocate once it is running -- and so cannot provide
 * `ws`.  The paper has no counterpart; this is a convenience of the library.
 *   Scratch: a fixed 8 MiB array in device memory, part of the library image
 *   (every GPU that loads the library holds it until the process exits).
 *   That covers images up to about 512 x 512 with K = 32 (the CSR index needs
 *   12 (H W + 1) + 4 G K bytes); larger sizes return GBM3D_ENOMEM without
 *   launching anything.
 *   The call allocates nothing.  Its first call on a device looks up the
 *   array's device address (cudaGetSymbolAddress) and caches it for the rest
 *   of the process; make that first call before any stream capture on that
 *   device.  Resetting the device (cudaDeviceReset) after that first call is
 *   not supported: the cached address would belong to the old context.
 *   All calls on a device share the one array, and each call clears the
 *   parts it needs zeroed: calls whose executions overlap on the GPU (other
 *   streams, other host threads) race on it and must be serialised by the
 *   caller.  Arguments and result as gbm3d_aggregate. */
int gbm3d_aggregate_noalloc(const float *groups, const float *w, const int32_t *idx, int K, int H, int W,
                            int pitch, const gbm3d_params *p, float window_beta, float *out,
                            gbm3d_stream_t stream);

/* Whole method (Sec. 1.1 BM3D1/BM3D2 with translation averaging, eq.
 * firstEst): the inputs are the noisy image and the noise standard deviation
 * (Sec. 1 states the problem with just these two inputs), the output is the
 * denoised image.  Stage 1 with k1, then (stages == 2) stage 2 matching on the
 * stage-1 estimate with k2 and Wiener filtering, each stage averaged over
 * `translations` circular image shifts.
 *   noisy : H x W, pitch;  out : H x W, same pitch (must not alias noisy).
 *   ws    : scratch, gbm3d_workspace_bytes. */
int gbm3d_denoise(const float *noisy, int H, int W, int pitch, float sigma, const gbm3d_params *p,
                  float *out, void *ws, gbm3d_stream_t stream);

/* Colour denoising, an extension (the paper is grayscale only): the RGB
 * planes are mapped per pixel to opponent planes Y = (R+G+B)/3,
 * U = (R-B)/2, V = (R-2G+B)/4 (orthogonal rows: independent channel noise of
 * deviation sigma becomes sigma/sqrt(3), sigma/sqrt(2), sigma sqrt(3/8));
 * each stage matches once, on Y (stage 2: on the Y of the stage-1 estimate),
 * and filters every channel through those groups with its own sigma, weights
 * and aggregation; the result is mapped back (R = Y+U+2V/3, G = Y-4V/3,
 * B = Y-U+2V/3).  translations must be 1 (else GBM3D_EUNSUPPORTED).
 *   noisy : planes R, G, B of H x W with row pitch `pitch`; plane c starts at
 *           noisy + c * plane_stride (elements, >= (H-1) pitch + W).
 *   out   : same layout; must not overlap noisy.
 *   ws    : scratch, gbm3d_workspace_bytes_color (the grayscale workspace
 *           plus six H x W planes). */
int gbm3d_workspace_bytes_color(int H, int W, const gbm3d_params *p, size_t *bytes);
int gbm3d_denoise_color(const float *noisy, int H, int W, int pitch, long long plane_stride, float sigma,
                        const gbm3d_params *p, float *out, void *ws, gbm3d_stream_t stream);

/* Counters of the tensor-core matcher on the current device, cumulative since
 * the library was loaded:
 *   timeouts  : bounded device-side waits that gave up (0 when healthy; the
 *               tile is then re-matched by the direct engine, so results are
 *               unaffected);
 *   rematched : references whose candidate list could not be certified
 *               (near-ties wider than the error margin, non-finite pixels,
 *               a timeout) and were re-matched by the direct engine.
 * Synchronous (waits for the device's pending work).  EINVAL if a pointer is
 * NULL, ECUDA if the read fails. */
int gbm3d_match_stats(unsigned long long *timeouts, unsigned long long *rematched);

/* Measurement of the roofline's FP32 denominator (no counterpart in the
 * paper): runs FMA chains on every SM of the current device (8 CTAs of 256
 * threads per SM, 8 independent chains per thread) and returns the best of
 * three timed runs, in TFLOP/s (2 FLOP per FMA), for scalar fma.rn.f32
 * (*scalar_tflops) and packed fma.rn.f32x2 (*packed_tflops).  Synchronous
 * (waits for the runs), allocates nothing.  EINVAL for a NULL pointer, ECUDA
 * if a launch fails. */
int gbm3d_measure_fp32_peak(double *scalar_tflops, double *packed_tflops, gbm3d_stream_t stream);

/* Measurement hook.  events: NULL (off, the default) or an array of four
 * cudaEvent_t created by the caller on the current device.  While set, each
 * gbm3d_denoise on this host thread records events[0] / events[1] on its
 * stream just before / after the stage-1 block-matching launch and events[2]
 * / events[3] around the stage-2 one (with translations > 1: the last
 * translation's), so cudaEventElapsedTime gives the matching time inside a
 * real denoise.  The array must stay valid while set.  Always GBM3D_OK. */
int gbm3d_set_match_events(void *events);

/* ---- Plug-and-play ADMM deconvolution (Sec. 1: plug-and-play priors couple a
 * denoiser with inverse problems such as deconvolution, one denoiser call per
 * iteration; Sec. 6).  The paper does not state the iteration; the library runs
 * the standard scaled-dual ADMM for y = h * x + n (circular convolution with a
 * separable symmetric point-spread function h = g g^T, white noise sigma_n):
 *   x <- (H^T H + rho I)^-1 (H^T y + rho (v - u))      (exact, see below)
 *   v <- gbm3d_denoise(x + u, sigma_n / sqrt(rho))     (the data-term weight
 *                                                       lambda = sigma_n^2)
 *   u <- u + x - v
 * from v = y, u = 0; the result is v after `iters` iterations.  The x-update
 * is exact up to FP32 rounding: H^T H + rho I is diagonal in the separable
 * discrete Hartley basis, applied as dense matrix products on the tensor
 * cores with FP32-accurate results (each operand split into two tf32 parts,
 * three products accumulated in FP32; any image side that is a multiple of
 * 8).  A plan binds a batch of images of uneven
 * sizes, each with its own sigma_n, to caller buffers. */
typedef struct {
    int iters;     /* ADMM iterations (>= 1)                                   */
    float rho;     /* penalty (> 0); the denoiser runs at sigma_n / sqrt(rho)  */
    int use_graph; /* 1: one iteration of all images captured as a CUDA graph, */
                   /* one branch per image, replayed iters times; 0: the same  */
                   /* launches image after image on the caller's stream.       */
                   /* Same results, bit for bit.                               */
    int autotune;  /* 1: time the tile shapes of the x-update's products per   */
                   /* (M, N, K) at plan creation and keep the fastest (every   */
                   /* shape gives the same bits); 0: the first shape           */
} gbm3d_pnp_params;

typedef struct gbm3d_pnp_plan_st *gbm3d_pnp_plan;

/* Device scratch for a plan over n images of H[i] x W[i] (sides multiples of
 * 8) denoised with *p: per image the gbm3d_denoise workspace and six H x W
 * planes, plus the transform tables of every distinct side.  Host-only. */
int gbm3d_pnp_workspace_bytes(int n, const int *H, const int *W, const gbm3d_params *p, size_t *bytes);

/* Plan for n problems.  Host arrays of n entries: H, W; y[i] (device, the
 * blurred noisy image, row pitch ypitch[i] elements); out[i] (device, result,
 * pitch opitch[i]); sigma[i] (noise deviation sigma_n).  psf: host array of
 * the 1-D factor g of the point-spread function, odd length psf_len <= 63,
 * centred and symmetric (g[c-t] == g[c+t]); h[a][b] = g[a] g[b].  ws: device
 * scratch of ws_bytes >= gbm3d_pnp_workspace_bytes, 256-byte aligned, owned
 * by the caller and used by the plan until it is destroyed.  The call builds
 * the transform tables on `stream`, autotunes (q->autotune), synchronises the
 * stream and, with q->use_graph, captures the iteration graph (it creates
 * streams, events and the graph; no device memory).  y, out and ws are bound
 * to the plan: refill y and rerun.  EINVAL/ENOMEM/EUNSUPPORTED for bad
 * arguments (before any launch), ECUDA if a CUDA call fails. */
int gbm3d_pnp_plan_create(int n, const int *H, const int *W, const float *const *y, const int *ypitch,
                          float *const *out, const int *opitch, const float *sigma, const float *psf,
                          int psf_len, const gbm3d_params *p, const gbm3d_pnp_params *q, void *ws,
                          size_t ws_bytes, gbm3d_stream_t stream, gbm3d_pnp_plan *plan);

/* Runs the whole ADMM loop of every image of the plan on `stream`
 * (asynchronous): H^T y and the start values, `iters` iterations, v copied to
 * out.  EINVAL for a NULL plan, ECUDA on a failed launch. */
int gbm3d_pnp_run(gbm3d_pnp_plan plan, gbm3d_stream_t stream);

/* Frees the plan's host objects, streams, events and graph (not ws).  NULL
 * is accepted.  Always GBM3D_OK. */
int gbm3d_pnp_plan_destroy(gbm3d_pnp_plan plan);

/* The tile shapes (0: 128x128, 1: 128x64 outputs per CTA) the plan uses for
 * image `image`'s products with contraction length H and W. */
int gbm3d_pnp_gemm_config(gbm3d_pnp_plan plan, int image, int *cfg_k_h, int *cfg_k_w);

/* ---- Learned pilot: an extension (the paper's method has no learned part).
 * A small network imitates the stage-1 estimate (Sec. 3), which stage 2
 * (Sec. 4) then uses as its pilot.  Per pixel: input (Z, sigma); sixteen
 * zero-padded 3 x 3 convolutions 2 -> 32 -> ... -> 32 -> 1 with biases and
 * ReLU after the first fifteen (receptive field 33 x 33); pilot = Z - output;
 * training loss
 * mean (pilot - Y1)^2.  Parameters: one flat FP32 vector theta of
 * gbm3d_pilot_param_count() values, per layer the weights W[tap][ci][co]
 * (tap = 3 (dy + 1) + (dx + 1)) then the biases.  Convolutions use the
 * weights rounded to BF16 and accumulate in FP32; the hidden activations
 * (outputs of the first fifteen layers) are stored in BF16, rounded to
 * nearest-even, and the fourteen 32 -> 32 layers run on the tensor cores.
 * Batches: B images of H x W, contiguous ([B][H][W] float, device);
 * sigma: device array of B noise levels.  EINVAL for an empty or oversized
 * batch, a NULL pointer or a ws not 256-byte aligned; ECUDA if a launch
 * fails. */
int gbm3d_pilot_param_count(void);
/* Scratch of a forward pass (train = 0) or a gradient / training step (1). */
int gbm3d_pilot_workspace_bytes(int B, int H, int W, int train, size_t *bytes);
/* pilot[B][H][W] = the network's estimate for Z. */
int gbm3d_pilot_forward(const float *Z, int B, int H, int W, const float *sigma, const float *theta, float *pilot,
                        void *ws, gbm3d_stream_t stream);
/* Loss against the targets Y1 (device scalar *loss, nullable) and its
 * gradient with respect to theta (grad, nullable, gbm3d_pilot_param_count()
 * floats).  Weight gradients are summed per CTA and then in a fixed order:
 * the result is deterministic. */
int gbm3d_pilot_loss_grad(const float *Z, const float *Y1, int B, int H, int W, const float *sigma,
                          const float *theta, float *grad, float *loss, void *ws, gbm3d_stream_t stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected at step >= 1,
 * learning rate lr) on theta with moment vectors adam_m, adam_v (device,
 * zero at step 1); the loss before the step goes to *loss (nullable). */
int gbm3d_pilot_train_step(const float *Z, const float *Y1, int B, int H, int W, const float *sigma, float *theta,
                           float *adam_m, float *adam_v, int step, float lr, float *loss, void *ws,
                           gbm3d_stream_t stream);
/* Two-stage denoising with the network's estimate in place of stage 1
 * (stages 2, translations 1).  ws: gbm3d_workspace_bytes_learned. */
int gbm3d_workspace_bytes_learned(int H, int W, const gbm3d_params *p, size_t *bytes);
int gbm3d_denoise_learned(const float *noisy, int H, int W, int pitch, float sigma, const gbm3d_params *p,
                          const float *theta, float *out, void *ws, gbm3d_stream_t stream);

/* Description of the last failure on this host thread ("" if none). */
const char *gbm3d_last_error_string(void);

/* Library version string. */
const char *gbm3d_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GBM3D_H */
