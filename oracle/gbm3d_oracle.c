/*
 * gbm3d_oracle.c -- plain FP64 CPU oracle for the G-BM3D hot path
 * (Sanders & Larkin, "New Computational Techniques for a Faster Variation of
 * BM3D Image Denoising", arXiv 2103.10765).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the method computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant generator with the CUDA library, and the CUDA
 * library never calls it.
 *
 * Every value is computed in double precision.  Images come in as double
 * (callers promote FP32 images losslessly).  Loops follow the definitions in
 * the order the paper states them; no blocking, fusion or reordering beyond
 * what the definitions say.  Readings of points the paper leaves open are
 * marked "Reading:".
 *
 * Pins (checked by the CPU tests against things other than this file):
 *   grid ............ closed-form counts
 *   match ........... brute-force enumeration; Theorem 1 (Sec. 2) evaluated
 *                     through FFT cross-correlation (eq. CCF); planted copies
 *   wavelets ........ published bior1.5 taps, perfect reconstruction,
 *                     vanishing moments, Haar Parseval
 *   hard threshold .. exact-threshold case of the operator in Sec. 3.1
 *   global HT ....... independent dense-matrix evaluation on tiny volumes
 *   DCT / Haar ...... scipy's orthonormal DCT-II, Parseval, round trip
 *   Kaiser window ... numpy.kaiser
 *   aggregation ..... weighted-average invariants (constant image, sigma = 0)
 *   whole pipeline .. sigma = 0 identity, constant image, PSNR monotonicity
 * Absolute PSNR values on natural images: parity unpinned (the paper's test
 * images are not available).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

#define SQRT1_2 0.70710678118654752440
#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Periodic index, eq. (1): Z[i,j] := Z[i mod My, j mod Mx].                 */
static int pmod(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

/* ------------------------------------------------------------------------ */
/* Reference grid (Sec. 3.1 tiling of reference blocks).
 * Reading: reference stride s (s = N gives the paper's non-overlapping
 * tiling); positions 0, s, 2s, ... <= M-N, plus M-N itself when it is not on
 * that lattice, so that reference blocks cover the whole image instead of
 * mirror padding the image.  Returns the count, writes positions to out
 * (which may be NULL). */
int orc_grid(int M, int N, int s, int32_t *out)
{
    if (M < N || N <= 0 || s <= 0)
        return 0;
    int n = 0;
    int last = -1;
    for (int p = 0; p <= M - N; p += s) {
        if (out)
            out[n] = p;
        n++;
        last = p;
    }
    if (last != M - N) {
        if (out)
            out[n] = M - N;
        n++;
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Squared block distance, eq. (dfg): d(z^{ij}, z^{kl}) = ||z^{ij} - z^{kl}||^2
 * with z^{ij}[a,b] = Z[i+a, j+b] (eq. Fblock). */
static double block_dist(const double *X, int W, int i, int j, int k, int l, int N)
{
    double d = 0.0;
    for (int a = 0; a < N; a++)
        for (int b = 0; b < N; b++) {
            double t = X[(size_t)(i + a) * W + (j + b)] - X[(size_t)(k + a) * W + (l + b)];
            d += t * t;
        }
    return d;
}

double orc_patch_dist(const double *X, int H, int W, int N, int i, int j, int k, int l)
{
    (void)H;
    return block_dist(X, W, i, j, k, l, N);
}

typedef struct {
    double d;
    int k, l;
} cand_t;

/* Reading: ties in arg_K are broken by (d ascending, row ascending, column
 * ascending). */
static int cand_cmp(const void *pa, const void *pb)
{
    const cand_t *a = (const cand_t *)pa, *b = (const cand_t *)pb;
    if (a->d < b->d) return -1;
    if (a->d > b->d) return 1;
    if (a->k != b->k) return a->k < b->k ? -1 : 1;
    if (a->l != b->l) return a->l < b->l ? -1 : 1;
    return 0;
}

/* Block matching for a list of reference positions (Sec. 2, Algorithm 1;
 * Sec. 3.1 S^K_pq = arg_K min over the local search window).
 * Reading: the window holds every top-left (k,l) with |k-i| <= R, |l-j| <= R,
 * clipped to valid blocks [0,H-N] x [0,W-N] (no wrap in matching).  Slot 0 is
 * the reference block itself (Sec. 3: the first slice holds the noisy image);
 * slots 1..K-1 are the K-1 nearest other blocks in (d, k, l) order.
 * idx[t*K + r] = k*W + l; dist (nullable) gets the FP64 distances. */
int orc_match_refs(const double *X, int H, int W, int N, int R, int K,
                   const int32_t *ri, const int32_t *rj, int nrefs,
                   int32_t *idx, double *dist, int nthreads)
{
    if (!X || !ri || !rj || !idx || N <= 0 || R < 0 || K <= 0 || H < N || W < N)
        return ORC_EINVAL;
    int wy = (H - N < R ? H - N : R) + 1, wx = (W - N < R ? W - N : R) + 1;
    if ((long)wy * wx < K)
        return ORC_EINVAL;
    int maxc = (2 * R + 1) * (2 * R + 1);
    int status = ORC_OK;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        cand_t *c = (cand_t *)malloc(sizeof(cand_t) * (size_t)maxc);
        if (!c) {
#pragma omp atomic write
            status = ORC_ENOMEM;
        }
#pragma omp for schedule(dynamic, 8)
        for (int t = 0; t < nrefs; t++) {
            if (!c) continue;
            int i = ri[t], j = rj[t];
            int k0 = i - R < 0 ? 0 : i - R, k1 = i + R > H - N ? H - N : i + R;
            int l0 = j - R < 0 ? 0 : j - R, l1 = j + R > W - N ? W - N : j + R;
            int n = 0;
            for (int k = k0; k <= k1; k++)
                for (int l = l0; l <= l1; l++) {
                    if (k == i && l == j) continue;
                    c[n].d = block_dist(X, W, i, j, k, l, N);
                    c[n].k = k;
                    c[n].l = l;
                    n++;
                }
            qsort(c, (size_t)n, sizeof(cand_t), cand_cmp);
            idx[(size_t)t * K] = i * W + j;
            if (dist) dist[(size_t)t * K] = 0.0;
            for (int r = 1; r < K; r++) {
                idx[(size_t)t * K + r] = c[r - 1].k * W + c[r - 1].l;
                if (dist) dist[(size_t)t * K + r] = c[r - 1].d;
            }
        }
        free(c);
    }
    return status;
}

/* Matching for every reference block of the grid, refs in row-major (p,q). */
int orc_match(const double *X, int H, int W, int N, int s, int R, int K,
              int32_t *idx, double *dist, int nthreads)
{
    int By = orc_grid(H, N, s, NULL), Bx = orc_grid(W, N, s, NULL);
    if (By <= 0 || Bx <= 0) return ORC_EINVAL;
    int32_t *gy = malloc(sizeof(int32_t) * By), *gx = malloc(sizeof(int32_t) * Bx);
    int32_t *ri = malloc(sizeof(int32_t) * (size_t)By * Bx), *rj = malloc(sizeof(int32_t) * (size_t)By * Bx);
    int st = ORC_ENOMEM;
    if (gy && gx && ri && rj) {
        orc_grid(H, N, s, gy);
        orc_grid(W, N, s, gx);
        for (int p = 0; p < By; p++)
            for (int q = 0; q < Bx; q++) {
                ri[p * Bx + q] = gy[p];
                rj[p * Bx + q] = gx[q];
            }
        st = orc_match_refs(X, H, W, N, R, K, ri, rj, By * Bx, idx, dist, nthreads);
    }
    free(gy); free(gx); free(ri); free(rj);
    return st;
}

/* ------------------------------------------------------------------------ */
/* One-dimensional periodic wavelet filter banks (Sec. 5 parameter list:
 * biorthogonal 1.5 in the two spatial dimensions, Haar along the group).
 *
 * bior1.5 analysis low-pass (the Cohen-Daubechies-Feauveau spline pair with
 * one vanishing moment on the synthesis side and five on the analysis side):
 *   h0 = [3, -3, -22, 22, 128, 128, 22, -22, -3, 3] / (128 sqrt 2)
 * applied as lo[m] = sum_t h0[t] x[2m - 4 + t]; analysis high-pass is the Haar
 * difference hi[m] = (x[2m] - x[2m+1]) / sqrt 2.  Synthesis: low-pass is the
 * Haar pair (1, 1)/sqrt 2 at 2m, 2m+1, high-pass is
 *   g1 = [3, 3, -22, -22, 128, -128, 22, 22, -3, -3] / (128 sqrt 2)
 * placed at 2m - 4 .. 2m + 5 (the unique inverse of the analysis pair).
 * Reading: periodic extension (eq. (1)); phase chosen so that each low-pass
 * output is centred on its input pair. */
#define WAV_HAAR 0
#define WAV_BIOR15 1

static const double H0_INT[10] = {3, -3, -22, 22, 128, 128, 22, -22, -3, 3};
static const double G1_INT[10] = {3, 3, -22, -22, 128, -128, 22, 22, -3, -3};

void orc_bior15_filters(double *h0, double *g1)
{
    for (int t = 0; t < 10; t++) {
        if (h0) h0[t] = H0_INT[t] / (128.0 * sqrt(2.0));
        if (g1) g1[t] = G1_INT[t] / (128.0 * sqrt(2.0));
    }
}

/* x has n (even) samples at stride xs; lo/hi get n/2 samples at stride os. */
static void ana1(const double *x, int n, int xs, int kind, double *lo, double *hi, int os)
{
    double h0[10];
    orc_bior15_filters(h0, NULL);
    for (int m = 0; m < n / 2; m++) {
        hi[m * os] = (x[(2 * m) * xs] - x[(2 * m + 1) * xs]) * SQRT1_2;
        if (kind == WAV_HAAR) {
            lo[m * os] = (x[(2 * m) * xs] + x[(2 * m + 1) * xs]) * SQRT1_2;
        } else {
            double s = 0.0;
            for (int t = 0; t < 10; t++)
                s += h0[t] * x[pmod(2 * m - 4 + t, n) * xs];
            lo[m * os] = s;
        }
    }
}

static void syn1(const double *lo, const double *hi, int is, int n, int kind, double *x, int xs)
{
    double g1[10];
    orc_bior15_filters(NULL, g1);
    for (int t = 0; t < n; t++) x[t * xs] = 0.0;
    for (int m = 0; m < n / 2; m++) {
        x[(2 * m) * xs] += SQRT1_2 * lo[m * is];
        x[(2 * m + 1) * xs] += SQRT1_2 * lo[m * is];
        if (kind == WAV_HAAR) {
            x[(2 * m) * xs] += SQRT1_2 * hi[m * is];
            x[(2 * m + 1) * xs] -= SQRT1_2 * hi[m * is];
        } else {
            for (int t = 0; t < 10; t++)
                x[pmod(2 * m - 4 + t, n) * xs] += g1[t] * hi[m * is];
        }
    }
}

/* Exported 1-D single-level transforms (for the wavelet pins). */
int orc_dwt1(const double *x, int n, int kind, double *lo, double *hi)
{
    if (n < 2 || (n & 1)) return ORC_EINVAL;
    ana1(x, n, 1, kind, lo, hi, 1);
    return ORC_OK;
}

int orc_idwt1(const double *lo, const double *hi, int n, int kind, double *x)
{
    if (n < 2 || (n & 1)) return ORC_EINVAL;
    syn1(lo, hi, 1, n, kind, x, 1);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* 3-D wavelet transform T_3D of a volume v[y][x][z] (dims Y, X, Z), levels L,
 * in place, Mallat layout (eq. BM3DHT: T_3D; Sec. 5: 3 levels).
 * Reading: Mallat 3-D decomposition -- each level splits the current
 * approximation cube along y and x (bior1.5) and z (Haar); the next level
 * recurses on the low-low-low cube. */
static int lines(double *v, int Y, int X, int Z, int h, int w, int k, int axis, int kind, int inverse, int nt)
{
    /* Applies the 1-D transform to every line along `axis` inside the
     * sub-cube [0,h) x [0,w) x [0,k).  Lines are independent: with nt > 1
     * they are shared among threads, each line still transformed by the
     * same operations in the same order. */
    int n = axis == 0 ? h : axis == 1 ? w : k;
    int stride = axis == 0 ? X * Z : axis == 1 ? Z : 1;
    int c1 = axis == 0 ? w : h, c2 = axis == 2 ? w : k;
    int failed = 0;
#pragma omp parallel num_threads(nt > 0 ? nt : 1)
    {
        double *buf_in = malloc(sizeof(double) * n), *buf_out = malloc(sizeof(double) * n);
        if (!buf_in || !buf_out) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for collapse(2) schedule(static)
        for (int u = 0; u < c1; u++)
            for (int t = 0; t < c2; t++) {
                if (!buf_in || !buf_out) continue;
                size_t base;
                if (axis == 0) base = (size_t)u * Z + t;                  /* (x=u, z=t) */
                else if (axis == 1) base = (size_t)u * X * Z + t;         /* (y=u, z=t) */
                else base = (size_t)u * X * Z + (size_t)t * Z;            /* (y=u, x=t) */
                for (int e = 0; e < n; e++) buf_in[e] = v[base + (size_t)e * stride];
                if (!inverse) {
                    ana1(buf_in, n, 1, kind, buf_out, buf_out + n / 2, 1);
                } else {
                    syn1(buf_in, buf_in + n / 2, 1, n, kind, buf_out, 1);
                }
                for (int e = 0; e < n; e++) v[base + (size_t)e * stride] = buf_out[e];
            }
        free(buf_in);
        free(buf_out);
    }
    (void)Y;
    return failed ? ORC_ENOMEM : ORC_OK;
}

/* Hard threshold Upsilon (Sec. 3.1): keep alpha if |alpha| >= lambda. */
static double upsilon(double a, double lam)
{
    return fabs(a) >= lam ? a : 0.0;
}

double orc_upsilon(double a, double lam) { return upsilon(a, lam); }

/* Forward transform, then (if tau != NULL) hard thresholding of every detail
 * coefficient of level l (1 = finest) with tau[l-1]; the final approximation
 * cube is kept.  Reading: all seven detail bands of each level are
 * thresholded; the coarsest approximation is not. */
static int dwt3_forward(double *v, int Y, int X, int Z, int L, const double *tau, int nt)
{
    int h = Y, w = X, k = Z, st = ORC_OK;
    for (int lev = 1; lev <= L && st == ORC_OK; lev++) {
        st = lines(v, Y, X, Z, h, w, k, 0, WAV_BIOR15, 0, nt);
        if (st == ORC_OK) st = lines(v, Y, X, Z, h, w, k, 1, WAV_BIOR15, 0, nt);
        if (st == ORC_OK) st = lines(v, Y, X, Z, h, w, k, 2, WAV_HAAR, 0, nt);
        if (tau && st == ORC_OK) {
#pragma omp parallel for num_threads(nt > 0 ? nt : 1) schedule(static)
            for (int y = 0; y < h; y++)
                for (int x = 0; x < w; x++)
                    for (int z = 0; z < k; z++)
                        if (y >= h / 2 || x >= w / 2 || z >= k / 2) {
                            size_t o = ((size_t)y * X + x) * Z + z;
                            v[o] = upsilon(v[o], tau[lev - 1]);
                        }
        }
        h /= 2; w /= 2; k /= 2;
    }
    return st;
}

static int dwt3_inverse(double *v, int Y, int X, int Z, int L, int nt)
{
    int st = ORC_OK;
    for (int lev = L; lev >= 1 && st == ORC_OK; lev--) {
        int h = Y >> (lev - 1), w = X >> (lev - 1), k = Z >> (lev - 1);
        st = lines(v, Y, X, Z, h, w, k, 2, WAV_HAAR, 1, nt);
        if (st == ORC_OK) st = lines(v, Y, X, Z, h, w, k, 1, WAV_BIOR15, 1, nt);
        if (st == ORC_OK) st = lines(v, Y, X, Z, h, w, k, 0, WAV_BIOR15, 1, nt);
    }
    return st;
}

static int dims_ok(int Y, int X, int Z, int L)
{
    int d = 1 << L;
    return L >= 1 && Y > 0 && X > 0 && Z > 0 && Y % d == 0 && X % d == 0 && Z % d == 0;
}

/* Exported: forward (optionally thresholded) and inverse 3-D transforms. */
int orc_dwt3(double *v, int Y, int X, int Z, int L, const double *tau, int nthreads)
{
    if (!v || !dims_ok(Y, X, Z, L)) return ORC_EINVAL;
    return dwt3_forward(v, Y, X, Z, L, tau, nthreads > 0 ? nthreads : 1);
}

int orc_idwt3(double *v, int Y, int X, int Z, int L, int nthreads)
{
    if (!v || !dims_ok(Y, X, Z, L)) return ORC_EINVAL;
    return dwt3_inverse(v, Y, X, Z, L, nthreads > 0 ? nthreads : 1);
}

/* w = 1 / max(TV(u), eps_w) for one filtered group u[r][a][b] (N x N x K):
 * TV is the sum of |forward differences| along a, b and r inside the
 * group, without wrap (Sec. 3.1; reading: anisotropic L1). */
static double tv_weight(const double *o, int N, int K, double eps_w)
{
    double tv = 0.0;
    for (int r = 0; r < K; r++)
        for (int a = 0; a < N; a++)
            for (int b = 0; b < N; b++) {
                double c = o[(r * N + a) * N + b];
                if (a + 1 < N) tv += fabs(o[(r * N + a + 1) * N + b] - c);
                if (b + 1 < N) tv += fabs(o[(r * N + a) * N + b + 1] - c);
                if (r + 1 < K) tv += fabs(o[((r + 1) * N + a) * N + b] - c);
            }
    return 1.0 / (tv > eps_w ? tv : eps_w);
}

/* ------------------------------------------------------------------------ */
/* Stage 1: global volume hard thresholding (Sec. 3, Sec. 3.1).
 *
 * V[pN+a, qN+b, r] = z^{ij}[a,b] for the r-th block [i,j] of S^K_pq.
 * Reading (reference stride s < N): the volume is the mosaic of groups, with
 * group (p,q) at spatial tile (pN, qN); its dims are (By N) x (Bx N) x K.
 * For s = N this is the paper's image-sized volume.
 *
 * U_h = S_{-h} T3D^-1 Upsilon T3D S_h V for h = 0..C-1 (cycle spinning), with
 * S_h the circular shift by h along every axis: (S_h V)[y,x,z] =
 * V[y-h, x-h, z-h].  U = (1/C) sum_h U_h.
 * Thresholds per level l = 1..L: tau_l = sigma (tau_a - tau_b l) (Sec. 5).
 * Weights w_pq = 1 / TV(u^{pq}); reading: anisotropic L1 total variation of
 * forward differences inside the N x N x K block (no wrap), guarded below by
 * eps_w.
 * Outputs groups[g][r][a][b] = U[pN+a, qN+b, r] and w[g], g = p*Bx + q.
 * nthreads: threads that share the independent lines of each 1-D transform
 * and the independent planes of the volume copies (same arithmetic). */
int orc_filter_ht(const double *Z, int H, int W, const int32_t *idx, int By, int Bx,
                  int N, int K, double sigma, int L, int C, double tau_a, double tau_b,
                  double eps_w, double *groups, double *w, int nthreads)
{
    const int nt = nthreads > 0 ? nthreads : 1;
    if (!Z || !idx || !groups || !w || By <= 0 || Bx <= 0 || C <= 0 || sigma < 0) return ORC_EINVAL;
    int Yd = By * N, Xd = Bx * N, Zd = K;
    if (!dims_ok(Yd, Xd, Zd, L)) return ORC_EINVAL;
    size_t nv = (size_t)Yd * Xd * Zd;
    double *V = malloc(sizeof(double) * nv), *S = malloc(sizeof(double) * nv);
    double *U = calloc(nv, sizeof(double));
    double *tau = malloc(sizeof(double) * L);
    if (!V || !S || !U || !tau) { free(V); free(S); free(U); free(tau); return ORC_ENOMEM; }
    for (int l = 1; l <= L; l++) tau[l - 1] = sigma * (tau_a - tau_b * l);

    for (int p = 0; p < By; p++)
        for (int q = 0; q < Bx; q++)
            for (int r = 0; r < K; r++) {
                int v = idx[((size_t)p * Bx + q) * K + r];
                int i = v / W, j = v % W;
                for (int a = 0; a < N; a++)
                    for (int b = 0; b < N; b++)
                        V[((size_t)(p * N + a) * Xd + (q * N + b)) * Zd + r] = Z[(size_t)(i + a) * W + (j + b)];
            }

    int st = ORC_OK;
    for (int h = 0; h < C && st == ORC_OK; h++) {
#pragma omp parallel for num_threads(nt) schedule(static)
        for (int y = 0; y < Yd; y++)
            for (int x = 0; x < Xd; x++)
                for (int z = 0; z < Zd; z++)
                    S[((size_t)y * Xd + x) * Zd + z] =
                        V[((size_t)pmod(y - h, Yd) * Xd + pmod(x - h, Xd)) * Zd + pmod(z - h, Zd)];
        st = dwt3_forward(S, Yd, Xd, Zd, L, tau, nt);
        if (st == ORC_OK) st = dwt3_inverse(S, Yd, Xd, Zd, L, nt);
#pragma omp parallel for num_threads(nt) schedule(static)
        for (int y = 0; y < Yd; y++)
            for (int x = 0; x < Xd; x++)
                for (int z = 0; z < Zd; z++)
                    U[((size_t)y * Xd + x) * Zd + z] +=
                        S[((size_t)pmod(y + h, Yd) * Xd + pmod(x + h, Xd)) * Zd + pmod(z + h, Zd)] / C;
    }

    for (int p = 0; p < By && st == ORC_OK; p++)
        for (int q = 0; q < Bx; q++) {
            size_t g = (size_t)p * Bx + q;
            double *o = groups + g * K * N * N;
            for (int r = 0; r < K; r++)
                for (int a = 0; a < N; a++)
                    for (int b = 0; b < N; b++)
                        o[(r * N + a) * N + b] = U[((size_t)(p * N + a) * Xd + (q * N + b)) * Zd + r];
            w[g] = tv_weight(o, N, K, eps_w);
        }
    free(V); free(S); free(U); free(tau);
    return st;
}

/* Exported: the weights w[g] = 1 / max(TV(u^g), eps_w) of G filtered groups
 * groups[g][r][a][b] (the rule orc_filter_ht applies). */
int orc_tv_weights(const double *groups, int G, int K, int N, double eps_w, double *w)
{
    if (!groups || !w || G <= 0 || K <= 0 || N <= 0) return ORC_EINVAL;
    for (int g = 0; g < G; g++) w[g] = tv_weight(groups + (size_t)g * K * N * N, N, K, eps_w);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Stage 2 transforms (Sec. 4): 2-D DCT in the block plane, 1-D Haar along the
 * group.  Reading: orthonormal DCT-II
 *   X[u] = alpha(u) sum_n x[n] cos(pi (2n+1) u / (2N)),
 *   alpha(0) = sqrt(1/N), alpha(u>0) = sqrt(2/N),
 * and a full-depth orthonormal Haar transform along the K blocks. */
static void dct1(const double *x, int n, int xs, double *out, int os)
{
    for (int u = 0; u < n; u++) {
        double s = 0.0;
        for (int t = 0; t < n; t++) s += x[t * xs] * cos(ORC_PI * (2 * t + 1) * u / (2.0 * n));
        out[u * os] = s * (u == 0 ? sqrt(1.0 / n) : sqrt(2.0 / n));
    }
}

static void idct1(const double *X, int n, int xs, double *out, int os)
{
    for (int t = 0; t < n; t++) {
        double s = 0.0;
        for (int u = 0; u < n; u++)
            s += (u == 0 ? sqrt(1.0 / n) : sqrt(2.0 / n)) * X[u * xs] * cos(ORC_PI * (2 * t + 1) * u / (2.0 * n));
        out[t * os] = s;
    }
}

/* 2-D DCT of an N x N block in place (rows then columns). */
static void dct2(double *blk, int N, int inverse)
{
    double tmp[64 * 64];
    double line[64];
    for (int a = 0; a < N; a++) {
        if (!inverse) dct1(blk + a * N, N, 1, line, 1); else idct1(blk + a * N, N, 1, line, 1);
        for (int b = 0; b < N; b++) tmp[a * N + b] = line[b];
    }
    for (int b = 0; b < N; b++) {
        if (!inverse) dct1(tmp + b, N, N, line, 1); else idct1(tmp + b, N, N, line, 1);
        for (int a = 0; a < N; a++) blk[a * N + b] = line[a];
    }
}

int orc_dct2(double *blk, int N, int inverse)
{
    if (!blk || N <= 0 || N > 64) return ORC_EINVAL;
    dct2(blk, N, inverse);
    return ORC_OK;
}

/* Full-depth orthonormal Haar on x[0..n) at stride xs (n a power of two). */
static void haar_full(double *x, int n, int xs, int inverse)
{
    double t[1024];
    if (!inverse) {
        for (int len = n; len >= 2; len /= 2) {
            for (int m = 0; m < len / 2; m++) {
                t[m] = (x[(2 * m) * xs] + x[(2 * m + 1) * xs]) * SQRT1_2;
                t[len / 2 + m] = (x[(2 * m) * xs] - x[(2 * m + 1) * xs]) * SQRT1_2;
            }
            for (int m = 0; m < len; m++) x[m * xs] = t[m];
        }
    } else {
        for (int len = 2; len <= n; len *= 2) {
            for (int m = 0; m < len / 2; m++) {
                double lo = x[m * xs], hi = x[(len / 2 + m) * xs];
                t[2 * m] = (lo + hi) * SQRT1_2;
                t[2 * m + 1] = (lo - hi) * SQRT1_2;
            }
            for (int m = 0; m < len; m++) x[m * xs] = t[m];
        }
    }
}

int orc_haar(double *x, int n, int inverse)
{
    if (!x || n < 1 || n > 1024 || (n & (n - 1))) return ORC_EINVAL;
    haar_full(x, n, 1, inverse);
    return ORC_OK;
}

/* T applied to a whole group g[r][a][b] (K x N x N). */
static void group_transform(double *g, int K, int N, int inverse)
{
    if (!inverse) {
        for (int r = 0; r < K; r++) dct2(g + (size_t)r * N * N, N, 0);
        for (int e = 0; e < N * N; e++) haar_full(g + e, K, N * N, 0);
    } else {
        for (int e = 0; e < N * N; e++) haar_full(g + e, K, N * N, 1);
        for (int r = 0; r < K; r++) dct2(g + (size_t)r * N * N, N, 1);
    }
}

/* Stage 2 empirical Wiener filtering of every group (Sec. 4).
 * Reading (the paper defers to the original BM3D rules): with P = T(G_pilot),
 * shrinkage omega = P^2 / (P^2 + sigma^2) (0 where that denominator is 0),
 * filtered group T^-1(omega . T(G_noisy)), group weight
 * w = 1 / max(sigma^2 sum omega^2, eps_w). */
int orc_filter_wiener(const double *Z, const double *Yp, int H, int W, const int32_t *idx, int G,
                      int N, int K, double sigma, double eps_w, double *groups, double *w, int nthreads)
{
    if (!Z || !Yp || !idx || !groups || !w || G <= 0 || N <= 0 || N > 64 || K <= 0 || K > 1024 ||
        (K & (K - 1)) || sigma < 0)
        return ORC_EINVAL;
    (void)H;
    int status = ORC_OK;
    size_t gs = (size_t)K * N * N;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        double *P = malloc(sizeof(double) * gs), *Q = malloc(sizeof(double) * gs);
        if (!P || !Q) {
#pragma omp atomic write
            status = ORC_ENOMEM;
        }
#pragma omp for schedule(dynamic, 16)
        for (int g = 0; g < G; g++) {
            if (!P || !Q) continue;
            for (int r = 0; r < K; r++) {
                int v = idx[(size_t)g * K + r];
                int i = v / W, j = v % W;
                for (int a = 0; a < N; a++)
                    for (int b = 0; b < N; b++) {
                        P[((size_t)r * N + a) * N + b] = Yp[(size_t)(i + a) * W + (j + b)];
                        Q[((size_t)r * N + a) * N + b] = Z[(size_t)(i + a) * W + (j + b)];
                    }
            }
            group_transform(P, K, N, 0);
            group_transform(Q, K, N, 0);
            double s2 = sigma * sigma, sw = 0.0;
            for (size_t e = 0; e < gs; e++) {
                double p2 = P[e] * P[e];
                double om = (p2 + s2) > 0.0 ? p2 / (p2 + s2) : 0.0;
                Q[e] *= om;
                sw += om * om;
            }
            group_transform(Q, K, N, 1);
            memcpy(groups + (size_t)g * gs, Q, sizeof(double) * gs);
            double den = s2 * sw;
            w[g] = 1.0 / (den > eps_w ? den : eps_w);
        }
        free(P); free(Q);
    }
    return status;
}

/* ------------------------------------------------------------------------ */
/* Kaiser window for the stage-2 aggregation (Sec. 4 defers to the original
 * BM3D aggregation rules).  Reading: kappa[n] = I0(beta sqrt(1 - (2n/(N-1) -
 * 1)^2)) / I0(beta), with I0 the modified Bessel function of the first kind,
 * order 0, summed from its power series sum_k ((x/2)^k / k!)^2. */
double orc_bessel_i0(double x)
{
    double s = 1.0, t = 1.0;
    for (int k = 1; k < 200; k++) {
        t *= (x / 2.0) / k;
        s += t * t;
        if (t * t < 1e-300) break;
    }
    return s;
}

int orc_kaiser(int N, double beta, double *out)
{
    if (!out || N <= 0) return ORC_EINVAL;
    for (int n = 0; n < N; n++) {
        if (beta <= 0.0 || N == 1) { out[n] = 1.0; continue; }
        double r = 2.0 * n / (N - 1) - 1.0;
        double arg = 1.0 - r * r;
        out[n] = orc_bessel_i0(beta * sqrt(arg > 0 ? arg : 0.0)) / orc_bessel_i0(beta);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Aggregation (Sec. 3.1): Y = sum w_pq U^{pq}_{ij} / sum w_pq chi_{ij}, each
 * filtered block put back at the position of the block it came from.  With a
 * window (stage 2, beta > 0) every block value and its support are also
 * multiplied by kappa[a] kappa[b]. */
int orc_aggregate(const double *groups, const double *w, const int32_t *idx, int G, int K,
                  int H, int W, int N, double beta, double *out, int require_cover)
{
    if (!groups || !w || !idx || !out || G <= 0 || K <= 0 || H < N || W < N || N <= 0 || N > 64)
        return ORC_EINVAL;
    double kap[64];
    orc_kaiser(N, beta, kap);
    double *num = calloc((size_t)H * W, sizeof(double)), *den = calloc((size_t)H * W, sizeof(double));
    if (!num || !den) { free(num); free(den); return ORC_ENOMEM; }
    for (int g = 0; g < G; g++)
        for (int r = 0; r < K; r++) {
            int v = idx[(size_t)g * K + r];
            int i = v / W, j = v % W;
            const double *u = groups + ((size_t)g * K + r) * N * N;
            for (int a = 0; a < N; a++)
                for (int b = 0; b < N; b++) {
                    double wt = w[g] * kap[a] * kap[b];
                    num[(size_t)(i + a) * W + (j + b)] += wt * u[a * N + b];
                    den[(size_t)(i + a) * W + (j + b)] += wt;
                }
        }
    int st = ORC_OK;
    for (size_t e = 0; e < (size_t)H * W; e++) {
        if (den[e] > 0.0) out[e] = num[e] / den[e];
        else { out[e] = 0.0; if (require_cover) st = ORC_EINVAL; } /* a pixel no block covers */
    }
    free(num); free(den);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Whole method: Y1 = G-BM3D stage 1, Y2 = stage 2 (Sec. 1.1 BM3D1 / BM3D2),
 * each averaged over image translations (eq. firstEst):
 *   Y_f = (1/T) sum_h S_{-h}(phi(S_h Z)),  h in {0, N/4, N/2}[:T],
 * with S_h the circular 2-D shift (S_h Z)[y,x] = Z[y-h, x-h].
 * Reading: stage 2 matches on the stage-1 estimate (Sec. 1.1) and filters the
 * noisy image with the stage-1 estimate as pilot (Sec. 4); both images are
 * translated together. */
/* patch / step: block side N and grid stride of stage 1; patch2 / step2 those
 * of stage 2 (0 = the stage-1 value).  Sec. 5 uses N = 16 in stage 1 and
 * N = 8 in stage 2, each grid tiling the image (s = N). */
typedef struct {
    int patch, step, search_radius, k1, k2, levels, cycle_spins, translations, stages;
    double tau_a, tau_b, kaiser_beta, eps_w;
    int patch2, step2;
} orc_params;

static int stage_patch(const orc_params *p, int stage)
{
    return (stage == 2 && p->patch2 > 0) ? p->patch2 : p->patch;
}

static int stage_step(const orc_params *p, int stage)
{
    return (stage == 2 && p->step2 > 0) ? p->step2 : p->step;
}

/* Reading: the translations h in {0, N/4, N/2} of eq. firstEst use the block
 * side N of the stage they wrap (stage 2 repeats the strategy "just as in the
 * first step", Sec. 4, with its own N). */
static void stage_shifts(const orc_params *p, int stage, int hs[3])
{
    const int N = stage_patch(p, stage);
    hs[0] = 0;
    hs[1] = N / 4;
    hs[2] = N / 2;
}

static void shift2(const double *src, double *dst, int H, int W, int h)
{
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++)
            dst[(size_t)y * W + x] = src[(size_t)pmod(y - h, H) * W + pmod(x - h, W)];
}

static int stage1(const double *Z, int H, int W, double sigma, const orc_params *p, double *out, int nt)
{
    int N = p->patch, K = p->k1;
    int By = orc_grid(H, N, p->step, NULL), Bx = orc_grid(W, N, p->step, NULL);
    size_t G = (size_t)By * Bx;
    int32_t *idx = malloc(sizeof(int32_t) * G * K);
    double *gr = malloc(sizeof(double) * G * K * N * N), *w = malloc(sizeof(double) * G);
    int st = ORC_ENOMEM;
    if (idx && gr && w) {
        st = orc_match(Z, H, W, N, p->step, p->search_radius, K, idx, NULL, nt);
        if (st == ORC_OK)
            st = orc_filter_ht(Z, H, W, idx, By, Bx, N, K, sigma, p->levels, p->cycle_spins, p->tau_a,
                               p->tau_b, p->eps_w, gr, w, nt);
        if (st == ORC_OK) st = orc_aggregate(gr, w, idx, (int)G, K, H, W, N, 0.0, out, 1);
    }
    free(idx); free(gr); free(w);
    return st;
}

static int stage2(const double *Z, const double *Y1, int H, int W, double sigma, const orc_params *p,
                  double *out, int nt)
{
    int N = stage_patch(p, 2), K = p->k2, s = stage_step(p, 2);
    int By = orc_grid(H, N, s, NULL), Bx = orc_grid(W, N, s, NULL);
    size_t G = (size_t)By * Bx;
    int32_t *idx = malloc(sizeof(int32_t) * G * K);
    double *gr = malloc(sizeof(double) * G * K * N * N), *w = malloc(sizeof(double) * G);
    int st = ORC_ENOMEM;
    if (idx && gr && w) {
        st = orc_match(Y1, H, W, N, s, p->search_radius, K, idx, NULL, nt);
        if (st == ORC_OK) st = orc_filter_wiener(Z, Y1, H, W, idx, (int)G, N, K, sigma, p->eps_w, gr, w, nt);
        if (st == ORC_OK) st = orc_aggregate(gr, w, idx, (int)G, K, H, W, N, p->kaiser_beta, out, 1);
    }
    free(idx); free(gr); free(w);
    return st;
}

int orc_denoise(const double *Z, int H, int W, double sigma, const orc_params *p, double *out,
                double *y1_out, int nthreads)
{
    if (!Z || !p || !out || H < p->patch || W < p->patch || H < stage_patch(p, 2) || W < stage_patch(p, 2) ||
        p->translations < 1 || p->translations > 3 || p->stages < 1 || p->stages > 2 || sigma < 0)
        return ORC_EINVAL;
    size_t n = (size_t)H * W;
    int hs[3], hs2[3];
    stage_shifts(p, 1, hs);
    stage_shifts(p, 2, hs2);
    double *zs = malloc(sizeof(double) * n), *ys = malloc(sizeof(double) * n);
    double *o = malloc(sizeof(double) * n), *y1 = calloc(n, sizeof(double));
    int st = (zs && ys && o && y1) ? ORC_OK : ORC_ENOMEM;
    for (int t = 0; t < p->translations && st == ORC_OK; t++) {
        shift2(Z, zs, H, W, hs[t]);
        st = stage1(zs, H, W, sigma, p, o, nthreads);
        shift2(o, ys, H, W, -hs[t]);
        for (size_t e = 0; e < n; e++) y1[e] += ys[e] / p->translations;
    }
    if (st == ORC_OK && y1_out) memcpy(y1_out, y1, sizeof(double) * n);
    if (st == ORC_OK && p->stages == 1) memcpy(out, y1, sizeof(double) * n);
    if (st == ORC_OK && p->stages == 2) {
        double *y2 = calloc(n, sizeof(double)), *y1s = malloc(sizeof(double) * n);
        if (!y2 || !y1s) st = ORC_ENOMEM;
        for (int t = 0; t < p->translations && st == ORC_OK; t++) {
            shift2(Z, zs, H, W, hs2[t]);
            shift2(y1, y1s, H, W, hs2[t]);
            st = stage2(zs, y1s, H, W, sigma, p, o, nthreads);
            shift2(o, ys, H, W, -hs2[t]);
            for (size_t e = 0; e < n; e++) y2[e] += ys[e] / p->translations;
        }
        if (st == ORC_OK) memcpy(out, y2, sizeof(double) * n);
        free(y2); free(y1s);
    }
    free(zs); free(ys); free(o); free(y1);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Colour extension.  The paper is grayscale only; this is the usual colour
 * use of BM3D (reading C1-C4):
 *   C1 opponent transform per pixel: Y = (R+G+B)/3, U = (R-B)/2,
 *      V = (R-2G+B)/4 (rows orthogonal, so independent channel noise stays
 *      independent), inverse R = Y+U+2V/3, G = Y-4V/3, B = Y-U+2V/3;
 *   C2 channel c carries noise sigma_c = sigma |row_c| (sigma/sqrt3,
 *      sigma/sqrt2, sigma sqrt(3/8)) for i.i.d. noise of deviation sigma in
 *      R, G, B;
 *   C3 each stage matches once, on Y (stage 2: on the Y of the stage-1
 *      estimate), and every channel is filtered through those groups with
 *      its own sigma_c, its own weights and its own aggregation;
 *   C4 translations as in orc_denoise, applied to all channels together. */
static const double ORC_OPP_F[3][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3}, {0.5, 0.0, -0.5}, {0.25, -0.5, 0.25}};
static const double ORC_OPP_I[3][3] = {{1.0, 1.0, 2.0 / 3}, {1.0, 0.0, -4.0 / 3}, {1.0, -1.0, 2.0 / 3}};

/* x (3 planes of n values, plane c at x + c n) -> y = M x per pixel
 * (inverse = 0: forward opponent transform, 1: its inverse). */
int orc_opp(const double *x, size_t n, int inverse, double *y)
{
    if (!x || !y) return ORC_EINVAL;
    const double (*M)[3] = inverse ? ORC_OPP_I : ORC_OPP_F;
    for (size_t e = 0; e < n; e++) {
        const double a = x[e], b = x[n + e], c = x[2 * n + e];
        for (int r = 0; r < 3; r++) y[r * n + e] = M[r][0] * a + M[r][1] * b + M[r][2] * c;
    }
    return ORC_OK;
}

/* sigma_c / sigma = |row c of the forward transform| (reading C2). */
double orc_opp_sigma_scale(int c)
{
    if (c < 0 || c > 2) return 0.0;
    const double *r = ORC_OPP_F[c];
    return sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
}

/* One colour stage on (possibly shifted) opponent planes Zo: matching on the
 * guide plane (Zo[0] in stage 1, Y1o[0] in stage 2), then per channel the
 * stage's filter and aggregation into out (3 planes). */
static int stage_color(const double *Zo, const double *Y1o, int H, int W, double sigma, const orc_params *p,
                       double *out, int nt)
{
    const int sg = Y1o ? 2 : 1;
    const int N = stage_patch(p, sg), K = Y1o ? p->k2 : p->k1, s = stage_step(p, sg);
    const int By = orc_grid(H, N, s, NULL), Bx = orc_grid(W, N, s, NULL);
    const size_t G = (size_t)By * Bx, n = (size_t)H * W;
    int32_t *idx = malloc(sizeof(int32_t) * G * K);
    double *gr = malloc(sizeof(double) * G * K * N * N), *w = malloc(sizeof(double) * G);
    int st = (idx && gr && w) ? ORC_OK : ORC_ENOMEM;
    if (st == ORC_OK) st = orc_match(Y1o ? Y1o : Zo, H, W, N, s, p->search_radius, K, idx, NULL, nt);
    for (int c = 0; c < 3 && st == ORC_OK; c++) {
        const double sc = sigma * orc_opp_sigma_scale(c);
        if (!Y1o) {
            st = orc_filter_ht(Zo + c * n, H, W, idx, By, Bx, N, K, sc, p->levels, p->cycle_spins, p->tau_a,
                               p->tau_b, p->eps_w, gr, w, nt);
            if (st == ORC_OK) st = orc_aggregate(gr, w, idx, (int)G, K, H, W, N, 0.0, out + c * n, 1);
        } else {
            st = orc_filter_wiener(Zo + c * n, Y1o + c * n, H, W, idx, (int)G, N, K, sc, p->eps_w, gr, w, nt);
            if (st == ORC_OK) st = orc_aggregate(gr, w, idx, (int)G, K, H, W, N, p->kaiser_beta, out + c * n, 1);
        }
    }
    free(idx); free(gr); free(w);
    return st;
}

/* Colour denoising of Z (3 planes R, G, B of H x W) into out (3 planes). */
int orc_denoise_color(const double *Z, int H, int W, double sigma, const orc_params *p, double *out, int nthreads)
{
    if (!Z || !p || !out || H < p->patch || W < p->patch || H < stage_patch(p, 2) || W < stage_patch(p, 2) ||
        p->translations < 1 || p->translations > 3 || p->stages < 1 || p->stages > 2 || sigma < 0)
        return ORC_EINVAL;
    const size_t n = (size_t)H * W;
    int hs[3], hs2[3];
    stage_shifts(p, 1, hs);
    stage_shifts(p, 2, hs2);
    double *zo = malloc(sizeof(double) * 3 * n), *zs = malloc(sizeof(double) * 3 * n);
    double *o = malloc(sizeof(double) * 3 * n), *os = malloc(sizeof(double) * 3 * n);
    double *y1 = calloc(3 * n, sizeof(double)), *y1s = malloc(sizeof(double) * 3 * n);
    double *acc = calloc(3 * n, sizeof(double));
    int st = (zo && zs && o && os && y1 && y1s && acc) ? ORC_OK : ORC_ENOMEM;
    if (st == ORC_OK) st = orc_opp(Z, n, 0, zo);
    for (int t = 0; t < p->translations && st == ORC_OK; t++) {
        for (int c = 0; c < 3; c++) shift2(zo + c * n, zs + c * n, H, W, hs[t]);
        st = stage_color(zs, NULL, H, W, sigma, p, o, nthreads);
        for (int c = 0; c < 3 && st == ORC_OK; c++) {
            shift2(o + c * n, os + c * n, H, W, -hs[t]);
            for (size_t e = 0; e < n; e++) y1[c * n + e] += os[c * n + e] / p->translations;
        }
    }
    if (st == ORC_OK && p->stages == 1) memcpy(acc, y1, sizeof(double) * 3 * n);
    for (int t = 0; p->stages == 2 && t < p->translations && st == ORC_OK; t++) {
        for (int c = 0; c < 3; c++) {
            shift2(zo + c * n, zs + c * n, H, W, hs2[t]);
            shift2(y1 + c * n, y1s + c * n, H, W, hs2[t]);
        }
        st = stage_color(zs, y1s, H, W, sigma, p, o, nthreads);
        for (int c = 0; c < 3 && st == ORC_OK; c++) {
            shift2(o + c * n, os + c * n, H, W, -hs2[t]);
            for (size_t e = 0; e < n; e++) acc[c * n + e] += os[c * n + e] / p->translations;
        }
    }
    if (st == ORC_OK) st = orc_opp(acc, n, 1, out);
    free(zo); free(zs); free(o); free(os); free(y1); free(y1s); free(acc);
    return st;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
