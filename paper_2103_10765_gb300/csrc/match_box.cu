// match_box.cu -- block matching by shared box sums (Sec. 2 eq. dfg, Sec. 3.1
// S^K_pq): exact FP32 squared distances and exact top-(K-1) lists, for grids
// whose stride is small against the block side (s <= 3, N = 8; the default
// grid is s = 3).
//
// For one offset (dy, dx) the distance of every reference block of a tile to
// its candidate at that offset is a box sum of the same squared-difference
// image: neighbouring references (stride 3 < 8) share most of it.  A CTA
// owns a tile of 16 x 16 references and walks all (2R + 1)^2 offsets, four
// at a time (dx .. dx + 3):
//   phase A  row sums Sx[y][q] = sum_b (T[y][j_q + b] - Z[y + dy][j_q + b + dx])^2
//            for every pixel row y of the tile and reference column q; a
//            worker thread owns one row and four lattice columns q (17 pixels
//            of the tile row in registers for the whole kernel, 20 pixels of
//            the shifted row loaded per batch);
//   phase B  thread (p, q) adds its 8 rows: D = sum_a Sx[i_p + a][q]
//            (ascending a), tests it against its current (K-1)-th key and
//            queues it.
// Every distance is a fixed sequence of FP32 operations (so the lists are
// deterministic); parity with the FP64 definition is at FP32 rounding.
// Selection: each thread keeps its LP smallest keys (distance, k*W + l) in
// registers, sorted; keys below the (K-1)-th go to a per-thread queue in
// shared memory, and a warp whose lanes hold 16 queued keys merges them with
// a branch-free sorting network (exact lexicographic order).  Offsets are
// visited by increasing |dy| so that thresholds tighten early.
#include <limits.h>

#include "internal.cuh"

namespace gbm3d {
namespace {

constexpr int kTP = 16, kTQ = 16, kThr = kTP * kTQ; // references per tile, one per thread
constexpr int kQG = 4;                               // lattice columns per phase-A worker
constexpr int kDX = 4;                               // offsets (consecutive dx) per batch
constexpr int kQCap = 24, kFlush = 16;               // per-thread key queue
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ bool kless(float da, int ia, float db, int ib)
{
    return da < db || (da == db && ia < ib);
}

// Compare-exchange in (distance, index) order.
__device__ __forceinline__ void kcex(float &a, int &ia, float &b, int &ib)
{
    const bool sw = kless(b, ib, a, ia);
    const float ta = sw ? b : a, tb = sw ? a : b;
    const int tia = sw ? ib : ia, tib = sw ? ia : ib;
    a = ta;
    b = tb;
    ia = tia;
    ib = tib;
}

// Batcher's odd-even merge sort of 16 keys.
__device__ __forceinline__ void ksort16(float (&k)[16], int (&v)[16])
{
#define CX(i, j) kcex(k[i], v[i], k[j], v[j])
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

// lk (ascending, LP keys) <- the LP smallest of lk and pk (16 keys): sort
// pk, keep min(lk[LP-16+t], pk[15-t]) (a bitonic sequence holding the LP
// smallest), bitonic merge.  Branch-free.
template <int LP>
__device__ __forceinline__ void kmerge16(float (&lk)[LP], int (&li)[LP], float (&pk)[16], int (&pi)[16])
{
    ksort16(pk, pi);
#pragma unroll
    for (int t = 0; t < 16; t++) {
        const float a = lk[LP - 16 + t], b = pk[15 - t];
        const int ia = li[LP - 16 + t], ib = pi[15 - t];
        const bool sw = kless(b, ib, a, ia);
        lk[LP - 16 + t] = sw ? b : a;
        li[LP - 16 + t] = sw ? ib : ia;
    }
#pragma unroll
    for (int st = LP / 2; st > 0; st >>= 1)
#pragma unroll
        for (int i = 0; i < LP; i++)
            if ((i & st) == 0) kcex(lk[i], li[i], lk[i + st], li[i + st]);
}

struct BoxArgs {
    const float *img;
    int H, W, pitch, By, Bx, s, R, K;
    int RW;        // shared row stride of the staged region (floats)
    int sx_off;    // float offset of the row-sum buffers in shared memory
    int q_off;     // float offset of the key queue
    int32_t *idx;
    float *dist;
};

// Order of the dx batches [dx0, dx0 + 3] (dx0 = -R + 4 b) within a row of
// offsets: by increasing distance of their centre from 0, nearest candidates
// first so that the thresholds tighten early.  Rows go by increasing |dy|
// (0, 1, -1, 2, ...).
constexpr int kMaxNbx = 32; // R <= 125

__device__ __forceinline__ int batch_dy(int row) { return (row & 1) ? (row + 1) >> 1 : -(row >> 1); }

__device__ void batch_order(int R, int nbx, int *dx0)
{
    // b0: the batch whose centre -R + 4 b0 + 1.5 is nearest 0; then b0 + 1,
    // b0 - 1, b0 + 2, ... (those inside [0, nbx))
    const int b0 = (R + 1) / kDX - ((R + 1) % kDX == 0 ? 1 : 0);
    int n = 0;
    for (int t = 0; n < nbx; t++) {
        const int cand = b0 + ((t & 1) ? (t + 1) >> 1 : -(t >> 1));
        if (cand >= 0 && cand < nbx) dx0[n++] = -R + kDX * cand;
    }
}

// SS: the grid stride (compile time, so the row windows stay in registers).
template <int LP, int SS>
__global__ void __launch_bounds__(kThr, 2) k_match_box(BoxArgs A)
{
    extern __shared__ __align__(16) float sm[];
    const int H = A.H, W = A.W, R = A.R, K = A.K, RW = A.RW;
    constexpr int s = SS;
    constexpr int N = kPatch;
    const int tid = threadIdx.x, lane = tid & 31;
    const int p0 = blockIdx.y * kTP, q0 = blockIdx.x * kTQ;
    const int np = min(kTP, A.By - p0), nq = min(kTQ, A.Bx - q0);
    const int iF = grid_pos(p0, s, H, N), iL = grid_pos(p0 + np - 1, s, H, N);
    const int jF = grid_pos(q0, s, W, N), jL = grid_pos(q0 + nq - 1, s, W, N);
    const int TH = iL - iF + N, TW = jL - jF + N; // tile pixels
    const int ry0 = iF - R, rx0 = jF - R;         // region origin (may be negative: zero fill)
    // staged region: the tile, R pixels around it, and kDX zero columns on the
    // right that the last offset batch (dx up to R + 3) may read
    const int RH = TH + 2 * R, RWd = TW + 2 * R + kDX;
    float *reg = sm;                                  // [RH][RW]
    float *sx = sm + A.sx_off;                        // [2][kDX][kTQ][TH] row sums, double-buffered
    float *qk = sm + A.q_off;                         // [kQCap][kThr] queued distances
    int *qi = reinterpret_cast<int *>(qk + kQCap * kThr); // [kQCap][kThr] queued indices
    const int sxs = kDX * kTQ * TH;                   // floats of one row-sum buffer

    { // eight loads per thread in flight before their stores
        constexpr int kLd = 8;
        for (int e0 = tid; e0 < RH * RWd; e0 += kLd * kThr) {
            float v[kLd];
#pragma unroll
            for (int u = 0; u < kLd; u++) {
                const int e = e0 + u * kThr;
                const int y = e / RWd, x = e - y * RWd, gy = ry0 + y, gx = rx0 + x;
                v[u] = (e < RH * RWd && gy >= 0 && gy < H && gx >= 0 && gx < W)
                           ? __ldg(A.img + (size_t)gy * A.pitch + gx)
                           : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kLd; u++) {
                const int e = e0 + u * kThr;
                if (e < RH * RWd) {
                    const int y = e / RWd, x = e - y * RWd;
                    reg[y * RW + x] = v[u];
                }
            }
        }
    }
    __syncthreads();

    // ---- phase-A role: row y = tid / 4 (TH <= 53 < 64 rows for s <= 3),
    // lattice columns 4 g .. 4 g + 3 of the tile
    static_assert(kThr / kQG >= (kTP - 1) * 3 + kPatch, "phase-A rows");
    const int ay = tid >> 2, ag = tid & 3;
    // columns of the tile's references relative to jF (the last grid column
    // may sit off the lattice: it is summed separately)
    const int qa = kQG * ag;
    bool arow = ay < TH && qa < nq;
    constexpr int span = (kQG - 1) * SS + N; // tile pixels of a worker (17 for s = 3)
    float T[span];
#pragma unroll
    for (int x = 0; x < span; x++) T[x] = 0.f;
    if (arow) {
        const float *tr = reg + (ay + R) * RW + R + (grid_pos(q0 + qa, s, W, N) - jF);
        const int avail = TW - (grid_pos(q0 + qa, s, W, N) - jF); // pixels of the tile row from there
#pragma unroll
        for (int x = 0; x < span; x++)
            if (x < avail) T[x] = tr[x];
    }
    // is column q of the group on the lattice (j_q - j_qa = s (q - qa))?
    unsigned on_lat = 0;
#pragma unroll
    for (int c = 0; c < kQG; c++) {
        const int q = q0 + qa + c;
        if (qa + c < nq && grid_pos(q, s, W, N) - grid_pos(q0 + qa, s, W, N) == s * c) on_lat |= 1u << c;
    }

    // ---- phase-B role: reference (p, q) = (tid / 16, tid % 16)
    const int bp = tid / kTQ, bq = tid % kTQ;
    const bool bref = bp < np && bq < nq;
    const int ri = bref ? grid_pos(p0 + bp, s, H, N) : 0, rj = bref ? grid_pos(q0 + bq, s, W, N) : 0;
    const int ky0 = max(0, ri - R) - ri, ky1 = min(H - N, ri + R) - ri; // dy window of this reference
    const int kx0 = max(0, rj - R) - rj, kx1 = min(W - N, rj + R) - rj;
    const int brow = ri - iF; // first tile row of the block
    const float kInf = __int_as_float(0x7f800000);
    // the list: LP - K + 1 sentinels (-inf, smaller than every key, never
    // displaced) below the K - 1 real keys, so that the (K-1)-th smallest real
    // key always sits in the last slot
    float lk[LP];
    int li[LP];
    const int nsent = LP - K + 1;
#pragma unroll
    for (int t = 0; t < LP; t++) {
        lk[t] = t < nsent ? -kInf : kInf;
        li[t] = t < nsent ? INT_MIN : INT_MAX;
    }
    float thr = kInf;
    int thri = INT_MAX;
    int qn = 0;

    const int nbx = (2 * R + 1 + kDX - 1) / kDX, nrow = 2 * R + 1;
    const int nb = nrow * nbx;
    __shared__ int s_dx0[kMaxNbx];
    if (tid == 0) batch_order(R, nbx, s_dx0);
    __syncthreads();
    for (int o = 0, row = 0, k = 0; o < nb; o++) {
        const int dy = batch_dy(row), dx0 = s_dx0[k];
        if (++k == nbx) {
            k = 0;
            row++;
        }
        float *sxb = sx + (o & 1) * sxs;
        // phase A: row sums of this row for 4 offsets and 4 lattice columns
        if (arow) {
            const float *sr = reg + (ay + R + dy) * RW + R + (grid_pos(q0 + qa, s, W, N) - jF) + dx0;
            const int avail = TW + R + kDX - (grid_pos(q0 + qa, s, W, N) - jF) - dx0; // staged pixels from sr
            float S[span + kDX - 1];
#pragma unroll
            for (int x = 0; x < span + kDX - 1; x++) S[x] = x < avail ? sr[x] : 0.f;
#pragma unroll
            for (int d = 0; d < kDX; d++) {
#pragma unroll
                for (int c = 0; c < kQG; c++) {
                    if (!((on_lat >> c) & 1)) continue;
                    float acc = 0.f;
#pragma unroll
                    for (int b = 0; b < N; b++) {
                        const float dv = T[SS * c + b] - S[SS * c + b + d];
                        acc = fmaf(dv, dv, acc);
                    }
                    sxb[(d * kTQ + qa + c) * TH + ay] = acc;
                }
            }
        }
        // off-lattice reference columns (the clamped last grid column): their
        // row sums straight from shared memory
        if (ay < TH && qa < nq && on_lat != ((1u << min(kQG, nq - qa)) - 1)) {
#pragma unroll 1
            for (int c = 0; c < kQG; c++) {
                if (qa + c >= nq || ((on_lat >> c) & 1)) continue;
                const int xc = R + grid_pos(q0 + qa + c, s, W, N) - jF;
                const float *tr = reg + (ay + R) * RW + xc, *sr = reg + (ay + R + dy) * RW + xc + dx0;
                for (int d = 0; d < kDX; d++) {
                    float acc = 0.f;
                    for (int b = 0; b < N; b++) {
                        const float dv = tr[b] - sr[b + d];
                        acc = fmaf(dv, dv, acc);
                    }
                    sxb[(d * kTQ + qa + c) * TH + ay] = acc;
                }
            }
        }
        __syncthreads();
        // phase B: box sums, threshold test, queue
        if (bref && dy >= ky0 && dy <= ky1) {
            const float *col = sxb + bq * TH + brow;
#pragma unroll
            for (int d = 0; d < kDX; d++) {
                const int dx = dx0 + d;
                if (dx < kx0 || dx > kx1 || (dx == 0 && dy == 0)) continue;
                const float *c8 = col + d * kTQ * TH;
                float D = 0.f;
#pragma unroll
                for (int a = 0; a < N; a++) D += c8[a];
                const int id = (ri + dy) * W + (rj + dx);
                if (kless(D, id, thr, thri)) {
                    qk[qn * kThr + tid] = D;
                    qi[qn * kThr + tid] = id;
                    qn++;
                }
            }
        }
        // merge when some lane of the warp holds kFlush queued keys
        if (__ballot_sync(kFull, qn >= kFlush)) {
            float pk[16];
            int pi[16];
#pragma unroll
            for (int t = 0; t < 16; t++) {
                const bool v = t < qn;
                pk[t] = v ? qk[t * kThr + tid] : kInf;
                pi[t] = v ? qi[t * kThr + tid] : INT_MAX;
            }
            kmerge16<LP>(lk, li, pk, pi);
            const int rest = qn > 16 ? qn - 16 : 0;
            for (int t = 0; t < rest; t++) {
                qk[t * kThr + tid] = qk[(16 + t) * kThr + tid];
                qi[t * kThr + tid] = qi[(16 + t) * kThr + tid];
            }
            qn = rest;
            // threshold: the (K-1)-th smallest key, in the last slot (keys queued
            // before this merge that no longer qualify are merged later and
            // fall out exactly)
            thr = lk[LP - 1];
            thri = li[LP - 1];
        }
    }
    // final merges (the queue may hold up to kFlush - 1 + kDX keys)
    while (__ballot_sync(kFull, qn > 0)) {
        float pk[16];
        int pi[16];
#pragma unroll
        for (int t = 0; t < 16; t++) {
            const bool v = t < qn;
            pk[t] = v ? qk[t * kThr + tid] : kInf;
            pi[t] = v ? qi[t * kThr + tid] : INT_MAX;
        }
        kmerge16<LP>(lk, li, pk, pi);
        const int rest = qn > 16 ? qn - 16 : 0;
        for (int t = 0; t < rest; t++) {
            qk[t * kThr + tid] = qk[(16 + t) * kThr + tid];
            qi[t * kThr + tid] = qi[(16 + t) * kThr + tid];
        }
        qn = rest;
    }
    if (!bref) return;
    const size_t gi = ((size_t)(p0 + bp) * A.Bx + (q0 + bq)) * K;
    A.idx[gi] = ri * W + rj;
    if (A.dist) A.dist[gi] = 0.f;
#pragma unroll
    for (int t = 0; t < LP; t++)
        if (t >= nsent) {
            A.idx[gi + 1 + t - nsent] = li[t];
            if (A.dist) A.dist[gi + 1 + t - nsent] = lk[t];
        }
}

struct BoxLayout {
    int RW, sx_off, q_off;
    size_t bytes;
};

BoxLayout box_layout(int s, int R)
{
    BoxLayout L{};
    const int TH = (kTP - 1) * s + kPatch, TW = (kTQ - 1) * s + kPatch;
    const int RH = TH + 2 * R, RWd = TW + 2 * R + kDX;
    L.RW = RWd | 1; // odd stride
    L.sx_off = (RH * L.RW + 3) / 4 * 4;
    L.q_off = L.sx_off + (2 * kDX * kTQ * TH + 3) / 4 * 4;
    L.bytes = (size_t)(L.q_off + 2 * kQCap * kThr) * sizeof(float);
    return L;
}

} // namespace

bool match_box_supported(int N, int s, int R, int K)
{
    // the 64 phase-A rows (256 threads, 4 per row) cover the tile's
    // (kTP - 1) s + N pixel rows for s <= 3
    return N == kPatch && s >= 1 && s <= 3 && K >= 2 && K <= kMaxK && (2 * R + 1 + kDX - 1) / kDX <= kMaxNbx &&
           box_layout(s, R).bytes <= 200 * 1024;
}

cudaError_t launch_match_box(const float *img, int H, int W, int pitch, int By, int Bx, int s, int R, int K,
                             int32_t *idx, float *dist, cudaStream_t st)
{
    const BoxLayout L = box_layout(s, R);
    void (*kern)(BoxArgs) = nullptr;
    const bool small = K <= 17;
    switch (s) {
    case 1: kern = small ? k_match_box<16, 1> : k_match_box<32, 1>; break;
    case 2: kern = small ? k_match_box<16, 2> : k_match_box<32, 2>; break;
    case 3: kern = small ? k_match_box<16, 3> : k_match_box<32, 3>; break;
    default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
    if (e != cudaSuccess) return e;
    const BoxArgs a{img, H, W, pitch, By, Bx, s, R, K, L.RW, L.sx_off, L.q_off, idx, dist};
    dim3 grid((Bx + kTQ - 1) / kTQ, (By + kTP - 1) / kTP);
    kern<<<grid, kThr, L.bytes, st>>>(a);
    return cudaGetLastError();
}

} // namespace gbm3d
