// internal.cuh -- declarations shared by the CUDA translation units of
// libgbm3d (launch wrappers, workspace layout helpers).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "gbm3d.h"

namespace gbm3d {

constexpr int kPatch = 8;      // block side of the Wiener filter and of the tensor-core matcher
constexpr int kMaxPatch = 16;  // largest block side (stage 1 of the Sec. 5 parameters)
constexpr int kMaxK = 32;      // largest group size (one warp lane per list slot)
constexpr size_t kAlign = 256; // workspace sub-buffer alignment

inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Reference-grid count: positions 0, s, 2s, ... <= M-N plus M-N itself.
inline int grid_count(int M, int N, int s)
{
    if (M < N || N <= 0 || s <= 0) return 0;
    int n = (M - N) / s + 1;
    return ((M - N) % s) ? n + 1 : n;
}

// Position of reference p on a grid of stride s (the last one clamps to M-N).
__host__ __device__ inline int grid_pos(int p, int s, int M, int N)
{
    int v = p * s;
    return v < M - N ? v : M - N;
}

// Top-left (k, l) of the N x N block at position pos = k*W + l, clamped so
// that an out-of-range entry in a caller-supplied match list can never
// address memory outside the image (such entries yield garbage, not a fault).
__device__ __forceinline__ void block_kl(int pos, int H, int W, int N, int &k, int &l)
{
    if (pos < 0 || pos >= H * W) pos = 0;
    k = pos / W;
    l = pos - k * W;
    k = k < H - N ? k : H - N;
    l = l < W - N ? l : W - N;
}

// True when pos is a valid N x N block top-left for an H x W image.
__device__ __forceinline__ bool block_ok(int pos, int H, int W, int N)
{
    if (pos < 0 || pos >= H * W) return false;
    const int k = pos / W, l = pos - k * W;
    return k <= H - N && l <= W - N;
}

// Where the filters put block r of group g (entry e = g*K + r), row a:
//   base + slot(e) * s_slot + a * s_row   (N consecutive floats, b = 0..N-1),
// slot(e) = slot_of[e] (position-sorted order used by the aggregation) or e
// itself (the group-major [G][K][N][N] layout of the public calls).  Weights
// go to w[g] (per_slot = 0) or to w[slot(e)] for each of the group's K
// entries (per_slot = 1).
struct GroupOut {
    float *base;
    const int *slot_of;
    long long s_slot, s_row;
    float *w;
    int per_slot;
    __device__ __forceinline__ long long slot(long long e) const { return slot_of ? (long long)__ldg(slot_of + e) : e; }
    __device__ __forceinline__ float *row(long long e, int a) const { return base + slot(e) * s_slot + a * s_row; }
};

inline GroupOut group_major(float *groups, float *w, int N)
{
    return GroupOut{groups, nullptr, (long long)N * N, N, w, 0};
}

inline GroupOut position_planar(float *planes, const int *slot_of, long long n_entries, float *w_slot, int N)
{
    return GroupOut{planes, slot_of, N, n_entries * N, w_slot, 1};
}

// Geometry of the stage-1 mosaic volume and of its wavelet pyramid.
struct HtGeom {
    int N;                  // block side (8 or 16)
    int By, Bx, K;          // groups along y, x; blocks per group
    int Yd, Xd;             // mosaic dims (By*N, Bx*N)
    int levels;
    size_t level_elems[4];  // elements of the coefficient buffer of level l (1-based)
    size_t level_off[4];    // byte offset of each level buffer in the HT scratch
    size_t ofs_off;         // byte offset of the pixel-offset table (G*K ints)
    size_t gm_off;          // byte offset of the group-major block scratch (G*K*N*N floats)
    size_t bytes;           // total HT scratch
};
HtGeom ht_geom(int By, int Bx, int K, int levels, int N);

struct AggLayout {
    size_t cnt, off, cursor, list, slot_of, lpos, bsum, bytes; // byte offsets and total
    int npos, nblk;
};
AggLayout agg_layout(int H, int W, int G, int K, bool with_slots = false);

// Inverted match lists (block position -> entries, entries ascending within a
// position) in the aggregation scratch; with_slots also fills slot_of.
// N: block side (entries that are not valid N x N block positions are skipped).
cudaError_t build_csr(const int32_t *idx, int G, int K, int H, int W, int N, void *agg_ws, bool with_slots,
                      cudaStream_t st);

size_t match_smem_bytes(int s, int R, int N);

// Size of the fixed device scratch used by gbm3d_aggregate_noalloc, and its
// device address on the current device (looked up once per device).
constexpr size_t kFixedScratchBytes = size_t(8) << 20;
cudaError_t fixed_scratch(void **ptr);

// Sets the thread's last-error message (gbm3d_last_error_string) and returns code.
int set_error(int code, const char *msg);
// Replaces the thread's measurement-hook events (gbm3d_set_match_events); returns the old ones.
cudaEvent_t *swap_match_events(cudaEvent_t *events);

// Learned pilot (pilot.cu): scratch of one H x W forward pass, and the pass
// (Z and pilot with their pitches; theta: the flat FP32 parameter vector).
size_t pilot_infer_bytes(int H, int W);
cudaError_t launch_pilot(const float *Z, int H, int W, int pitch, float sigma, const float *theta, float *pilot,
                         int ppitch, void *ws, cudaStream_t st);

// ---- launch wrappers (each returns cudaGetLastError()) -------------------
// Direct FP32 block matching, N = 8 or 16.
cudaError_t launch_match(const float *img, int H, int W, int pitch, int By, int Bx, int N, int s, int R, int K,
                         int32_t *idx, float *dist, cudaStream_t st);

// Tensor-core matching (same results as launch_match, bit for bit) where the
// geometry fits (N = 8, union of 8 grid columns' windows <= 64 columns,
// K <= 32); it ends with launch_match_fix, which re-matches with the direct
// kernel the references it marked (slot 0 < 0).
bool match_tc_supported(int H, int W, int N, int s, int R, int K);
cudaError_t launch_match_tc(const float *img, int H, int W, int pitch, int By, int Bx, int s, int R, int K,
                            int32_t *idx, float *dist, cudaStream_t st);
cudaError_t launch_match_fix(const float *img, int H, int W, int pitch, int By, int Bx, int s, int R, int K,
                             int32_t *idx, float *dist, cudaStream_t st);
// Box-sum matching (same lists as launch_match up to FP32 rounding of the
// distances; exact selection) for N = 8 and strides 1..3.
bool match_box_supported(int N, int s, int R, int K);
cudaError_t launch_match_box(const float *img, int H, int W, int pitch, int By, int Bx, int s, int R, int K,
                             int32_t *idx, float *dist, cudaStream_t st);
// Cumulative counts of the tensor-core matcher on the current device: bounded
// waits that gave up, references re-matched by the direct kernel
// (synchronous read).
cudaError_t tc_stats(unsigned long long *timeouts, unsigned long long *rematched);

// launch_filter_ht in two parts: the cycle-spun transforms into the
// group-major scratch (needs only idx), then the TV weights and, for a
// position-planar out, the permutation (needs out's slot table).
cudaError_t launch_ht_transforms(const float *img, int H, int W, int pitch, const int32_t *idx, const HtGeom &g,
                                 float sigma, float tau_a, float tau_b, int cycle_spins, const GroupOut &out,
                                 void *ht_ws, cudaStream_t st);
cudaError_t launch_ht_weights(const HtGeom &g, float eps_w, const GroupOut &out, void *ht_ws, cudaStream_t st);
cudaError_t launch_filter_ht(const float *img, int H, int W, int pitch, const int32_t *idx, const HtGeom &g,
                             float sigma, float tau_a, float tau_b, int cycle_spins, float eps_w, const GroupOut &out,
                             void *ht_ws, cudaStream_t st);

cudaError_t launch_filter_wiener(const float *noisy, int npitch, const float *pilot, int ppitch, int H, int W,
                                 const int32_t *idx, int G, int K, float sigma, float eps_w, const GroupOut &out,
                                 cudaStream_t st);

// Aggregation from the position-planar layout written through a GroupOut
// made by position_planar() with the slot_of of build_csr.  window: the N
// per-axis window factors.
cudaError_t launch_aggregate_planar(const float *planes, const float *w_slot, int n_entries, int H, int W, int N,
                                    int pitch, const float *window, float *out, const void *agg_ws, cudaStream_t st);

cudaError_t launch_aggregate(const float *groups, const float *w, const int32_t *idx, int G, int K, int H, int W,
                             int N, int pitch, const float *window, float *out, void *agg_ws, cudaStream_t st);

cudaError_t launch_shift(const float *src, int spitch, float *dst, int dpitch, int H, int W, int h, float scale,
                         int accumulate, cudaStream_t st);

} // namespace gbm3d
