// Internal definitions shared by the rasterizer's CUDA translation units.
//
// Data layout in HBM (all owned by the context workspace):
//   rec_hot  [F][N][HOT4] float4  per-(frame, Gaussian) compositing record:
//            {mu_x_hi, mu_y_hi, mu_x_lo, mu_y_lo}  double-float pixel-space centre
//            {u11, u12, u22, alpha}                Cholesky factor of Sigma_2D^-1 (scaled)
//            {colour 0..3}, {colour 4..7}          C = 3 uses one colour vector, C = 8 two
//   rec_cold [F][N][2] float4     {n_c.x, n_c.y, n_c.z, d0 = p_c . n_c},
//                                 {z_c, rank (int bits), pixel rect lo (x0|y0<<16), hi (x1|y1<<16)}
//   rec_box  [F][N] float2        half-extents of the alpha_min support box around mu
//   ntiles   [F][N] uint32        masked tiles touched (0 = culled or off-mask)
//   cand     [F*N] uint32         (frame, Gaussian) pairs f * N + i that passed the coarse cull
//   scand    [F*N] uint32         window cache: projected (frame, stable Gaussian) pairs, whose
//                                 records stay valid while the window is open
//   stage    [pairs] uint4        (tile, slot, key) of every pair, written by the projection
//   keys     [pairs] uint64       (float bits of z_c) << 32 | Gaussian index, bucketed by tile
//   sorted   [pairs] uint32       Gaussian index, each tile's bucket in front-to-back order
//   px_list  [F*T][tile pixels] u8 masked pixels of each render tile (index in the tile),
//                                 compacted in the tile's Z order
//   items    [groups] uint32      (tile << 3 | 32-pixel group) work items, longest list first
//   px_*     [F][H][W]            per-pixel state saved by the forward for the backward
//   grad2d   [F][N][G2] float     per-(frame, unstable Gaussian) screen-space gradients
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rtg.h"

namespace rtg {

constexpr int kTile = RTG_TILE;              // 16 x 16 tiles of the unstable-mask rule
constexpr int kTileShift = 4;                // log2(kTile)
constexpr int kTilePix = kTile * kTile;      // 256 pixels = 256 threads per mask-tile CTA
constexpr int kMaxTilePix = 256;             // largest render tile (pixel index fits a byte)
constexpr int kMaxFrames = RTG_MAX_FRAMES;
// q = t1^2 + t2^2 with t = U d and U scaled by sqrt(log2(e) / 2), so exp(-p/2) = 2^-q
constexpr float kQScale = 0.84932180028801904272f;   // sqrt(0.5 * log2(e))
constexpr float kLn2 = 0.69314718055994530942f;
constexpr float kQScale2 = 0.72134752044448170368f;  // kQScale^2 = 0.5 * log2(e)

// Counter slots in Work::counters (uint64).  Each counter sits on its own 128-byte line:
// thousands of blocks reserve staging ranges with atomics on them in the same kernels, and
// atomics on one line serialise in one L2 slice even when their addresses differ.
constexpr int kCounterStride = 16;  // uint64 per 128-byte line
enum Counter {
  kPairs = 0 * kCounterStride,
  kFragments = 1 * kCounterStride,
  kVisible = 2 * kCounterStride,
  kMaskedPix = 3 * kCounterStride,
  kNumUnstable = 4 * kCounterStride,
  kMaxTilePairs = 5 * kCounterStride,
  kSkip = 6 * kCounterStride,         // non-zero: pairs overflowed, downstream kernels skip
  kCand = 7 * kCounterStride,         // (frame, Gaussian) candidates that passed the coarse cull
  kStaged = 8 * kCounterStride,       // (Gaussian, tile) pairs staged for the scatter into buckets
  kItems = 9 * kCounterStride,        // (tile, 32-pixel group) work items of the persistent schedule
  kQFwd = 10 * kCounterStride,        // next item of the persistent forward (past the first one per warp)
  kQBwd = 11 * kCounterStride,        // next item of the persistent backward
  kWarpRecords = 12 * kCounterStride, // records the forward's warps walked after culling
  kBwdSteps = 13 * kCounterStride,    // steps of the backward's per-lane fragment replay (warp-wide)
  kDepthPix = 14 * kCounterStride,    // pixels in the last fused L1 loss's depth term (D_hat != -1, D > 0)
  kWinStable = 15 * kCounterStride,   // projected (frame, stable Gaussian) entries of the open window (kept)
  kBSeg0 = 16 * kCounterStride,       // backward segments queued in cost bins 0..kSegBins-1 (one slot each)
  kSortTiles = 20 * kCounterStride,   // tiles with keys, listed in tile_order for the sort
};
constexpr int kNumCounterSlots = 21;  // slots; all but kWinStable are cleared at the start of every call
constexpr int kNumCounters = kNumCounterSlots * kCounterStride;  // array length

struct DevCam {
  float fx, fy, cx, cy;
  int W, H;
  float R[9];  // camera-to-world, row-major
  float t[3];
  float lim_x, lim_y;  // guard band on |X/Z| and |Y/Z|
  int tiles_x, tiles_y;    // render tiles of 2^tws x 2^ths pixels
  int tws, ths;
  int mtiles_x, mtiles_y;  // 16 x 16 tiles of the unstable-mask rule
};

struct Prm {
  float near_z, alpha_min, f_max, t_eps, delta_alpha, cos_max, lowpass, guard, discard;
};

struct GaussPtrs {
  const float *means, *scales, *quats, *opacity, *colors;
  const uint8_t *unstable;
  const float *u_means, *u_scales, *u_quats, *u_opacity, *u_colors;
  int64_t n;
  int C;                // colour channels of a render (3 with SH)
  const int32_t *rank_map, *unstable_ids;  // optional precomputed unstable index
  int64_t n_unstable;
  int sh_degree;        // 0: colours are the channels; 1..3: SH coefficients [(d+1)^2][3]
  int col_stride;       // colour values per Gaussian: C, or 3 (d+1)^2
};

// Inputs of the L1 loss fused into the forward / backward (tcolor == nullptr: not fused).
struct L1Fused {
  const float *tcolor, *tdepth;  // targets [F,C,H,W], [F,H,W]
  const float *color, *depth;    // the forward's rendered colour and depth
};

// Backward segments.  The persistent backward takes a 32-pixel group's list in segments of
// kSeg entries (the last of kSegMax segments runs to the end of the list), so that no warp
// replays a whole long list alone.  The forward leaves, for each pixel and each segment
// boundary it walked past, the transmission and the colour composited in front of it
// (Eq. 1 and 3 over the entries before the boundary), and the final pair after its walk;
// the backward starts a segment from them.  Finished segments go to one of kSegBins queues
// by their cost (the most fragments a lane composited in them), the costliest first.
constexpr int kSeg = 64;
constexpr int kSegMax = 8;
constexpr int kSegBins = 4;
__host__ __device__ inline int ck4_of(int C) { return (C + 4) / 4; }  // float4 per checkpoint: T, C colours

struct Work {
  DevCam *cams;
  unsigned long long *counters;
  int32_t *rank;        // [N] compact unstable index, -1 if stable
  int32_t *ids;         // [N] compact -> original index
  int32_t *block_cnt;   // [ceil(N / kScanBlock)]
  uint32_t *cand;       // [F*N] candidates f * N + i of the coarse cull, dense, in no particular order
  uint32_t *scand;      // [F*N] projected (frame, stable Gaussian) entries of the open window
  float4 *rec_hot;
  float4 *rec_cold;
  float2 *rec_box;      // [F][N] support half-extents (rx, ry) around mu
  uint32_t *ntiles;     // [F*N] non-zero iff the (frame, Gaussian) entry has a pair in a masked tile
  uint32_t *tile_npix;  // [F*T] masked pixels per tile
  uint32_t *tile_count; // [F*T + 1]
  uint32_t *tile_offset;// [F*T + 1]
  uint32_t *tile_cursor;// [F*T]
  unsigned long long *keys;
  unsigned long long *keys_alt;
  uint4 *stage;         // [pairs] (global tile, slot in its bucket, key lo, key hi)
  uint8_t *px_list;     // [F*T << (tws + ths)] masked pixels of each render tile
  uint32_t *items;      // [groups] work items of the persistent schedule
  uint32_t *tile_order; // [F*T] the tiles with keys, longest list first (the sort's CTA order)
  unsigned long long *scan_part;  // [scan blocks][4] partials of the multi-block tile scan
  uint32_t *scan_hist;            // [scan blocks][queue classes] per-block class counts, then starts
  uint32_t *sorted;
  float *px_T;
  uint32_t *px_last;
  int32_t *px_hit;
  float *grad2d;
  float *loss_part;     // [kLossBlocks * 4]
  float *tile_loss;     // [groups][4] per-(tile, 32-pixel group) fused L1 partials (colour, depth, depth count)
  float *loss_scal;     // [4]: L, Lc, Ld, (unused); [4..5] gradient scales
  uint32_t *loss_done;
  double *loss_acc;     // [4] FP64 sums of the persistent forward's fused L1 (colour, depth, depth
                        // count); the CTA that finalizes the loss returns them to zero
  uint32_t *status;     // host-mapped status word (device pointer)
  float4 *ckpt;         // [kSegMax][px_cap][ck4]: (T, colour in front) at entry boundaries
                        // kSeg, 2 kSeg, ..., then the pixel's final (T, colour) at index kSegMax - 1
  uint32_t *bseg;       // [kSegBins][bseg_cap] queued backward segments: tile << 6 | segment << 3 | group
  uint4 *gstate;        // [groups][32] a fused-loss forward's pixel state for the backward:
                        // (px | py << 16, or ~0 without a pixel; T bits; last; hit)
  uint32_t *gsign;      // [groups][32] its L1 signs, 2 bits a channel then depth (1: +, 2: -)
  int64_t px_cap;       // pixels of the capacity (frames x width x height)
  int64_t bseg_cap;     // entries per segment bin
};

// ----------------------------------------------------------------------------- sizes

__host__ __device__ inline int hot4_of(int C) { return C <= 4 ? 3 : 4; }
__host__ __device__ inline int g2_of(int C) { return C <= 5 ? 16 : 20; }  // 11 + C padded to float4
// grad2d row: [0..1] dL/dmu, [2..4] dL/d(conic a', b', c'), [5] dL/dalpha, [6..6+C) dL/dcolour,
// then the depth terms [6+C] dL/dd0, [7+C..9+C] dL/dn_c, [10+C] dL/dz_c.
constexpr int kG2Mu = 0, kG2Conic = 2, kG2Alpha = 5, kG2Col = 6;
__host__ __device__ inline int g2_d0(int C) { return 6 + C; }
__host__ __device__ inline int g2_nc(int C) { return 7 + C; }
__host__ __device__ inline int g2_z(int C) { return 10 + C; }

// ----------------------------------------------------------------------------- double-float
// Error-free transformations (Knuth's TwoSum, Dekker's product via FMA) and the
// "double-float" arithmetic built on them (Dekker 1971; Hida, Li & Bailey, QD library).
// Used to keep the world->camera transform and the pixel-space centre accurate to
// ~2^-44 relative, so that d = u - mu is exact to FP32 rounding even at |mu| ~ 10^3 px.
struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return quick_two_sum(s.hi, lo);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_div(df a, df b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  df r = df_add(a, df_mul_f(b, -q1));
  float q2 = __fdiv_rn(r.hi, b.hi);
  return quick_two_sum(q1, q2);
}

// a / b in double-float given rb ~ 1/b.hi (a few ulp suffice: the remainder step corrects q1)
__device__ __forceinline__ df df_div_rcp(df a, df b, float rb) {
  const float q1 = __fmul_rn(a.hi, rb);
  const df r = df_add(a, df_mul_f(b, -q1));
  return quick_two_sum(q1, __fmul_rn(r.hi, rb));
}

// ----------------------------------------------------------------------------- small math

// 2^x with the hardware approximation (relative error ~2^-22), flushing denormals.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float R[9]) {
  R[0] = 1.f - 2.f * (y * y + z * z);
  R[1] = 2.f * (x * y - w * z);
  R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);
  R[4] = 1.f - 2.f * (x * x + z * z);
  R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);
  R[7] = 2.f * (y * z + w * x);
  R[8] = 1.f - 2.f * (x * x + y * y);
}

__device__ __forceinline__ int argmin3(float a, float b, float c) {
  return (a <= b && a <= c) ? 0 : (b <= c ? 1 : 2);
}

// Parameters of Gaussian i, from the compact override when it is unstable and one is given.
struct GParams {
  float p[3], s[3], q[4], alpha;
};

// Gaussian i's parameters; with the optimiser's compact arrays (u_*), an unstable one's come
// from its row r = rank[i] (load_params_r: r given, -1 for a stable Gaussian).
__device__ __forceinline__ bool load_params_r(const GaussPtrs &g, int64_t i, int r, GParams &P) {
  const float *pm = g.means + 3 * i, *ps = g.scales + 3 * i, *pq = g.quats + 4 * i, *po = g.opacity + i;
  if (g.u_means != nullptr) {
    if (r >= 0) {
      pm = g.u_means + 3 * (int64_t)r;
      ps = g.u_scales + 3 * (int64_t)r;
      pq = g.u_quats + 4 * (int64_t)r;
      po = g.u_opacity + r;
    }
  }
  P.p[0] = pm[0]; P.p[1] = pm[1]; P.p[2] = pm[2];
  P.s[0] = ps[0]; P.s[1] = ps[1]; P.s[2] = ps[2];
  P.q[0] = pq[0]; P.q[1] = pq[1]; P.q[2] = pq[2]; P.q[3] = pq[3];
  P.alpha = *po;
  bool ok = isfinite(P.p[0]) && isfinite(P.p[1]) && isfinite(P.p[2]) && isfinite(P.s[0]) && isfinite(P.s[1]) &&
            isfinite(P.s[2]) && isfinite(P.q[0]) && isfinite(P.q[1]) && isfinite(P.q[2]) && isfinite(P.q[3]) &&
            isfinite(P.alpha);
  float qq = P.q[0] * P.q[0] + P.q[1] * P.q[1] + P.q[2] * P.q[2] + P.q[3] * P.q[3];
  return ok && qq > 0.f;
}

__device__ __forceinline__ bool load_params(const GaussPtrs &g, const int32_t *rank, int64_t i, GParams &P) {
  return load_params_r(g, i, g.u_means != nullptr ? rank[i] : -1, P);
}

__device__ __forceinline__ const float *color_ptr_r(const GaussPtrs &g, int64_t i, int r) {
  if (g.u_colors != nullptr && r >= 0) return g.u_colors + (int64_t)g.col_stride * r;
  return g.colors + (int64_t)g.col_stride * i;
}

__device__ __forceinline__ const float *color_ptr(const GaussPtrs &g, const int32_t *rank, int64_t i) {
  return color_ptr_r(g, i, g.u_colors != nullptr ? rank[i] : -1);
}

}  // namespace rtg
