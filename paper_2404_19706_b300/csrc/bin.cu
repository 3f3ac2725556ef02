// Projection and tile binning (Section 3.1 rendering on screen tiles; the unstable-mask
// passes use the 16 x 16 tiles of Supplement B, the render passes the tuned tile):
// per-tile masked-pixel counts and pixel lists, the unstable index, the EWA projection
// of every Gaussian into every frame, the exclusive scan of per-tile pair counts (and
// the work queue of the persistent schedule) and the emission of (depth, index) keys
// into per-tile buckets.
#include <mutex>

#include "kernels.cuh"
#include "project.cuh"

namespace rtg {

// --------------------------------------------------------------------------- setup + tile mask
// CTAs of kMaxTilePix threads over the (frame, tile)s of a grid of 2^tws x 2^ths pixel
// tiles, one thread per pixel: a CTA takes kMaxTilePix / 2^(tws+ths) consecutive tiles (so
// small tiles do not make thousands of tiny CTAs).  Counts the masked in-image pixels of
// each tile, clears its pair counter and, with `lists`, writes the tile's masked pixels
// (raster index within the tile) compacted in the tile's Z order (tile_order_pixel): the
// forward and backward give each 32 of them to one warp.  With `setup`, block 0 also
// publishes the cameras and clears the per-call counters.
// early: the kernel in front is the call's own frame decode, which reads only the sensor
// frame and writes only the targets; this pass reads the mask and writes the tile arrays,
// cameras and counters, so it runs whole before the wait on the decode (which it still
// makes before completing, so that later kernels find the targets written).
__global__ void __launch_bounds__(kMaxTilePix) k_tile_mask(FrameSet fs, Work w, const uint8_t *__restrict__ mask,
                                                           int T, int tiles_x, int tws, int ths, int setup,
                                                           int lists, long long nu_preset, int early) {
  if (!early) grid_dep_wait();
  __shared__ int s_wcnt[kMaxTilePix / 32];
  if (setup && blockIdx.x == 0) {
    for (int i = threadIdx.x; i < fs.F; i += blockDim.x) w.cams[i] = fs.cam[i];
    const int c = (int)threadIdx.x * kCounterStride;
    if ((int)threadIdx.x < kNumCounterSlots && c != kWinStable)
      w.counters[c] = (c == kNumUnstable && nu_preset >= 0) ? (unsigned long long)nu_preset : 0ull;
  }
  const int sh = tws + ths;  // log2 pixels per tile
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int tile = (int)blockIdx.x * (kMaxTilePix >> sh) + (tid >> sh);
  const int pix = tile_order_pixel(tid & ((1 << sh) - 1), tws, ths);  // threads take the tile in Z order
  const int FT = fs.F * T;
  const bool live = tile < FT;
  const int f = live ? tile / T : 0, lt = tile - f * T;
  const DevCam &cam = fs.cam[f];
  const int tx = lt % tiles_x, ty = lt / tiles_x;
  const int px = (tx << tws) + (pix & ((1 << tws) - 1)), py = (ty << ths) + (pix >> tws);
  bool in = live && px < cam.W && py < cam.H;
  if (in && mask != nullptr) in = mask[((int64_t)f * cam.H + py) * cam.W + px] != 0;
  const unsigned bal = __ballot_sync(0xffffffffu, in);
  if (lane == 0) s_wcnt[wid] = __popc(bal);
  __syncthreads();
  // warps of this tile: [w0, w0 + wpt) (a tile has at least 8 x 8 pixels, two warps)
  const int wpt = 1 << (sh - 5), w0 = wid & ~(wpt - 1);
  int before = 0, total = 0;
  for (int k = w0; k < w0 + wpt; ++k) {
    const int c = s_wcnt[k];
    before += k < wid ? c : 0;
    total += c;
  }
  if (lists && in) w.px_list[((int64_t)tile << sh) + before + __popc(bal & lanemask_lt())] = (uint8_t)pix;
  if (live && pix == 0) {
    w.tile_npix[tile] = (uint32_t)total;
    w.tile_count[tile] = 0u;
  }
  if (early) grid_dep_wait();
}

// --------------------------------------------------------------------------- unstable index
// Two-kernel scan: per-block counts, then each block adds its predecessors' counts.
// Each thread handles kRankPer consecutive flags (one 16-byte load when aligned), so a
// block of kRankThreads covers kRankPerBlock Gaussians.
constexpr int kRankThreads = 256, kRankPer = 16, kRankPerBlock = kRankThreads * kRankPer;

__device__ __forceinline__ uint32_t load_flags(const uint8_t *__restrict__ unstable, int64_t n, int64_t i0,
                                               uint8_t (&f)[kRankPer]) {
  uint32_t cnt = 0;
  if (i0 + kRankPer <= n && ((reinterpret_cast<uintptr_t>(unstable + i0) & 15u) == 0)) {
    const uint4 v = *reinterpret_cast<const uint4 *>(unstable + i0);
    const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < kRankPer; ++k) f[k] = (uint8_t)((wv[k >> 2] >> (8 * (k & 3))) & 0xffu);
  } else {
#pragma unroll
    for (int k = 0; k < kRankPer; ++k) f[k] = (i0 + k < n) ? unstable[i0 + k] : (uint8_t)0;
  }
#pragma unroll
  for (int k = 0; k < kRankPer; ++k) cnt += f[k] != 0;
  return cnt;
}

__global__ void __launch_bounds__(kRankThreads) k_rank_count(const uint8_t *__restrict__ unstable, int64_t n,
                                                             int32_t *__restrict__ block_cnt) {
  grid_dep_wait();
  __shared__ int s_warp[kRankThreads / 32];
  uint8_t fl[kRankPer];
  const int64_t i0 = ((int64_t)blockIdx.x * kRankThreads + threadIdx.x) * kRankPer;
  const int c = block_sum_int((int)load_flags(unstable, n, i0, fl), s_warp);
  if (threadIdx.x == 0) block_cnt[blockIdx.x] = c;
}

__global__ void __launch_bounds__(kRankThreads) k_rank_write(const uint8_t *__restrict__ unstable, int64_t n,
                                                             const int32_t *__restrict__ block_cnt,
                                                             int32_t *__restrict__ rank, int32_t *__restrict__ ids,
                                                             unsigned long long *nu_counter, int64_t *nu_out) {
  grid_dep_wait();
  __shared__ int s_warp[kRankThreads / 32];
  __shared__ int s_base;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // predecessors' total
  int acc = 0;
  for (int b = threadIdx.x; b < (int)blockIdx.x; b += kRankThreads) acc += block_cnt[b];
  acc = block_sum_int(acc, s_warp);
  if (threadIdx.x == 0) s_base = acc;
  __syncthreads();
  uint8_t fl[kRankPer];
  const int64_t i0 = ((int64_t)blockIdx.x * kRankThreads + threadIdx.x) * kRankPer;
  const int mine = (int)load_flags(unstable, n, i0, fl);
  // exclusive scan of the per-thread counts across the block
  int inc = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) s_warp[wid] = inc;
  __syncthreads();
  int before = s_base + inc - mine;
  for (int k = 0; k < wid; ++k) before += s_warp[k];
#pragma unroll
  for (int k = 0; k < kRankPer; ++k) {
    const int64_t i = i0 + k;
    if (i < n) {
      const bool u = fl[k] != 0;
      if (rank != nullptr) rank[i] = u ? before : -1;
      if (u && ids != nullptr) ids[before] = (int32_t)i;
      before += u;
    }
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kRankThreads - 1) {
    if (nu_counter != nullptr) nu_counter[kNumUnstable] = (unsigned long long)before;
    if (nu_out != nullptr) *nu_out = before;
  }
}

// --------------------------------------------------------------------------- tile rects
// Flattened warp walk.  Each lane of a warp holds one (frame, Gaussian) entry with a tile
// rectangle [tx0, tx1] x [ty0, ty1] (empty when tx1 < tx0) in the frame whose per-tile
// arrays start at fbase, rows of tiles_x tiles.  The rectangles are concatenated in lane
// order into one sequence of A tiles, which the warp takes 32 x kWalkRounds tiles per pass:
// a lane finds the rectangle that holds each of its tiles by a binary search over the
// warp's prefix of areas, then issues the loads (and later the slot atomics) of all its
// tiles of the pass before it waits for any.  A pass costs one L2 round trip per stage
// however the tiles are spread over the lanes, so a Gaussian near the camera that spans
// hundreds of tiles is walked by the whole warp in a few passes instead of holding it (and,
// through the block's reservation barrier, its block) for a chain of round trips.  All 32
// lanes call these functions together.
constexpr int kWalkRounds = 4;

struct WarpRects {
  int P;                          // exclusive prefix of the lanes' areas: this lane's first item
  int A;                          // the warp's total area (the same in every lane)
  int tx0, ty0, rw, fbase, tiles_x;  // this lane's rectangle
};

__device__ __forceinline__ WarpRects warp_rects(int tiles_x, int fbase, int tx0, int ty0, int tx1, int ty1) {
  const int lane = threadIdx.x & 31;
  const int rw = tx1 - tx0 + 1, area = (tx1 < tx0 || ty1 < ty0) ? 0 : rw * (ty1 - ty0 + 1);
  int incl = area;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  return WarpRects{incl - area, __shfl_sync(0xffffffffu, incl, 31), tx0, ty0, rw, fbase, tiles_x};
}

// Item `it` (0 <= it < A) of the warp's sequence: the lane whose rectangle holds it (the
// last lane whose first item is at most `it`; lanes with empty rectangles share their
// successor's first item and are passed over) and the item's index into the per-tile arrays.
__device__ __forceinline__ int warp_rect_item(const WarpRects &r, int it, int &owner) {
  int lo = 0;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1)
    if (__shfl_sync(0xffffffffu, r.P, lo + s) <= it) lo += s;
  owner = lo;
  const int j = it - __shfl_sync(0xffffffffu, r.P, lo);
  const int rw = __shfl_sync(0xffffffffu, r.rw, lo);
  const int tx0 = __shfl_sync(0xffffffffu, r.tx0, lo), ty0 = __shfl_sync(0xffffffffu, r.ty0, lo);
  const int fb = __shfl_sync(0xffffffffu, r.fbase, lo), tw = __shfl_sync(0xffffffffu, r.tiles_x, lo);
  const int yy = j / rw;
  return fb + (ty0 + yy) * tw + tx0 + (j - yy * rw);
}

// Tiles with masked pixels over the warp's rectangles: the warp total (in every lane); `vis`
// gets a bit per lane whose rectangle holds at least one.  all_on: every tile of every
// rectangle has pixels (a grid without a mask, rectangles clamped to the image), so the
// total is the area and nothing is loaded.
__device__ __forceinline__ uint32_t warp_count_rects(const uint32_t *__restrict__ npix, const WarpRects &r,
                                                     unsigned &vis, bool all_on = false) {
  const int lane = threadIdx.x & 31;
  uint32_t total = 0;
  vis = 0u;
  if (all_on) {
    vis = __ballot_sync(0xffffffffu, __shfl_down_sync(0xffffffffu, r.P, 1) > r.P || (lane == 31 && r.A > r.P));
    return (uint32_t)r.A;
  }
  for (int b0 = 0; b0 < r.A; b0 += 32 * kWalkRounds) {
    uint32_t v[kWalkRounds];
    int own[kWalkRounds];
#pragma unroll
    for (int u = 0; u < kWalkRounds; ++u) {
      const int it = b0 + u * 32 + lane;
      const int t = warp_rect_item(r, min(it, r.A - 1), own[u]);
      v[u] = it < r.A ? npix[t] : 0u;
    }
#pragma unroll
    for (int u = 0; u < kWalkRounds; ++u) {
      const bool on = v[u] != 0u;
      total += (uint32_t)__popc(__ballot_sync(0xffffffffu, on));
      vis |= __reduce_or_sync(0xffffffffu, on ? 1u << own[u] : 0u);
    }
  }
  return total;
}

// Stages one (global tile, slot, key lo, key hi) per masked tile over the warp's rectangles
// at positions first, first + 1, ... (`first`: the warp's reservation, the same in every
// lane; the keys are each owner lane's).  A tile's slots come from one atomic per distinct
// tile of a round (match.any): lanes of a warp hold neighbouring Gaussians and often share
// tiles, and the peers take consecutive slots.
__device__ __forceinline__ void warp_stage_rects(uint4 *__restrict__ stage, const uint32_t *__restrict__ npix,
                                                 uint32_t *__restrict__ tcount, const WarpRects &r, uint32_t klo,
                                                 uint32_t khi, unsigned long long first, int64_t max_pairs,
                                                 bool all_on = false) {
  const int lane = threadIdx.x & 31;
  unsigned long long pos = first;
  for (int b0 = 0; b0 < r.A; b0 += 32 * kWalkRounds) {
    int t[kWalkRounds], own[kWalkRounds];
    bool on[kWalkRounds];
#pragma unroll
    for (int u = 0; u < kWalkRounds; ++u) {
      const int it = b0 + u * 32 + lane;
      t[u] = warp_rect_item(r, min(it, r.A - 1), own[u]);
      on[u] = it < r.A && (all_on || npix[t[u]] != 0u);
    }
    unsigned peers[kWalkRounds];
    uint32_t base[kWalkRounds];
#pragma unroll
    for (int u = 0; u < kWalkRounds; ++u) {
      peers[u] = __match_any_sync(0xffffffffu, on[u] ? t[u] : -1 - lane);
      base[u] = 0u;
      if (on[u] && lane == __ffs(peers[u]) - 1) base[u] = atomicAdd(tcount + t[u], (uint32_t)__popc(peers[u]));
    }
#pragma unroll
    for (int u = 0; u < kWalkRounds; ++u) {
      const uint32_t b = __shfl_sync(0xffffffffu, base[u], __ffs(peers[u]) - 1);
      const uint32_t lo = __shfl_sync(0xffffffffu, klo, own[u]), hi = __shfl_sync(0xffffffffu, khi, own[u]);
      const unsigned bal = __ballot_sync(0xffffffffu, on[u]);
      if (on[u]) {
        const unsigned long long idx = pos + (unsigned long long)__popc(bal & lanemask_lt());
        if (idx < (unsigned long long)max_pairs)
          stage[idx] = make_uint4((uint32_t)t[u], b + (uint32_t)__popc(peers[u] & lanemask_lt()), lo, hi);
      }
      pos += (unsigned long long)__popc(bal);
    }
  }
}

// --------------------------------------------------------------------------- projection
// Two stages.  k_cull tests every (frame, Gaussian) with plain FP32 against the near plane
// and the guard band, with a relative margin so that it never drops a pair the exact test
// keeps, clears the tile count of the pairs it drops, and appends the rest to a dense
// candidate list (one atomic per warp).  k_project then runs the exact double-float
// projection over that list only, so its warps stay full.
// kSet selects the Gaussians considered (CullSet: all, unstable, stable).  With `ids` (the
// precomputed unstable list) the threads walk that list instead of all N; entries of other
// Gaussians keep their tile counts, which nothing reads before they are rewritten.
template <int kSet>
__global__ void __launch_bounds__(256) k_cull(GaussPtrs g, Work w, Prm prm, int F, const int32_t *__restrict__ ids,
                                              int64_t count) {
  grid_dep_wait();
  __shared__ uint32_t s_w[8];
  __shared__ unsigned long long s_base;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t N = g.n;
  int64_t i = t;
  bool live = t < N;
  if (ids != nullptr) {
    live = t < count;
    i = live ? (int64_t)ids[t] : 0;
  } else if (kSet == kCullUnstable && live) {
    live = g.unstable[i] != 0;
  } else if (kSet == kCullStable && live) {
    live = g.unstable[i] == 0;
  }
  float p[3] = {0.f, 0.f, 0.f};
  if (live) {
    const float *pm = g.means + 3 * i;
    if (g.u_means != nullptr) {
      const int r = w.rank[i];
      if (r >= 0) pm = g.u_means + 3 * (int64_t)r;
    }
    p[0] = pm[0]; p[1] = pm[1]; p[2] = pm[2];
  }
  for (int f = 0; f < F; ++f) {
    bool cand = false;
    if (live) {
      const DevCam &cam = w.cams[f];
      const float d0 = p[0] - cam.t[0], d1 = p[1] - cam.t[1], d2 = p[2] - cam.t[2];
      const float X = cam.R[0] * d0 + cam.R[3] * d1 + cam.R[6] * d2;
      const float Y = cam.R[1] * d0 + cam.R[4] * d1 + cam.R[7] * d2;
      const float Z = cam.R[2] * d0 + cam.R[5] * d1 + cam.R[8] * d2;
      const float tol = 1e-4f * (fabsf(d0) + fabsf(d1) + fabsf(d2)) + 1e-6f;
      cand = Z > prm.near_z - tol && fabsf(X) <= cam.lim_x * (Z + tol) + tol &&
             fabsf(Y) <= cam.lim_y * (Z + tol) + tol;
    }
    if ((ids != nullptr ? live : i < N) && !cand) w.ntiles[(int64_t)f * N + i] = 0u;
    const unsigned long long slot = block_reserve(w.counters + kCand, cand ? 1u : 0u, s_w, &s_base);
    if (cand) w.cand[slot] = (uint32_t)((int64_t)f * N + i);
  }
}

// kMode = kProjForward: records and pairs for the masked tiles of a forward.
// kMode = kProjMask: the unstable-mask pass (only unstable Gaussians reach this kernel
//   through k_cull<true>); no gradient rows are cleared and no visibility is counted.
// kMode = kProjFused: first half of rtg_render_forward_masked: every projected candidate
//   gets its records (its tile count is set later by k_bin, once the mask is known), and
//   only the unstable ones are binned, into every tile, for the coverage test.
// kMode = kProjWindow: rtg_window_begin: records only, and every projected candidate is
//   appended to the window's list (stable Gaussians reach this kernel through the cull).
// Every pair (candidate, masked tile) is staged as (tile, slot, key): the block reserves its
// staging range with one atomic, and each pair's slot in its tile bucket is the value the
// tile counter returns, so the later scatter into buckets needs no atomics.
// With `ids` (the precomputed unstable list, nids entries) the kernel walks every (frame,
// listed Gaussian) itself instead of the cull's candidates: the exact projection culls them,
// one launch fewer for a short list.
template <int C, int kMode>
__global__ void __launch_bounds__(256) k_project(GaussPtrs g, Work w, Prm prm, int T, int64_t max_pairs,
                                                 const int32_t *__restrict__ ids, int64_t nids, int F) {
  grid_dep_wait();
  constexpr int H4 = (C <= 4) ? 3 : 4;
  constexpr int G2 = (C <= 5) ? 16 : 20;
  __shared__ uint32_t s_w[16];
  __shared__ unsigned long long s_base;
  const int64_t N = g.n;
  const int64_t ncand = ids != nullptr ? (int64_t)F * nids : (int64_t)w.counters[kCand];
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < ncand; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = base + threadIdx.x;
    uint32_t e = 0;
    int f = 0, tx0 = 0, tx1 = -1, ty0 = 0, ty1 = -1;
    int64_t i = 0;
    int rkk = -1;  // the compact unstable row, known when walking the unstable list (rank[ids[j]] = j)
    bool ok = false;
    Projected o;
    GParams P;
    float col[C];
    if (k < ncand) {
      if (ids != nullptr) {
        f = (int)(k / nids);
        rkk = (int)(k - (int64_t)f * nids);
        i = (int64_t)ids[rkk];
        e = (uint32_t)((int64_t)f * N + i);
      } else {
        e = w.cand[k];
        f = (int)(e / (uint64_t)N);
        i = (int64_t)e - (int64_t)f * N;
        rkk = w.rank[i];
      }
      ok = load_params_r(g, i, rkk, P);
      const float *cp = color_ptr_r(g, i, rkk);
      if (C == 3 && g.sh_degree > 0) {  // the colour seen from this frame's camera
        float c3[3];
        sh_color(g.sh_degree, cp, P.p, w.cams[f].t, c3);
#pragma unroll
        for (int c = 0; c < C; ++c) col[c] = c3[c < 3 ? c : 0];
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) col[c] = cp[c];
      }
#pragma unroll
      for (int c = 0; c < C; ++c) ok = ok && isfinite(col[c]);
      if (ok) {
        float R[9];
        const float rq = rsqrtf(P.q[0] * P.q[0] + P.q[1] * P.q[1] + P.q[2] * P.q[2] + P.q[3] * P.q[3]);
        quat_to_rot(P.q[0] * rq, P.q[1] * rq, P.q[2] * rq, P.q[3] * rq, R);
        const int kmin = argmin3(P.s[0], P.s[1], P.s[2]);
        ok = project_gaussian(w.cams[f], prm, P, R, kmin, o);
      }
      if (ok) {
        // the forward bins into the render grid, the mask passes into the 16 x 16 rule grid
        const DevCam &cam = w.cams[f];
        const int tws = kMode == kProjForward ? cam.tws : kTileShift;
        const int ths = kMode == kProjForward ? cam.ths : kTileShift;
        tx0 = o.x0 >> tws; tx1 = o.x1 >> tws; ty0 = o.y0 >> ths; ty1 = o.y1 >> ths;
        if (kMode == kProjWindow || (kMode == kProjFused && g.unstable[i] == 0)) tx1 = tx0 - 1;  // no pairs
      }
    }
    const int tiles_x = (k < ncand) ? (kMode == kProjForward ? w.cams[f].tiles_x : w.cams[f].mtiles_x) : 0;
    const WarpRects wr = warp_rects(tiles_x, f * T, tx0, ty0, tx1, ty1);
    // the mask passes bin into the 16 x 16 grid of a call without a mask: every tile of a
    // (clamped) rectangle has pixels
    constexpr bool all_on = kMode == kProjFused || kMode == kProjMask;
    unsigned vis = 0u;
    const uint32_t wtotal = warp_count_rects(w.tile_npix, wr, vis, all_on);
    const bool visible = (vis >> (threadIdx.x & 31)) & 1u;
    if (kMode == kProjWindow) {  // one atomic per block appends the projected entries
      const unsigned long long slot = block_reserve(w.counters + kWinStable, ok ? 1u : 0u, s_w, &s_base);
      if (ok) w.scand[slot] = e;
    }
    // block-level reservation of the warps' staging ranges (one atomic per block)
    const unsigned long long first = __shfl_sync(
        0xffffffffu,
        block_reserve(w.counters + kStaged, (threadIdx.x & 31) == 0 ? wtotal : 0u, s_w, &s_base,
                      kMode == kProjForward ? w.counters + kVisible : nullptr, visible ? 1u : 0u),
        0);
    if (ok && (visible || kMode == kProjFused || kMode == kProjWindow)) {
      const int rk = rkk;
      float4 *hot = w.rec_hot + ((int64_t)f * N + i) * H4;
      hot[0] = make_float4(o.mux.hi, o.muy.hi, o.mux.lo, o.muy.lo);
      hot[1] = make_float4(o.u11, o.u12, o.u22, P.alpha);
      float cc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
      for (int c = 0; c < C; ++c) cc[c] = col[c];
      // C = 3: the spare fourth slot carries the unstable rank for the backward
      hot[2] = make_float4(cc[0], cc[1], cc[2], C == 3 ? __int_as_float(rk) : cc[3]);
      if (H4 == 4) hot[3] = make_float4(cc[4], cc[5], cc[6], cc[7]);
      w.rec_box[(int64_t)f * N + i] = make_float2(o.rx, o.ry);
      float4 *cold = w.rec_cold + ((int64_t)f * N + i) * 2;
      cold[0] = make_float4(o.n[0], o.n[1], o.n[2], o.d0);
      cold[1] = make_float4(o.Z, __int_as_float(rk), __uint_as_float((uint32_t)o.x0 | ((uint32_t)o.y0 << 16)),
                            __uint_as_float((uint32_t)o.x1 | ((uint32_t)o.y1 << 16)));
      if (kMode != kProjMask && kMode != kProjWindow && rk >= 0) {
        float4 *g2 = reinterpret_cast<float4 *>(w.grad2d + ((int64_t)f * N + rk) * G2);
#pragma unroll
        for (int q = 0; q < G2 / 4; ++q) g2[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    // kProjFused: 1 marks "projected" for k_bin, which writes the final visibility
    if (k < ncand) w.ntiles[e] = (kMode == kProjFused || kMode == kProjWindow) ? (ok ? 1u : 0u) : (visible ? 1u : 0u);
    // the records are written; now the pairs
    warp_stage_rects(w.stage, w.tile_npix, w.tile_count, wr, (uint32_t)i, ok ? __float_as_uint(o.Z) : 0u, first,
                     max_pairs, all_on);
  }
}

// Bins projected (frame, Gaussian) entries into the render tiles that have masked pixels
// (tile_npix holds each tile's masked-pixel count): the second half of
// rtg_render_forward_masked (the cull's candidates that the fused projection marked
// projected), and, with an open window, the cached stable entries, whose records the window
// pass wrote.  Index k < ncand walks the candidates, the rest the window's list.
__global__ void __launch_bounds__(256) k_bin(Work w, int64_t N, int T, int64_t max_pairs, int cands, int stable) {
  grid_dep_wait();
  __shared__ uint32_t s_w[16];
  __shared__ unsigned long long s_base;
  if (w.counters[kSkip] != 0ull) return;
  const int64_t ncand = cands ? (int64_t)w.counters[kCand] : 0;
  const int64_t total = ncand + (stable ? (int64_t)w.counters[kWinStable] : 0);
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < total; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = base + threadIdx.x;
    uint32_t e = 0;
    int f = 0, tx0 = 0, tx1 = -1, ty0 = 0, ty1 = -1, tiles_x = 0;
    float4 c1 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k < total) {
      e = k < ncand ? w.cand[k] : w.scand[k - ncand];
      if (k >= ncand || w.ntiles[e] != 0u) {
        f = (int)(e / (uint64_t)N);
        const DevCam &cam = w.cams[f];
        tiles_x = cam.tiles_x;
        c1 = w.rec_cold[(int64_t)e * 2 + 1];
        const uint32_t lo = __float_as_uint(c1.z), hi = __float_as_uint(c1.w);
        tx0 = (int)(lo & 0xffffu) >> cam.tws; ty0 = (int)(lo >> 16) >> cam.ths;
        tx1 = (int)(hi & 0xffffu) >> cam.tws; ty1 = (int)(hi >> 16) >> cam.ths;
      }
    }
    const WarpRects wr = warp_rects(tiles_x, f * T, tx0, ty0, tx1, ty1);
    unsigned vis = 0u;
    const uint32_t wtotal = warp_count_rects(w.tile_npix, wr, vis);
    const bool visible = (vis >> (threadIdx.x & 31)) & 1u;
    const unsigned long long first = __shfl_sync(
        0xffffffffu,
        block_reserve(w.counters + kStaged, (threadIdx.x & 31) == 0 ? wtotal : 0u, s_w, &s_base,
                      w.counters + kVisible, visible ? 1u : 0u),
        0);
    if (k < total) w.ntiles[e] = visible ? 1u : 0u;
    warp_stage_rects(w.stage, w.tile_npix, w.tile_count, wr, (uint32_t)((int64_t)e - (int64_t)f * N),
                     __float_as_uint(c1.x), first, max_pairs);
  }
}

__global__ void k_window_reset(Work w) { grid_dep_wait(); w.counters[kWinStable] = 0ull; }

// --------------------------------------------------------------------------- tile scan
// Cost class of a tile list of n records for the persistent schedule's queue: 0 for an
// empty list, else four classes per octave of n (so the order is by n to within 19%).
__device__ __forceinline__ int queue_class(uint32_t n) {
  if (n == 0u) return 0;
  const int lg = 31 - __clz(n);
  const int sub = lg >= 2 ? (int)((n >> (lg - 2)) & 3u) : (int)((n << (2 - lg)) & 3u);
  return 1 + 4 * lg + sub;
}

// One CTA: exclusive scan of the per-tile pair counts into bucket offsets, capacity check.
// With gshift >= 0 it also lays out the persistent schedule's work: one item per 32
// masked pixels of each tile (2^gshift groups per tile at most), ordered by the tile's
// list length, longest first (a counting sort on queue_class; the order within a class
// is arbitrary and does not affect any result).
// With `extra` (an open window's cached stable lists), a tile with masked pixels holds
// tile_count[t] unstable pairs and extra[t] stable ones: its list length is their sum.
__device__ __forceinline__ uint32_t list_len(const Work &w, const uint32_t *extra, int t) {
  return w.tile_count[t] + ((extra != nullptr && w.tile_npix[t] != 0u) ? extra[t] : 0u);
}

// Starts of the queue's cost classes, costliest (highest class) first: s_cls holds each
// class's count on entry and its first queue position on return.  One warp: lane l takes
// kPer consecutive classes from the top, the lanes' sums are scanned with shuffles.
// Returns the total in every lane.
__device__ __forceinline__ uint32_t class_starts(uint32_t *s_cls, int lane) {
  constexpr int kPer = (kQueueClasses + 31) / 32;
  uint32_t c[kPer], local = 0u;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int k = kQueueClasses - 1 - (lane * kPer + j);
    c[j] = k >= 0 ? s_cls[k] : 0u;
    local += c[j];
  }
  uint32_t inc = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  uint32_t run = inc - local;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int k = kQueueClasses - 1 - (lane * kPer + j);
    if (k >= 0) s_cls[k] = run;
    run += c[j];
  }
  return __shfl_sync(0xffffffffu, inc, 31);
}

// Thread t owns tiles [t * per, t * per + per) (per <= kScanSingleMax / 1024): their counts
// are loaded once, all at once, and kept in registers for the offsets and the queue.
// kEmit: the scatter of the staged pairs into their buckets is fused in.  Every CTA scans
// the tiles itself into shared memory (the scan is small and deterministic, so all CTAs
// agree) and scatters its share of the pairs from there; CTA 0 alone writes the offsets,
// counters and item queue.  No CTA waits on another.
constexpr int kScanPer = kScanSingleMax / 1024;

template <bool kEmit>
__global__ void __launch_bounds__(1024) k_scan_tiles(Work w, int FT, int64_t max_pairs, int gshift,
                                                     const uint32_t *__restrict__ extra) {
  grid_dep_wait();
  extern __shared__ uint32_t s_off[];  // kEmit: the FT + 1 bucket offsets
  __shared__ unsigned long long s_total;
  const bool lead = blockIdx.x == 0;
  __shared__ unsigned long long s_warp[32];
  __shared__ uint32_t s_wmax[32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int per = (FT + 1023) / 1024;
  const int b = tid * per, e = min(FT, b + per);
  uint32_t len[kScanPer], npx[kScanPer];
#pragma unroll
  for (int u = 0; u < kScanPer; ++u) {
    const int t = b + u;
    const bool in = u < per && t < e;
    const uint32_t cnt = in ? w.tile_count[t] : 0u;
    npx[u] = in ? w.tile_npix[t] : 0u;
    const uint32_t ex = (in && extra != nullptr) ? extra[t] : 0u;
    len[u] = cnt + (npx[u] != 0u ? ex : 0u);
  }
  unsigned long long local = 0, npix = 0;
  uint32_t mx = 0;
#pragma unroll
  for (int u = 0; u < kScanPer; ++u) {
    local += len[u];
    npix += npx[u];
    mx = max(mx, len[u]);
  }
  // inclusive warp scan of `local`
  unsigned long long inc = local;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  unsigned long long np = npix;
  for (int o = 16; o > 0; o >>= 1) np += __shfl_xor_sync(0xffffffffu, np, o);
  __shared__ unsigned long long s_pix[32];
  if (lane == 31) s_warp[wid] = inc;
  if (lane == 0) {
    s_wmax[wid] = mx;
    s_pix[wid] = np;
  }
  __syncthreads();
  if (wid == 0) {
    unsigned long long v = s_warp[lane];
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    s_warp[lane] = v;  // inclusive totals per warp
    uint32_t m = s_wmax[lane];
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    s_wmax[lane] = m;
    unsigned long long pz = s_pix[lane];
    for (int o = 16; o > 0; o >>= 1) pz += __shfl_xor_sync(0xffffffffu, pz, o);
    s_pix[lane] = pz;
  }
  __syncthreads();
  unsigned long long run = (wid > 0 ? s_warp[wid - 1] : 0ull) + inc - local;
#pragma unroll
  for (int u = 0; u < kScanPer; ++u) {
    if (b + u < e) {
      if (lead) w.tile_offset[b + u] = (uint32_t)run;
      if (kEmit) s_off[b + u] = (uint32_t)run;
    }
    run += len[u];
  }
  if (tid == 1023) {  // the last thread's running offset is the pair total
    const unsigned long long total = run;
    s_total = total;
    if (lead) {
      w.tile_offset[FT] = (uint32_t)total;
      w.counters[kPairs] = total;
      w.counters[kMaskedPix] = s_pix[0];
      w.counters[kMaxTilePairs] = s_wmax[0];
      if (total > (unsigned long long)max_pairs || total > 0xffffffffull) {
        w.counters[kSkip] = 1ull;
        atomicCAS(w.status, 0u, (uint32_t)(int32_t)RTG_ERR_WORKSPACE);
      }
    }
  }
  if (kEmit) {
    __syncthreads();
    if (s_total <= (unsigned long long)max_pairs && s_total <= 0xffffffffull) {
      // with a queue to lay out, the lead CTA (whose queue ends the kernel) leaves the
      // scatter to the others
      const bool aside = gshift >= 0 && gridDim.x > 1;
      if (!(aside && lead)) {
        const int64_t nb = aside ? gridDim.x - 1 : gridDim.x, bi = aside ? blockIdx.x - 1 : blockIdx.x;
        const int64_t npairs = (int64_t)w.counters[kStaged];
        for (int64_t k = bi * blockDim.x + tid; k < npairs; k += nb * blockDim.x) {
          const uint4 st = w.stage[k];
          w.keys[(int64_t)s_off[st.x] + st.y] = ((unsigned long long)st.w << 32) | (unsigned long long)st.z;
        }
      }
    }
  }
  if (gshift < 0 || !lead) return;
  // ---- item queue, and the sort's tile order (the tiles with keys, by the same classes)
  __shared__ uint32_t s_cls[kQueueClasses], s_tcls[kQueueClasses];
  for (int k = tid; k < kQueueClasses; k += 1024) s_cls[k] = s_tcls[k] = 0u;
  __syncthreads();
#pragma unroll
  for (int u = 0; u < kScanPer; ++u) {
    if (npx[u] != 0u) atomicAdd(&s_cls[queue_class(len[u])], (npx[u] + 31u) >> 5);
    if (len[u] != 0u) atomicAdd(&s_tcls[queue_class(len[u])], 1u);
  }
  __syncthreads();
  if (wid == 0) {  // start of each class, classes in decreasing cost
    const uint32_t r = class_starts(s_cls, lane);
    if (lane == 0) {
      w.counters[kItems] = r;
      w.counters[kQFwd] = 0ull;
      w.counters[kQBwd] = 0ull;
      for (int b = 0; b < kSegBins; ++b) w.counters[kBSeg0 + b * kCounterStride] = 0ull;
    }
  } else if (wid == 1) {
    const uint32_t r = class_starts(s_tcls, lane);
    if (lane == 0) w.counters[kSortTiles] = r;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < kScanPer; ++u) {
    if (len[u] != 0u) w.tile_order[atomicAdd(&s_tcls[queue_class(len[u])], 1u)] = (uint32_t)(b + u);
    if (npx[u] == 0u) continue;
    const uint32_t ng = (npx[u] + 31u) >> 5;
    const uint32_t pos = atomicAdd(&s_cls[queue_class(len[u])], ng);
    for (uint32_t g = 0; g < ng; ++g) w.items[pos + g] = ((uint32_t)(b + u) << 3) | g;
  }
}

// --------------------------------------------------------------------------- emission
// Scatters every staged pair into its tile bucket: key = (IEEE bits of z_c) << 32 | i.
// Positive floats order like their bit patterns, so sorting a bucket by key orders it by
// depth, then by index.
__global__ void __launch_bounds__(256) k_emit(Work w) {
  grid_dep_wait();
  if (w.counters[kSkip] != 0ull) return;
  const int64_t npairs = (int64_t)w.counters[kStaged];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < npairs; k += (int64_t)gridDim.x * blockDim.x) {
    const uint4 st = w.stage[k];
    w.keys[(int64_t)w.tile_offset[st.x] + st.y] = ((unsigned long long)st.w << 32) | (unsigned long long)st.z;
  }
}

void launch_tile_mask(const FrameSet &fs, const Work &w, const uint8_t *mask, int T, int tiles_x, int tws, int ths,
                      bool setup, bool lists, long long nu_preset, cudaStream_t s, bool early) {
  const int per = kMaxTilePix >> (tws + ths);  // tiles per CTA
  launch(k_tile_mask, (fs.F * T + per - 1) / per, kMaxTilePix, 0, s, fs, w, mask, T, tiles_x, tws, ths, setup ? 1 : 0,
         lists ? 1 : 0, nu_preset, early ? 1 : 0);
}

void launch_rank(const uint8_t *unstable, int64_t n, int32_t *block_cnt, int32_t *rank, int32_t *ids,
                 unsigned long long *nu_counter, int64_t *nu_out, cudaStream_t s) {
  if (n <= 0) return;
  const int nb = (int)((n + kRankPerBlock - 1) / kRankPerBlock);  // <= ceil(n / kScanBlock) entries of block_cnt
  launch(k_rank_count, nb, kRankThreads, 0, s, unstable, n, block_cnt);
  launch(k_rank_write, nb, kRankThreads, 0, s, unstable, n, block_cnt, rank, ids, nu_counter, nu_out);
}

// Lists of the unstable Gaussians at most this long (times the frames) are projected
// without the cull pass.
constexpr int64_t kDirectProjectMax = 1 << 18;

void launch_project(const GaussPtrs &g, const Work &w, const Prm &prm, int F, int T, int mode, int cull_set,
                    int64_t max_pairs, cudaStream_t s) {
  if (g.n <= 0) return;
  const unsigned nb = (unsigned)((g.n + 255) / 256);
  const bool direct = cull_set == kCullUnstable && g.rank_map != nullptr &&
                      (mode == kProjForward || mode == kProjMask) && (int64_t)F * g.n_unstable <= kDirectProjectMax;
  const int32_t *dids = direct ? g.unstable_ids : nullptr;
  const int64_t dn = direct ? g.n_unstable : 0;
  if (direct) {
    // the projection walks the unstable list itself
  } else if (cull_set == kCullUnstable) {
    if (g.rank_map != nullptr) {
      if (g.n_unstable > 0)
        launch(k_cull<kCullUnstable>, (unsigned)((g.n_unstable + 255) / 256), 256, 0, s, g, w, prm, F, g.unstable_ids,
                                                                                   g.n_unstable);
    } else {
      launch(k_cull<kCullUnstable>, nb, 256, 0, s, g, w, prm, F, nullptr, 0);
    }
  } else if (cull_set == kCullStable) {
    launch(k_cull<kCullStable>, nb, 256, 0, s, g, w, prm, F, nullptr, 0);
  } else {
    launch(k_cull<kCullAll>, nb, 256, 0, s, g, w, prm, F, nullptr, 0);
  }
#define RTG_PROJ(CC, MM)                                                                  \
  launch(k_project<CC, MM>, resident_grid((const void *)k_project<CC, MM>, 256), 256, 0, s, g, w, prm, T, \
         max_pairs, dids, dn, F)
#define RTG_PROJ_C(CC)                              \
  switch (mode) {                                   \
    case kProjForward: RTG_PROJ(CC, kProjForward); break; \
    case kProjMask: RTG_PROJ(CC, kProjMask); break;       \
    case kProjFused: RTG_PROJ(CC, kProjFused); break;     \
    default: RTG_PROJ(CC, kProjWindow); break;            \
  }
  if (g.C == 3) {
    RTG_PROJ_C(3)
  } else {
    RTG_PROJ_C(8)
  }
#undef RTG_PROJ_C
#undef RTG_PROJ
}

void launch_bin(const Work &w, int64_t N, int T, int64_t max_pairs, bool cands, bool stable, cudaStream_t s) {
  if (N <= 0) return;
  launch(k_bin, resident_grid((const void *)k_bin, 256), 256, 0, s, w, N, T, max_pairs, cands ? 1 : 0,
                                                                stable ? 1 : 0);
}

void launch_window_reset(const Work &w, cudaStream_t s) { launch(k_window_reset, 1, 1, 0, s, w); }

// ---- multi-block tile scan (many tiles: batched keyframes at high resolution).  Three
// kernels, none of which waits on another block: per-block partials, one CTA that turns
// them into block bases and per-(block, class) queue starts and writes the totals, and a
// per-block pass that writes the offsets and scatters the queue items.  Thread t of block b
// owns tiles b * kScanBlockTiles + 4t .. + 3.
// With `requeue` they rebuild only the queue, for pixel lists narrowed after the forward:
// the list lengths come from the forward's offsets, which stay as they are, as do the totals.

__device__ __forceinline__ uint32_t scan_len(const Work &w, const uint32_t *extra, int t, int requeue) {
  return requeue ? w.tile_offset[t + 1] - w.tile_offset[t] : list_len(w, extra, t);
}

__global__ void __launch_bounds__(1024) k_scan_part(Work w, int FT, int gshift, const uint32_t *__restrict__ extra,
                                                    int requeue) {
  grid_dep_wait();
  __shared__ unsigned long long s_a[32], s_b[32];
  __shared__ uint32_t s_m[32];
  __shared__ uint32_t s_cls[kQueueClasses];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int k = tid; k < kQueueClasses; k += 1024) s_cls[k] = 0u;
  __syncthreads();
  const int t0 = blockIdx.x * kScanBlockTiles + tid * 4;
  unsigned long long len = 0, np = 0;
  uint32_t mx = 0;
  for (int t = t0; t < min(FT, t0 + 4); ++t) {
    const uint32_t l = scan_len(w, extra, t, requeue), p = w.tile_npix[t];
    len += l;
    np += p;
    mx = max(mx, l);
    if (gshift >= 0 && p != 0u) atomicAdd(&s_cls[queue_class(l)], (p + 31u) >> 5);
  }
  for (int o = 16; o > 0; o >>= 1) {
    len += __shfl_xor_sync(0xffffffffu, len, o);
    np += __shfl_xor_sync(0xffffffffu, np, o);
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (lane == 0) {
    s_a[wid] = len;
    s_b[wid] = np;
    s_m[wid] = mx;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long a = 0, b = 0;
    uint32_t m = 0;
    for (int k = 0; k < 32; ++k) {
      a += s_a[k];
      b += s_b[k];
      m = max(m, s_m[k]);
    }
    w.scan_part[blockIdx.x * 4 + 0] = a;
    w.scan_part[blockIdx.x * 4 + 1] = b;
    w.scan_part[blockIdx.x * 4 + 2] = m;
  }
  if (gshift >= 0)
    for (int k = tid; k < kQueueClasses; k += 1024) w.scan_hist[blockIdx.x * kQueueClasses + k] = s_cls[k];
}

__global__ void __launch_bounds__(1024) k_scan_bases(Work w, int FT, int64_t max_pairs, int gshift, int B,
                                                     int requeue) {
  grid_dep_wait();
  __shared__ unsigned long long s_w[32];
  __shared__ uint32_t s_start[kQueueClasses];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (!requeue) {  // block bases and totals
    // exclusive prefix of the block pair totals (B <= 1024)
    const unsigned long long v = tid < B ? w.scan_part[tid * 4] : 0ull;
    unsigned long long inc = v;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    unsigned long long pre = 0;
    for (int k = 0; k < wid; ++k) pre += s_w[k];
    if (tid < B) w.scan_part[tid * 4 + 3] = pre + inc - v;
    if (tid == 0) {
      unsigned long long total = 0, total_pix = 0, mx = 0;
      for (int b = 0; b < B; ++b) {
        total += w.scan_part[b * 4 + 0];
        total_pix += w.scan_part[b * 4 + 1];
        mx = max(mx, w.scan_part[b * 4 + 2]);
      }
      w.tile_offset[FT] = (uint32_t)total;
      w.counters[kPairs] = total;
      w.counters[kMaskedPix] = total_pix;
      w.counters[kMaxTilePairs] = mx;
      if (total > (unsigned long long)max_pairs || total > 0xffffffffull) {
        w.counters[kSkip] = 1ull;
        atomicCAS(w.status, 0u, (uint32_t)(int32_t)RTG_ERR_WORKSPACE);
      }
    }
  }
  if (gshift < 0) return;
  // queue: class totals, class starts in decreasing cost, then each block's start per class
  if (tid < kQueueClasses) {
    uint32_t c = 0;
    for (int b = 0; b < B; ++b) c += w.scan_hist[b * kQueueClasses + tid];
    s_start[tid] = c;
  }
  __syncthreads();
  if (tid < 32) {
    const uint32_t run = class_starts(s_start, tid);
    if (tid == 0) {
      w.counters[kItems] = run;
      w.counters[kQFwd] = 0ull;
      w.counters[kQBwd] = 0ull;
      for (int b = 0; b < kSegBins; ++b) w.counters[kBSeg0 + b * kCounterStride] = 0ull;
    }
  }
  __syncthreads();
  if (tid < kQueueClasses) {
    uint32_t run = s_start[tid];
    for (int b = 0; b < B; ++b) {
      const uint32_t c = w.scan_hist[b * kQueueClasses + tid];
      w.scan_hist[b * kQueueClasses + tid] = run;
      run += c;
    }
  }
}

__global__ void __launch_bounds__(1024) k_scan_write(Work w, int FT, int gshift, const uint32_t *__restrict__ extra,
                                                     int requeue) {
  grid_dep_wait();
  __shared__ unsigned long long s_w[32];
  __shared__ uint32_t s_cur[kQueueClasses];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (gshift >= 0)
    for (int k = tid; k < kQueueClasses; k += 1024) s_cur[k] = w.scan_hist[blockIdx.x * kQueueClasses + k];
  const int t0 = blockIdx.x * kScanBlockTiles + tid * 4, t1 = min(FT, t0 + 4);
  uint32_t l[4] = {0u, 0u, 0u, 0u};
  unsigned long long mine = 0;
  for (int t = t0; t < t1; ++t) {
    l[t - t0] = scan_len(w, extra, t, requeue);
    mine += l[t - t0];
  }
  unsigned long long inc = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) s_w[wid] = inc;
  __syncthreads();
  if (!requeue) {
    unsigned long long run = w.scan_part[blockIdx.x * 4 + 3] + inc - mine;
    for (int k = 0; k < wid; ++k) run += s_w[k];
    for (int t = t0; t < t1; ++t) {
      w.tile_offset[t] = (uint32_t)run;
      run += l[t - t0];
    }
  }
  if (gshift < 0) return;
  for (int t = t0; t < t1; ++t) {
    const uint32_t np = w.tile_npix[t];
    if (np == 0u) continue;
    const uint32_t ng = (np + 31u) >> 5;
    const uint32_t pos = atomicAdd(&s_cur[queue_class(l[t - t0])], ng);
    for (uint32_t g = 0; g < ng; ++g) w.items[pos + g] = ((uint32_t)t << 3) | g;
  }
}

void launch_scan_tiles(const Work &w, int FT, int64_t max_pairs, int gshift, const uint32_t *extra, cudaStream_t s,
                       bool emit) {
  if (FT <= kScanSingleMax) {
    if (emit)  // one CTA per SM, each scattering its share of the pairs
      launch(k_scan_tiles<true>, (unsigned)resident_grid((const void *)k_scan_tiles<true>, 1024,
                                                         (size_t)(FT + 1) * 4),
             1024, (size_t)(FT + 1) * 4, s, w, FT, max_pairs, gshift, extra);
    else
      launch(k_scan_tiles<false>, 1, 1024, 0, s, w, FT, max_pairs, gshift, extra);
    return;
  }
  const int B = (FT + kScanBlockTiles - 1) / kScanBlockTiles;  // <= 1024 (capacity check)
  launch(k_scan_part, B, 1024, 0, s, w, FT, gshift, extra, 0);
  launch(k_scan_bases, 1, 1024, 0, s, w, FT, max_pairs, gshift, B, 0);
  launch(k_scan_write, B, 1024, 0, s, w, FT, gshift, extra, 0);
  if (emit) launch_emit(w, s);
}

void launch_requeue(const Work &w, int FT, int gshift, cudaStream_t s) {
  const int B = (FT + kScanBlockTiles - 1) / kScanBlockTiles;
  launch(k_scan_part, B, 1024, 0, s, w, FT, gshift, nullptr, 1);
  launch(k_scan_bases, 1, 1024, 0, s, w, FT, 0, gshift, B, 1);
  launch(k_scan_write, B, 1024, 0, s, w, FT, gshift, nullptr, 1);
}

void launch_emit(const Work &w, cudaStream_t s) {
  launch(k_emit, resident_grid((const void *)k_emit, 256), 256, 0, s, w);
}

int resident_grid(const void *kernel, int block, size_t smem) {
  struct Entry {
    const void *kernel;
    int device, block, grid;
  };
  static std::mutex mu;
  static Entry cache[64];
  static int n = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  for (int k = 0; k < n; ++k)
    if (cache[k].kernel == kernel && cache[k].device == dev && cache[k].block == block) return cache[k].grid;
  int sms = 0, per = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 148;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, block, smem) != cudaSuccess || per < 1) per = 1;
  cudaGetLastError();
  const int grid = sms * per;
  if (n < 64) cache[n++] = Entry{kernel, dev, block, grid};
  return grid;
}

namespace {
thread_local bool tl_overlap = true;  // calls without a context launch with overlap
}
bool launch_overlap() { return tl_overlap; }
void set_launch_overlap(bool on) { tl_overlap = on; }

}  // namespace rtg
