// Forward compositing (Section 3.1): per render tile, the masked pixels composite the
// tile's front-to-back list: colour by alpha blending (Eq. 1) with the footprint of
// Eq. 2 and transmission of Eq. 3, stopping before a fragment that would take the
// transmission below t_eps.  Each pixel takes its depth from the first processed
// fragment with f > delta_alpha (the opaque-disc hit), through the ray/disc-plane
// intersection of Eq. 4 and the cases of Eq. 5.  Only the masked pixels of a tile are
// rendered (only pixels covered by unstable Gaussians, Supplement B): the tile-mask pass
// compacted them into a list, and each warp works alone on 32 of them.  It walks the
// tile's list in batches of B records and keeps only the records whose support box, and
// then whose footprint ellipse (reaches_box), reaches the warp's pixel box.  Both tests are
// conservative, so the result is that of the per-pixel alpha_min test.  A warp stops as soon as all its pixels have stopped.
// Two schedules share that per-warp body: one CTA per tile (one warp per 32 masked
// pixels), or persistent warps that take (tile, group) items from the cost-ordered queue
// spanning every frame of the call.
#include <type_traits>

#include "kernels.cuh"
#include "project.cuh"

namespace rtg {

struct FwdOut {
  float *color, *depth, *alpha;
  int32_t *index_map;
  const float *tcolor, *tdepth;  // fused L1 targets (nullptr: not fused)
  float *loss_out;               // non-null: the persistent forward finalizes the L1 loss
  float w_c, w_d;
  uint32_t *fmask;               // non-null: the composited-lane masks for the backward
  int segments;                  // non-zero: checkpoints and queued segments for the persistent backward
};

// Renders the pixels of group `grp` (32 consecutive entries of the tile's pixel list) of
// render tile `tile`.  Called by a whole warp; s_rec / s_jg are the warp's own staging.
template <int C, int B>
__device__ __forceinline__ void forward_group(const Work &w, const Prm &prm, int64_t N, int T, int tile, int grp,
                                              float4 (*s_rec)[B], uint2 *s_jg, const FwdOut &out,
                                              double *s_loss = nullptr, bool *pending_wait = nullptr) {
  constexpr int H4 = (C <= 4) ? 3 : 4;
  constexpr int R = B / 32;  // records per lane per batch
  const int lane = threadIdx.x & 31;
  const int f = tile / T, lt = tile - f * T;
  const DevCam &cam = w.cams[f];
  const int tws = cam.tws, ths = cam.ths;
  const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
  const int q = grp * 32 + lane;
  const bool has = q < (int)w.tile_npix[tile];
  const int my = has ? (int)w.px_list[((int64_t)tile << (tws + ths)) + q] : 0;
  const int px = (tx << tws) + (my & ((1 << tws) - 1)), py = (ty << ths) + (my >> tws);
  const float fpx = (float)px, fpy = (float)py;
  // bounding box of the warp's pixels: records whose support box misses it are skipped
  const int bx0 = __reduce_min_sync(0xffffffffu, has ? px : 0x7fffffff);
  const int bx1 = __reduce_max_sync(0xffffffffu, has ? px : -1);
  const int by0 = __reduce_min_sync(0xffffffffu, has ? py : 0x7fffffff);
  const int by1 = __reduce_max_sync(0xffffffffu, has ? py : -1);
  const float wcx = 0.5f * (float)(bx0 + bx1), whx = 0.5f * (float)(bx1 - bx0);
  const float wcy = 0.5f * (float)(by0 + by1), why = 0.5f * (float)(by1 - by0);
  const float wbx0 = (float)bx0, wbx1 = (float)bx1, wby0 = (float)by0, wby1 = (float)by1;
  const uint32_t off = w.tile_offset[tile];
  const uint32_t n = w.tile_offset[tile + 1] - off;
  const float4 *__restrict__ rec = w.rec_hot + (int64_t)f * N * H4;
  const float2 *__restrict__ box = w.rec_box + (int64_t)f * N;
  const int64_t pix = (int64_t)f * cam.H * cam.W + (int64_t)py * cam.W + px;

  float T_ = 1.f;
  float acc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] = 0.f;
  uint32_t last = 0, nfrag = 0, nrec = 0;
  int hit_gid = -1;  // the first fragment with f > delta_alpha (Eq. 4), its Gaussian
  bool done = !has;
  // With out.fmask, entry j of the tile's list gets, for this group, the mask of the lanes
  // that composited it (0 where culled or composited by none), at (off + j) * groups + grp:
  // the backward then replays each lane's own fragments only.  Every entry of a batch the
  // warp walks is written, and the backward walks no further than the last composited one.
  const int ngrp = 1 << (tws + ths - 5);
  using Bits = typename std::conditional<(B > 32), unsigned long long, uint32_t>::type;
  Bits ebits = 0;  // the batch's entries (list position - b0) this lane composited
  // backward segments: the segment being walked and this lane's fragments in it
  static_assert(kSeg % B == 0, "segment boundaries fall on batch ends");
  constexpr int CK4 = (C + 4) / 4;
  int cur_seg = 0;
  uint32_t segfrag = 0;
  auto write_ckpt = [&](int idx) {  // (T, colour composited so far) at checkpoint idx
    if (!has) return;
    float v[4 * CK4];
    v[0] = T_;
#pragma unroll
    for (int c = 0; c < C; ++c) v[1 + c] = acc[c];
#pragma unroll
    for (int c = C + 1; c < 4 * CK4; ++c) v[c] = 0.f;
    float4 *dst = w.ckpt + ((int64_t)idx * w.px_cap + pix) * CK4;
#pragma unroll
    for (int k = 0; k < CK4; ++k) dst[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  };
  auto emit_segment = [&](int sidx) {  // queue segment sidx of this group in its cost bin
    const uint32_t m = __reduce_max_sync(0xffffffffu, segfrag);
    if (lane == 0 && (m != 0u || sidx == 0)) {  // segment 0 also carries the depth gradient
      const int bin = m >= 32u ? 0 : (m >= 16u ? 1 : (m >= 8u ? 2 : 3));
      const unsigned long long at = atomicAdd(w.counters + kBSeg0 + bin * kCounterStride, 1ull);
      if (at < (unsigned long long)w.bseg_cap)
        w.bseg[(int64_t)bin * w.bseg_cap + (int64_t)at] = ((uint32_t)tile << 6) | ((uint32_t)sidx << 3) | (uint32_t)grp;
    }
    segfrag = 0u;
  };
  // everything above reads what the kernels before the sort wrote; the sorted list is the
  // sort's (pending_wait: this warp has not yet waited on it)
  if (pending_wait != nullptr && *pending_wait) {
    grid_dep_wait();
    *pending_wait = false;
  }
  // the records of batch b0 + B, and the indices of batch b0 + 2B, are fetched while batch
  // b0 is composited, so a batch waits on one L2 round trip rather than index -> record
  float4 r[R][H4];
  float2 bb[R];
  bool valid[R];
  uint32_t gnext[R], gcur[R];  // Gaussian ids of batch b0 + 2B and of the batch in r
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const uint32_t j = (uint32_t)(u * 32 + lane);
    valid[u] = j < n;
    bb[u] = make_float2(0.f, 0.f);
    gcur[u] = 0u;
    if (valid[u]) {
      const uint32_t gid = w.sorted[off + j];
      gcur[u] = gid;
#pragma unroll
      for (int k = 0; k < H4; ++k) r[u][k] = rec[(int64_t)gid * H4 + k];
      bb[u] = box[gid];
    }
    const uint32_t jn = (uint32_t)(B + u * 32 + lane);
    gnext[u] = jn < n ? w.sorted[off + jn] : 0u;
  }
  for (uint32_t b0 = 0; b0 < n; b0 += B) {
    if (__all_sync(0xffffffffu, done)) break;
    float4 rn[R][H4];
    float2 bn[R];
    bool vn[R];
    uint32_t gn[R];
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const uint32_t jn = b0 + B + (uint32_t)(u * 32 + lane);
      vn[u] = jn < n;
      bn[u] = make_float2(0.f, 0.f);
      gn[u] = gnext[u];
      if (vn[u]) {
        const uint32_t gid = gnext[u];
#pragma unroll
        for (int k = 0; k < H4; ++k) rn[u][k] = rec[(int64_t)gid * H4 + k];
        bn[u] = box[gid];
      }
      const uint32_t ja = b0 + 2 * B + (uint32_t)(u * 32 + lane);
      gnext[u] = ja < n ? w.sorted[off + ja] : 0u;
    }
    // keep the records whose support box reaches the warp's pixel box, in list order
    int cnt = 0;
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const bool keep = valid[u] && fabsf(r[u][0].x - wcx) <= whx + bb[u].x &&
                        fabsf(r[u][0].y - wcy) <= why + bb[u].y &&
                        reaches_box(r[u][0], r[u][1], wbx0, wbx1, wby0, wby1, prm.alpha_min);
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int slot = cnt + __popc(bal & lanemask_lt());
#pragma unroll
        for (int k = 0; k < H4; ++k) s_rec[k][slot] = r[u][k];
        s_jg[slot] = make_uint2(b0 + (uint32_t)(u * 32 + lane), gcur[u]);
      }
      cnt += __popc(bal);
    }
    nrec += (uint32_t)cnt;
    __syncwarp();
    if (!__all_sync(0xffffffffu, done)) {
      // composites fragment k (footprint fa) in list order, without branches: a fragment
      // below alpha_min, the fragment that would take the transmission below t_eps (the
      // pixel stops before it) and every fragment after the stop leave the pixel's state as
      // it is (weight 0, and fmaf(c, 0, a) = a)
      auto blend = [&](int k, float fa, bool valid) {
        const float Tn = T_ * (1.f - fa);
        const bool live = valid && !done && fa >= prm.alpha_min;
        const bool stop = live && Tn < prm.t_eps;
        const bool comp = live && !stop;
        done = done || stop;
        const float wgt = comp ? fa * T_ : 0.f;
        const float4 c0 = s_rec[2][k];
        float cw[8] = {c0.x, c0.y, c0.z, c0.w, 0.f, 0.f, 0.f, 0.f};
        if (H4 == 4) {
          const float4 c1 = s_rec[3 % H4][k];
          cw[4] = c1.x; cw[5] = c1.y; cw[6] = c1.z; cw[7] = c1.w;
        }
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] = fmaf(cw[c], wgt, acc[c]);
        const uint2 jg = s_jg[k];
        const uint32_t jj = jg.x;
        hit_gid = (comp && hit_gid < 0 && fa > prm.delta_alpha) ? (int)jg.y : hit_gid;
        T_ = comp ? Tn : T_;
        ebits |= comp ? ((Bits)1 << (jj - b0)) : (Bits)0;
      };
      auto alpha_of = [&](int k) {
        const float4 r0 = s_rec[0][k], r1 = s_rec[1][k];
        float dx, dy, t1, t2, g;
        return footprint(fpx, fpy, r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, prm.f_max, dx, dy, t1, t2, g);
      };
      // eight records a round in one block of straight-line code (a record past the batch's
      // end is blended as invalid, not branched around), so the compiler overlaps the
      // records' loads and footprints and only the transmission recurrence stays serial;
      // the warp leaves the batch once all its pixels stopped
      for (int k0 = 0; k0 < cnt; k0 += 8) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int k = min(k0 + q, cnt - 1);
          blend(k, alpha_of(k), k0 + q < cnt);
        }
        if (__all_sync(0xffffffffu, done)) break;
      }
    }
    __syncwarp();
    if (ebits != (Bits)0) {  // the batch's fragments of this lane: count, and the last one
      const uint32_t nb = (uint32_t)(sizeof(Bits) == 8 ? __popcll((unsigned long long)ebits) : __popc((uint32_t)ebits));
      nfrag += nb;
      segfrag += nb;
      last = b0 + (uint32_t)(sizeof(Bits) == 8 ? 64 - __clzll((long long)ebits) : 32 - __clz((int)ebits));
    }
    if (out.fmask != nullptr) {
      // lane L gets the composited lanes of entry b0 + 32u + L (a bit transpose of the
      // lanes' entry bits; culled entries get none) and stores them, one coalesced store per
      // 32 entries
#pragma unroll
      for (int u = 0; u < R; ++u) {
        const uint32_t wv = (uint32_t)(ebits >> (32 * u));
        uint32_t am = 0u;
        if (__any_sync(0xffffffffu, wv != 0u)) am = bit_transpose32(wv, lane);
        if (valid[u]) out.fmask[(int64_t)(off + b0 + (uint32_t)(u * 32 + lane)) * ngrp + grp] = am;
      }
    }
    ebits = 0;
    if (out.segments) {  // a segment boundary at the batch's end: checkpoint, queue the segment
      const uint32_t e = b0 + (uint32_t)B;
      if (e % kSeg == 0u && e / kSeg <= (uint32_t)(kSegMax - 1)) {
        write_ckpt((int)(e / kSeg) - 1);
        emit_segment(cur_seg);
        cur_seg = (int)(e / kSeg);
      }
    }
#pragma unroll
    for (int u = 0; u < R; ++u) {
#pragma unroll
      for (int k = 0; k < H4; ++k) r[u][k] = rn[u][k];
      bb[u] = bn[u];
      valid[u] = vn[u];
      gcur[u] = gn[u];
    }
  }
  if (out.segments) {  // the final (T, colour), and the segment the walk ended in
    write_ckpt(kSegMax - 1);
    emit_segment(cur_seg);
  }
  float lc = 0.f, ld = 0.f, nd = 0.f;
  uint32_t signs = 0u;  // the L1 signs for the backward: 2 bits a channel, then depth (1: +, 2: -)
  if (has) {
    const int64_t HW = (int64_t)cam.H * cam.W;
    // the epilogue's loads (the hit's depth plane, the targets) are issued together, ahead
    // of its stores, so they take one round trip
    float4 c0 = make_float4(0.f, 0.f, 0.f, 0.f), c1 = c0;
    if (hit_gid >= 0) {
      c0 = w.rec_cold[((int64_t)f * N + hit_gid) * 2];
      c1 = w.rec_cold[((int64_t)f * N + hit_gid) * 2 + 1];
    }
    float tc[C], td = 0.f;
    if (out.tcolor != nullptr) {
#pragma unroll
      for (int c = 0; c < C; ++c) tc[c] = out.tcolor[((int64_t)f * C + c) * HW + (int64_t)py * cam.W + px];
      td = out.tdepth[pix];
    }
#pragma unroll
    for (int c = 0; c < C; ++c) out.color[((int64_t)f * C + c) * HW + (int64_t)py * cam.W + px] = acc[c];
    out.alpha[pix] = 1.f - T_;
    float D = -1.f;
    if (hit_gid >= 0) {
      const float ux = (fpx - cam.cx) / cam.fx, uy = (fpy - cam.cy) / cam.fy;
      const float den = fmaf(c0.x, ux, fmaf(c0.y, uy, c0.z));
      const float nu = sqrtf(fmaf(ux, ux, fmaf(uy, uy, 1.f)));
      D = (fabsf(den) >= prm.cos_max * nu) ? c0.w / den : c1.x;
    }
    out.depth[pix] = D;
    if (out.index_map != nullptr) out.index_map[pix] = hit_gid;
    w.px_T[pix] = T_;
    w.px_last[pix] = last;
    w.px_hit[pix] = hit_gid;
    if (out.tcolor != nullptr) {  // fused L1 terms of this pixel (Eq. 7)
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const float d = acc[c] - tc[c];
        lc += fabsf(d);
        signs |= (d > 0.f ? 1u : (d < 0.f ? 2u : 0u)) << (2 * c);
      }
      if (D != -1.f && td > 0.f) {
        const float d = D - td;
        ld = fabsf(d);
        nd = 1.f;
        signs |= (d > 0.f ? 1u : (d < 0.f ? 2u : 0u)) << (2 * C);
      }
    }
  }
  if (out.tcolor != nullptr && out.fmask != nullptr) {  // the group's pixel state for the backward
    const int64_t gslot = (((int64_t)tile << (tws + ths - 5)) + grp) * 32 + lane;
    w.gstate[gslot] = has ? make_uint4((uint32_t)px | ((uint32_t)py << 16), __float_as_uint(T_), last, (uint32_t)hit_gid)
                          : make_uint4(0xffffffffu, 0u, 0u, 0xffffffffu);
    w.gsign[gslot] = signs;
  }
  if (out.tcolor != nullptr) {  // fixed-order per-group partials, summed by k_loss_finalize
    for (int o = 16; o > 0; o >>= 1) {
      lc += __shfl_xor_sync(0xffffffffu, lc, o);
      ld += __shfl_xor_sync(0xffffffffu, ld, o);
      nd += __shfl_xor_sync(0xffffffffu, nd, o);
    }
    if (lane == 0) {
      float *lp = w.tile_loss + (((int64_t)tile << (tws + ths - 5)) + grp) * 4;
      lp[0] = lc;
      lp[1] = ld;
      lp[2] = nd;
      if (s_loss != nullptr) {  // the CTA's FP64 sums: their order (the queue's) does not show
        atomicAdd(s_loss + 0, (double)lc);
        atomicAdd(s_loss + 1, (double)ld);
        atomicAdd(s_loss + 2, (double)nd);
      }
    }
  }
  // fragment and walked-record counters: one atomic each per warp
  const unsigned fr = __reduce_add_sync(0xffffffffu, nfrag);
  if (lane == 0 && fr) atomicAdd(w.counters + kFragments, (unsigned long long)fr);
  if (lane == 0 && nrec) atomicAdd(w.counters + kWarpRecords, (unsigned long long)nrec);
}

// Schedule 0: CTA `tile` with one warp per 32-pixel group of the tile's pixel list.
// Registers: two CTAs per SM for C <= 4 (up to 128 a thread, enough to keep the compositing
// state and the prefetched batch out of local memory; a third CTA at 80 registers spilled
// inside the blending loop and was slower); C = 8 keeps the registers it needs.
template <int C, int B>
constexpr int fwd_min_ctas() { return C <= 4 ? 2 : 1; }

template <int C, int B>
__global__ void __launch_bounds__(kMaxTilePix, fwd_min_ctas<C, B>()) k_forward(Work w, Prm prm, int64_t N, int T,
                                                                              FwdOut out) {
  grid_dep_wait();
  constexpr int H4 = (C <= 4) ? 3 : 4;
  __shared__ float4 s_rec[kMaxTilePix / 32][H4][B];
  __shared__ uint2 s_jg[kMaxTilePix / 32][B];
  if (w.counters[kSkip] != 0ull) return;
  const int tile = blockIdx.x, wid = threadIdx.x >> 5;
  if (wid * 32 >= (int)w.tile_npix[tile]) return;
  forward_group<C, B>(w, prm, N, T, tile, wid, s_rec[wid], s_jg[wid], out);
}

// Schedule 1: persistent warps.  Each warp starts with one of the first items; later items come
// from a shared counter, so warps that finish early take the remaining work.  The queue
// holds the longest lists first.  kW warps a CTA (8, or 10 for calls of many tiles).
template <int C, int B, int kW>
__global__ void __launch_bounds__(32 * kW, fwd_min_ctas<C, B>()) k_forward_queue(Work w, Prm prm, int64_t N, int T,
                                                                                 FwdOut out, int spread) {
  // The kernel in front is the call's tile sort, which writes only the sorted lists: a warp
  // takes its first item and sets up its pixels (queue, pixel lists, tile offsets, records,
  // all written earlier) before it waits on the sort, just before its first list read.
  bool pending = true;
  constexpr int H4 = (C <= 4) ? 3 : 4;
  __shared__ float4 s_rec[kW][H4][B];
  __shared__ uint2 s_jg[kW][B];
  __shared__ double s_loss[3];
  if (w.counters[kSkip] != 0ull) {
    grid_dep_wait();
    return;
  }
  if (threadIdx.x < 3) s_loss[threadIdx.x] = 0.0;
  __syncthreads();
  const uint32_t nitems = (uint32_t)w.counters[kItems];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t nwarps = gridDim.x * (uint32_t)kW;
  // the first eight warps of each CTA as first_item lays them out, the others after them
  uint32_t it = wid < 8 ? first_item(w, wid, spread) : (uint32_t)wid * gridDim.x + blockIdx.x;
  while (it < nitems) {
    const uint32_t item = w.items[it];
    forward_group<C, B>(w, prm, N, T, (int)(item >> 3), (int)(item & 7u), s_rec[wid], s_jg[wid], out,
                        out.loss_out != nullptr ? s_loss : nullptr, &pending);
    uint32_t nx = 0;
    if (lane == 0) nx = nwarps + (uint32_t)atomicAdd(w.counters + kQFwd, 1ull);
    it = __shfl_sync(0xffffffffu, nx, 0);
  }
  if (pending) grid_dep_wait();  // a warp without an item still waits before the kernel completes
  if (out.loss_out != nullptr) {  // the last CTA to finish finalizes the L1 loss (Eq. 7)
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x < 3) atomicAdd(w.loss_acc + threadIdx.x, s_loss[threadIdx.x]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(w.loss_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
      __threadfence();
      const double sc = __ldcg(w.loss_acc + 0), sd = __ldcg(w.loss_acc + 1), nd = __ldcg(w.loss_acc + 2);
      const float np = (float)w.counters[kMaskedPix];
      const float Lc = np > 0.f ? (float)sc / (np * (float)C) : 0.f;
      const float Ld = nd > 0.0 ? (float)(sd / nd) : 0.f;
      out.loss_out[0] = out.w_c * Lc + out.w_d * Ld;
      out.loss_out[1] = Lc;
      out.loss_out[2] = Ld;
      w.loss_scal[4] = np > 0.f ? out.w_c / (np * (float)C) : 0.f;
      w.loss_scal[5] = nd > 0.0 ? out.w_d / (float)nd : 0.f;
      w.loss_scal[1] = Lc;
      w.loss_scal[2] = Ld;
      w.counters[kDepthPix] = (unsigned long long)nd;
      w.loss_acc[0] = 0.0;
      w.loss_acc[1] = 0.0;
      w.loss_acc[2] = 0.0;
      *w.loss_done = 0u;
    }
  }
}

template <int C, int B>
static void launch_forward_cb(const Work &w, const Prm &prm, int64_t N, int F, int T, const Tuning &tn,
                              const FwdOut &out, cudaStream_t s) {
  if (tn.schedule == 1) {
    // a call of many tiles (batched keyframes) is bound by throughput: ten warps a CTA
    // there, as for its segmented backward; single-frame steps keep eight
    if constexpr (C <= 4 && B == 32) {
      if ((int64_t)F * T > kScanSingleMax) {
        launch(k_forward_queue<C, B, 10>, tn.num_sms * tn.ctas_per_sm, 320, 0, s, w, prm, N, T, out,
               tn.ctas_per_sm <= 2 ? 1 : 0);
        return;
      }
    }
    launch(k_forward_queue<C, B, 8>, tn.num_sms * tn.ctas_per_sm, 256, 0, s, w, prm, N, T, out,
           tn.ctas_per_sm <= 2 ? 1 : 0);
  } else
    launch(k_forward<C, B>, F * T, 1 << (tn.tws + tn.ths), 0, s, w, prm, N, T, out);
}

void launch_forward(int C, const Work &w, const Prm &prm, int64_t N, int F, int T, const Tuning &tn, float *color,
                    float *depth, float *alpha, int32_t *index_map, const float *tcolor, const float *tdepth,
                    float *loss_out, float w_c, float w_d, uint32_t *fmask, cudaStream_t s) {
  // the persistent schedule with composited-lane masks also leaves the backward's segments
  const FwdOut out{color, depth, alpha, index_map, tcolor, tdepth,
                   (tn.schedule == 1 && tcolor != nullptr) ? loss_out : nullptr, w_c, w_d, fmask,
                   (tn.schedule == 1 && fmask != nullptr) ? 1 : 0};
  if (C == 3) {
    if (tn.batch == 64) launch_forward_cb<3, 64>(w, prm, N, F, T, tn, out, s);
    else launch_forward_cb<3, 32>(w, prm, N, F, T, tn, out, s);
  } else {
    if (tn.batch == 64) launch_forward_cb<8, 64>(w, prm, N, F, T, tn, out, s);
    else launch_forward_cb<8, 32>(w, prm, N, F, T, tn, out, s);
  }
}

}  // namespace rtg
