// Global keyframe optimisation (Section 3.2, "Keyframes and global optimization"): each
// keyframe of a global step is optimised only on its pixels with the largest colour errors.
//
// Top-error selection: per frame, the k = floor(frac * H * W) pixels of largest colour error
// e = |c_0 - t_0| + |c_1 - t_1| + ... (float32, channel order), ties towards the lower
// pixel index.  Errors are non-negative (a sum of absolute values; a NaN sum is the positive
// canonical NaN), so their IEEE bit patterns order like the values and have bit 31 clear:
// the k-th largest is found exactly by a radix select on the 31 low bits, in three passes of
// 11, 10 and 10 bits, most significant first.  A pass histograms, over every frame at once,
// the digit of the keys that share the digits fixed so far; the last block of each frame to
// finish (a ticket counter) picks the digit that holds the k-th largest key.  Then per-block
// counts of keys equal to the threshold T, their exclusive scan, and a mark pass: key > T,
// or key == T among the first (k - #keys > T) of them in pixel order.
//
// Narrowing: the forward keeps its per-pixel state (final transmission, last fragment,
// depth hit) in image layout, and its per-tile sorted lists cover every tile it rendered.
// A backward over a subset of those pixels therefore needs only each tile's pixel list
// compacted to the subset (and the persistent schedule's queue rebuilt); the lists and
// records stay as they are.  With targets, the same kernel forms the fused L1 partials of
// the narrowed pixels (Eq. 7/8), so the fused backward can follow.
#include "kernels.cuh"

namespace rtg {

// ----------------------------------------------------------------------------- selection

// digit width, shift and histogram size of pass P (bits 30..20, 19..10, 9..0)
template <int P>
struct SelDigit {
  static constexpr int bits = P == 0 ? 11 : 10;
  static constexpr int shift = P == 0 ? 20 : (P == 1 ? 10 : 0);
  static constexpr int bins = 1 << bits;
};

template <int P>
__global__ void __launch_bounds__(kSelThreads) k_sel_pass(SelBufs b, int F, int C, int64_t n, int nb, uint32_t k,
                                                          const float *__restrict__ color,
                                                          const float *__restrict__ target) {
  grid_dep_wait();
  using D = SelDigit<P>;
  constexpr int kPer = kSelPerBlock / kSelThreads;  // pixels per thread
  constexpr int kChunk = D::bins / kSelThreads;     // histogram bins per thread
  __shared__ uint32_t s_h[D::bins];
  __shared__ uint32_t s_w[kSelThreads / 32];
  __shared__ int s_last;
  const int f = blockIdx.y, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int i = tid; i < D::bins; i += kSelThreads) s_h[i] = 0u;
  const uint32_t prefix = P > 0 ? b.state[2 * f] : 0u;
  __syncthreads();
  const int64_t i0 = (int64_t)blockIdx.x * kSelPerBlock;
  uint32_t *__restrict__ keys = b.keys + (int64_t)f * n;
  uint32_t key[kPer];
  bool use[kPer];
  if (P == 0) {  // errors from the images: every load of the block's pixels in flight at once
    float e[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) e[u] = 0.f;
    for (int c = 0; c < C; ++c) {
      float cv[kPer], tv[kPer];
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int64_t i = i0 + u * kSelThreads + tid;
        const int64_t o = ((int64_t)f * C + c) * n + i;
        cv[u] = i < n ? color[o] : 0.f;
        tv[u] = i < n ? target[o] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kPer; ++u) e[u] = __fadd_rn(e[u], fabsf(__fsub_rn(cv[u], tv[u])));
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int64_t i = i0 + u * kSelThreads + tid;
      key[u] = __float_as_uint(e[u]);
      use[u] = i < n;
      if (use[u]) keys[i] = key[u];
    }
  } else {
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int64_t i = i0 + u * kSelThreads + tid;
      key[u] = i < n ? keys[i] : 0u;
      use[u] = i < n && (key[u] >> (D::shift + D::bits)) == (prefix >> (D::shift + D::bits));
    }
  }
  // histogram of this pass's digit: lanes with the same digit add once (match.any)
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const uint32_t d = (key[u] >> D::shift) & (uint32_t)(D::bins - 1);
    const unsigned act = __ballot_sync(0xffffffffu, use[u]);
    if (use[u]) {
      const unsigned peers = __match_any_sync(act, d);
      if ((peers & lanemask_lt()) == 0u) atomicAdd(&s_h[d], (uint32_t)__popc(peers));
    }
  }
  __syncthreads();
  uint32_t *__restrict__ hist = b.hist + ((int64_t)P * F + f) * kSelHistStride;
  for (int i = tid; i < D::bins; i += kSelThreads)
    if (s_h[i]) atomicAdd(&hist[i], s_h[i]);
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&b.ticket[P * F + f], 1u) == (uint32_t)nb - 1u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last block of frame f: thread t owns the kChunk digits below D::bins - kChunk * t, and
  // the counts are accumulated from the largest digit down
  const uint32_t krem = P == 0 ? k : b.state[2 * f + 1];
  uint32_t h[kChunk], mine = 0;
#pragma unroll
  for (int q = 0; q < kChunk; ++q) {
    h[q] = __ldcg(&hist[D::bins - 1 - (kChunk * tid + q)]);
    mine += h[q];
  }
  uint32_t inc = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) s_w[wid] = inc;
  __syncthreads();
  uint32_t run = inc - mine;  // keys with a larger digit than this thread's chunk
  for (int q = 0; q < wid; ++q) run += s_w[q];
#pragma unroll
  for (int q = 0; q < kChunk; ++q) {
    if (run < krem && run + h[q] >= krem) {  // exactly one digit: the k-th largest key's
      const uint32_t d = (uint32_t)(D::bins - 1 - (kChunk * tid + q));
      b.state[2 * f] = prefix | (d << D::shift);
      b.state[2 * f + 1] = krem - run;
    }
    run += h[q];
  }
}

// Per-block counts of keys equal to the threshold, then (last block of each frame) their
// exclusive scan in place: the number of equal keys before each block.
__global__ void __launch_bounds__(kSelThreads) k_sel_ties(SelBufs b, int F, int64_t n, int nb) {
  grid_dep_wait();
  __shared__ int s_w[kSelThreads / 32];
  __shared__ uint32_t s_u[kSelThreads / 32];
  __shared__ int s_last;
  const int f = blockIdx.y, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t T = b.state[2 * f];
  const int64_t i0 = (int64_t)blockIdx.x * kSelPerBlock, i1 = min(n, i0 + kSelPerBlock);
  const uint32_t *__restrict__ keys = b.keys + (int64_t)f * n;
  int cnt = 0;
  for (int64_t i = i0 + tid; i < i1; i += kSelThreads) cnt += keys[i] == T;
  cnt = block_sum_int(cnt, s_w);
  uint32_t *__restrict__ tie = b.tie + (int64_t)f * nb;
  if (tid == 0) tie[blockIdx.x] = (uint32_t)cnt;
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&b.ticket[kSelPasses * F + f], 1u) == (uint32_t)nb - 1u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int per = (nb + kSelThreads - 1) / kSelThreads;
  const int e0 = min(nb, tid * per), e1 = min(nb, e0 + per);
  uint32_t mine = 0;
  for (int e = e0; e < e1; ++e) mine += __ldcg(&tie[e]);
  uint32_t inc = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) s_u[wid] = inc;
  __syncthreads();
  uint32_t run = inc - mine;
  for (int q = 0; q < wid; ++q) run += s_u[q];
  for (int e = e0; e < e1; ++e) {
    const uint32_t c = __ldcg(&tie[e]);
    tie[e] = run;
    run += c;
  }
}

__global__ void __launch_bounds__(kSelThreads) k_sel_mark(SelBufs b, int64_t n, int nb, uint8_t *__restrict__ mask) {
  grid_dep_wait();
  __shared__ uint32_t s_w[kSelThreads / 32];
  const int f = blockIdx.y, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t T = b.state[2 * f], krem = b.state[2 * f + 1];
  uint32_t base = b.tie[(int64_t)f * nb + blockIdx.x];  // equal keys in earlier blocks
  const int64_t i0 = (int64_t)blockIdx.x * kSelPerBlock, i1 = min(n, i0 + kSelPerBlock);
  const uint32_t *__restrict__ keys = b.keys + (int64_t)f * n;
  uint8_t *__restrict__ out = mask + (int64_t)f * n;
  for (int64_t r = i0; r < i1; r += kSelThreads) {  // rows of kSelThreads pixels, in order
    const int64_t i = r + tid;
    const bool in = i < i1;
    const uint32_t key = in ? keys[i] : 0u;
    bool sel = in && key > T;
    if (base < krem) {  // block-uniform: some equal keys may still be taken
      const bool eq = in && key == T;
      const unsigned bal = __ballot_sync(0xffffffffu, eq);
      if (lane == 0) s_w[wid] = __popc(bal);
      __syncthreads();
      uint32_t before = 0, total = 0;
#pragma unroll
      for (int q = 0; q < kSelThreads / 32; ++q) {
        const uint32_t c = s_w[q];
        before += q < wid ? c : 0u;
        total += c;
      }
      __syncthreads();
      if (eq && base + before + (uint32_t)__popc(bal & lanemask_lt()) < krem) sel = true;
      base += total;
    }
    if (in) out[i] = sel ? 1 : 0;
  }
}

void launch_select_top_error(const SelBufs &b, int F, int C, int64_t n, uint32_t k, const float *color,
                             const float *target, uint8_t *mask, cudaStream_t s) {
  const int nb = (int)((n + kSelPerBlock - 1) / kSelPerBlock);
  const dim3 grid((unsigned)nb, (unsigned)F);
  cudaMemsetAsync(b.hist, 0, sel_scratch_words(F) * sizeof(uint32_t), s);
  launch(k_sel_pass<0>, grid, kSelThreads, 0, s, b, F, C, n, nb, k, color, target);
  launch(k_sel_pass<1>, grid, kSelThreads, 0, s, b, F, C, n, nb, k, color, target);
  launch(k_sel_pass<2>, grid, kSelThreads, 0, s, b, F, C, n, nb, k, color, target);
  launch(k_sel_ties, grid, kSelThreads, 0, s, b, F, n, nb);
  launch(k_sel_mark, grid, kSelThreads, 0, s, b, n, nb, mask);
}

// ----------------------------------------------------------------------------- narrowing
// One CTA of 2^(tws+ths) threads per render tile of the last forward: keeps the entries of
// the tile's pixel list whose pixel is set in `mask`, in their order (the tile's Z order), and adds
// the tile's new pixel count to the masked-pixel counter.  With targets, warp g then forms
// the fused L1 partials (colour, depth, depth count) of the tile's new group g, as the
// forward does for its groups.
__global__ void __launch_bounds__(kMaxTilePix) k_narrow_pixels(Work w, int T, const uint8_t *__restrict__ mask,
                                                               NarrowLoss nl) {
  grid_dep_wait();
  __shared__ int s_wcnt[kMaxTilePix / 32];
  __shared__ uint8_t s_list[kMaxTilePix];
  const int tile = blockIdx.x;
  const uint32_t np = w.tile_npix[tile];
  if (np == 0u) return;
  const int f = tile / T, lt = tile - f * T;
  const DevCam &cam = w.cams[f];
  const int tws = cam.tws, ths = cam.ths;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  uint8_t *__restrict__ list = w.px_list + ((int64_t)tile << (tws + ths));
  const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
  int my = 0;
  bool keep = false;
  if ((uint32_t)tid < np) {
    my = list[tid];
    const int px = (tx << tws) + (my & ((1 << tws) - 1)), py = (ty << ths) + (my >> tws);
    keep = mask[((int64_t)f * cam.H + py) * cam.W + px] != 0;
  }
  const unsigned bal = __ballot_sync(0xffffffffu, keep);
  if (lane == 0) s_wcnt[wid] = __popc(bal);
  __syncthreads();  // every entry is read before any is rewritten
  int before = 0, total = 0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
    const int c = s_wcnt[q];
    before += q < wid ? c : 0;
    total += c;
  }
  if (keep) {
    const int slot = before + __popc(bal & lanemask_lt());
    list[slot] = (uint8_t)my;
    s_list[slot] = (uint8_t)my;
  }
  if (tid == 0) {
    w.tile_npix[tile] = (uint32_t)total;
    if (total) atomicAdd(w.counters + kMaskedPix, (unsigned long long)total);
  }
  __syncthreads();  // s_list complete (every thread of the block reaches this barrier)
  if (nl.tcolor == nullptr || wid * 32 >= total) return;
  // fused L1 partials of group wid (Eq. 7/8 terms), as the forward writes them
  const bool has = tid < total;
  float lc = 0.f, ld = 0.f, nd = 0.f;
  if (has) {
    const int q = s_list[tid];
    const int px = (tx << tws) + (q & ((1 << tws) - 1)), py = (ty << ths) + (q >> tws);
    const int64_t HW = (int64_t)cam.H * cam.W, pix = (int64_t)f * HW + (int64_t)py * cam.W + px;
    for (int c = 0; c < nl.C; ++c) {
      const int64_t o = ((int64_t)f * nl.C + c) * HW + (int64_t)py * cam.W + px;
      lc += fabsf(nl.color[o] - nl.tcolor[o]);
    }
    const float D = nl.depth[pix], td = nl.tdepth[pix];
    if (D != -1.f && td > 0.f) {
      ld = fabsf(D - td);
      nd = 1.f;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    lc += __shfl_xor_sync(0xffffffffu, lc, o);
    ld += __shfl_xor_sync(0xffffffffu, ld, o);
    nd += __shfl_xor_sync(0xffffffffu, nd, o);
  }
  if (lane == 0) {
    float *lp = w.tile_loss + (((int64_t)tile << (tws + ths - 5)) + wid) * 4;
    lp[0] = lc;
    lp[1] = ld;
    lp[2] = nd;
  }
}

void launch_narrow_pixels(const Work &w, int F, int T, int tws, int ths, const uint8_t *mask, int gshift,
                          const NarrowLoss &nl, cudaStream_t s) {
  cudaMemsetAsync(w.counters + kMaskedPix, 0, sizeof(unsigned long long), s);
  launch(k_narrow_pixels, F * T, 1 << (tws + ths), 0, s, w, T, mask, nl);
  if (gshift >= 0) launch_requeue(w, F * T, gshift, s);
}

}  // namespace rtg
