// Projection and tile binning (Section 3.1 rendering; tiles of 16 x 16 pixels as in
// Supplement B): per-tile masked-pixel counts, the unstable index, the EWA projection
// of every Gaussian into every frame, the exclusive scan of per-tile pair counts and
// the emission of (depth, index) keys into per-tile buckets.
#include "kernels.cuh"
#include "project.cuh"

namespace rtg {

// --------------------------------------------------------------------------- setup + tile mask
// One CTA per (frame, tile).  Counts the masked in-image pixels of the tile (the
// compacted pixel set of that tile) and clears its pair counter.  Block 0 also
// publishes the cameras and clears the per-call counters.
__global__ void __launch_bounds__(kTilePix) k_tile_mask(FrameSet fs, Work w, const uint8_t *__restrict__ mask,
                                                        int T) {
  const int tile = blockIdx.x;
  const int f = tile / T, lt = tile - f * T;
  const DevCam &cam = fs.cam[f];
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < fs.F; i += blockDim.x) w.cams[i] = fs.cam[i];
    if (threadIdx.x < kNumCounters) w.counters[threadIdx.x] = 0ull;
  }
  const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
  const int px = tx * kTile + (threadIdx.x & (kTile - 1)), py = ty * kTile + (threadIdx.x / kTile);
  bool in = px < cam.W && py < cam.H;
  if (in && mask != nullptr) in = mask[((int64_t)f * cam.H + py) * cam.W + px] != 0;
  const int cnt = __syncthreads_count(in);
  if (threadIdx.x == 0) {
    w.tile_npix[tile] = (uint32_t)cnt;
    w.tile_count[tile] = 0u;
  }
}

// --------------------------------------------------------------------------- unstable index
// Two-kernel scan: per-block counts, then each block adds its predecessors' counts.
__global__ void __launch_bounds__(kScanBlock) k_rank_count(const uint8_t *__restrict__ unstable, int64_t n,
                                                           int32_t *__restrict__ block_cnt) {
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  const bool u = i < n && unstable[i] != 0;
  const int c = __syncthreads_count(u);
  if (threadIdx.x == 0) block_cnt[blockIdx.x] = c;
}

__global__ void __launch_bounds__(kScanBlock) k_rank_write(const uint8_t *__restrict__ unstable, int64_t n,
                                                           const int32_t *__restrict__ block_cnt,
                                                           int32_t *__restrict__ rank, int32_t *__restrict__ ids,
                                                           unsigned long long *nu_counter, int64_t *nu_out) {
  __shared__ int s_warp[kScanBlock / 32];
  __shared__ int s_base;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // predecessors' total
  int acc = 0;
  for (int b = threadIdx.x; b < (int)blockIdx.x; b += kScanBlock) acc += block_cnt[b];
  acc = block_sum_int(acc, s_warp);
  if (threadIdx.x == 0) s_base = acc;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  const bool u = i < n && unstable[i] != 0;
  const unsigned bal = __ballot_sync(0xffffffffu, u);
  if (lane == 0) s_warp[wid] = __popc(bal);
  __syncthreads();
  int before = s_base;
  for (int k = 0; k < wid; ++k) before += s_warp[k];
  before += __popc(bal & ((1u << lane) - 1u));
  if (i < n) {
    if (rank != nullptr) rank[i] = u ? before : -1;
    if (u && ids != nullptr) ids[before] = (int32_t)i;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanBlock - 1) {
    int total = before + (u ? 1 : 0);
    if (nu_counter != nullptr) nu_counter[kNumUnstable] = (unsigned long long)total;
    if (nu_out != nullptr) *nu_out = total;
  }
}

// --------------------------------------------------------------------------- projection
// kMask = true projects only the unstable Gaussians (for the unstable-pixel mask): no
// gradient rows are cleared and no visibility is counted.
template <int C, bool kMask>
__global__ void __launch_bounds__(256) k_project(GaussPtrs g, Work w, Prm prm, int F, int T) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const int64_t N = g.n;
  if (kMask && g.unstable[i] == 0) {
    for (int f = 0; f < F; ++f) w.ntiles[(int64_t)f * N + i] = 0u;
    return;
  }
  GParams P;
  bool ok = load_params(g, w.rank, i, P);
  const float *cp = color_ptr(g, w.rank, i);
  float col[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    col[c] = cp[c];
    ok = ok && isfinite(col[c]);
  }
  const int rk = w.rank[i];
  float R[9];
  int kmin = 0;
  if (ok) {
    const float qn = sqrtf(P.q[0] * P.q[0] + P.q[1] * P.q[1] + P.q[2] * P.q[2] + P.q[3] * P.q[3]);
    quat_to_rot(P.q[0] / qn, P.q[1] / qn, P.q[2] / qn, P.q[3] / qn, R);
    kmin = argmin3(P.s[0], P.s[1], P.s[2]);
  }
  constexpr int H4 = (C <= 4) ? 3 : 4;
  constexpr int G2 = (C <= 5) ? 16 : 20;
  unsigned visible_frames = 0;
  for (int f = 0; f < F; ++f) {
    const DevCam &cam = w.cams[f];
    uint32_t nt = 0;
    Projected o;
    if (ok && project_gaussian(cam, prm, P, R, kmin, o)) {
      const int tx0 = o.x0 / kTile, tx1 = o.x1 / kTile, ty0 = o.y0 / kTile, ty1 = o.y1 / kTile;
      const uint32_t *npix = w.tile_npix + (int64_t)f * T;
      uint32_t *tcount = w.tile_count + (int64_t)f * T;
      for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) {
          const int t = ty * cam.tiles_x + tx;
          if (npix[t] != 0u) {
            ++nt;
            atomicAdd(tcount + t, 1u);
          }
        }
      if (nt > 0) {
        float4 *hot = w.rec_hot + ((int64_t)f * N + i) * H4;
        hot[0] = make_float4(o.mux.hi, o.muy.hi, o.mux.lo, o.muy.lo);
        hot[1] = make_float4(o.u11, o.u12, o.u22, P.alpha);
        float cc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int c = 0; c < C; ++c) cc[c] = col[c];
        hot[2] = make_float4(cc[0], cc[1], cc[2], cc[3]);
        if (H4 == 4) hot[3] = make_float4(cc[4], cc[5], cc[6], cc[7]);
        w.rec_box[(int64_t)f * N + i] = make_float2(o.rx, o.ry);
        float4 *cold = w.rec_cold + ((int64_t)f * N + i) * 2;
        cold[0] = make_float4(o.n[0], o.n[1], o.n[2], o.d0);
        cold[1] = make_float4(o.Z, __int_as_float(rk), __uint_as_float((uint32_t)tx0 | ((uint32_t)ty0 << 16)),
                              __uint_as_float((uint32_t)tx1 | ((uint32_t)ty1 << 16)));
        if (!kMask && rk >= 0) {
          float4 *g2 = reinterpret_cast<float4 *>(w.grad2d + ((int64_t)f * N + rk) * G2);
#pragma unroll
          for (int k = 0; k < G2 / 4; ++k) g2[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        ++visible_frames;
      }
    }
    w.ntiles[(int64_t)f * N + i] = nt;
  }
  if (!kMask && visible_frames) atomicAdd(w.counters + kVisible, (unsigned long long)visible_frames);
}

// --------------------------------------------------------------------------- tile scan
// One CTA: exclusive scan of the per-tile pair counts into bucket offsets, capacity check.
__global__ void __launch_bounds__(1024) k_scan_tiles(Work w, int FT, int64_t max_pairs) {
  __shared__ unsigned long long s_warp[32];
  __shared__ uint32_t s_wmax[32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int per = (FT + 1023) / 1024;
  const int b = tid * per, e = min(FT, b + per);
  unsigned long long local = 0, npix = 0;
  uint32_t mx = 0;
  for (int t = b; t < e; ++t) {
    local += w.tile_count[t];
    npix += w.tile_npix[t];
    mx = max(mx, w.tile_count[t]);
  }
  // inclusive warp scan of `local`
  unsigned long long inc = local;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 31) s_warp[wid] = inc;
  if (lane == 0) s_wmax[wid] = mx;
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
  }
  __syncthreads();
  unsigned long long run = (wid > 0 ? s_warp[wid - 1] : 0ull) + inc - local;
  for (int t = b; t < e; ++t) {
    w.tile_offset[t] = (uint32_t)run;
    w.tile_cursor[t] = 0u;
    run += w.tile_count[t];
  }
  // total masked pixels
  unsigned long long np = npix;
  for (int o = 16; o > 0; o >>= 1) np += __shfl_xor_sync(0xffffffffu, np, o);
  __syncthreads();
  if (lane == 0) s_warp[wid] = np;
  __syncthreads();
  if (tid == 0) {
    unsigned long long total_pix = 0;
    for (int k = 0; k < 32; ++k) total_pix += s_warp[k];
    // s_warp was overwritten; recompute the pair total from the last offset
    unsigned long long total = (unsigned long long)w.tile_offset[FT - 1] + w.tile_count[FT - 1];
    w.tile_offset[FT] = (uint32_t)total;
    w.counters[kPairs] = total;
    w.counters[kMaskedPix] = total_pix;
    w.counters[kMaxTilePairs] = s_wmax[0];
    if (total > (unsigned long long)max_pairs || total > 0xffffffffull) {
      w.counters[kSkip] = 1ull;
      atomicCAS(w.status, 0u, (uint32_t)(int32_t)RTG_ERR_WORKSPACE);
    }
  }
}

// --------------------------------------------------------------------------- emission
// Writes key = (IEEE bits of z_c) << 32 | i into the bucket of every masked tile the
// Gaussian's support box touches.  Positive floats order like their bit patterns, so
// sorting a bucket by key orders it by depth, then by index.
__global__ void __launch_bounds__(256) k_emit(Work w, int64_t N, int F, int T) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N || w.counters[kSkip] != 0ull) return;
  for (int f = 0; f < F; ++f) {
    if (w.ntiles[(int64_t)f * N + i] == 0u) continue;
    const int tiles_x = w.cams[f].tiles_x;
    const float4 c1 = w.rec_cold[((int64_t)f * N + i) * 2 + 1];
    const uint32_t lo = __float_as_uint(c1.z), hi = __float_as_uint(c1.w);
    const int tx0 = lo & 0xffff, ty0 = lo >> 16, tx1 = hi & 0xffff, ty1 = hi >> 16;
    const unsigned long long key = ((unsigned long long)__float_as_uint(c1.x) << 32) | (unsigned long long)(uint32_t)i;
    const uint32_t *npix = w.tile_npix + (int64_t)f * T;
    for (int ty = ty0; ty <= ty1; ++ty)
      for (int tx = tx0; tx <= tx1; ++tx) {
        const int t = ty * tiles_x + tx;
        if (npix[t] != 0u) {
          const int64_t gt = (int64_t)f * T + t;
          const uint32_t slot = atomicAdd(w.tile_cursor + gt, 1u);
          w.keys[(int64_t)w.tile_offset[gt] + slot] = key;
        }
      }
  }
}

void launch_tile_mask(const FrameSet &fs, const Work &w, const uint8_t *mask, int T, cudaStream_t s) {
  k_tile_mask<<<fs.F * T, kTilePix, 0, s>>>(fs, w, mask, T);
}

void launch_rank(const uint8_t *unstable, int64_t n, int32_t *block_cnt, int32_t *rank, int32_t *ids,
                 unsigned long long *nu_counter, int64_t *nu_out, cudaStream_t s) {
  if (n <= 0) return;
  const int nb = (int)((n + kScanBlock - 1) / kScanBlock);
  k_rank_count<<<nb, kScanBlock, 0, s>>>(unstable, n, block_cnt);
  k_rank_write<<<nb, kScanBlock, 0, s>>>(unstable, n, block_cnt, rank, ids, nu_counter, nu_out);
}

void launch_project(const GaussPtrs &g, const Work &w, const Prm &prm, int F, int T, cudaStream_t s) {
  if (g.n <= 0) return;
  const unsigned nb = (unsigned)((g.n + 255) / 256);
  if (g.C == 3)
    k_project<3, false><<<nb, 256, 0, s>>>(g, w, prm, F, T);
  else
    k_project<8, false><<<nb, 256, 0, s>>>(g, w, prm, F, T);
}

void launch_project_unstable(const GaussPtrs &g, const Work &w, const Prm &prm, int F, int T, cudaStream_t s) {
  if (g.n <= 0) return;
  const unsigned nb = (unsigned)((g.n + 255) / 256);
  if (g.C == 3)
    k_project<3, true><<<nb, 256, 0, s>>>(g, w, prm, F, T);
  else
    k_project<8, true><<<nb, 256, 0, s>>>(g, w, prm, F, T);
}

void launch_scan_tiles(const Work &w, int FT, int64_t max_pairs, cudaStream_t s) {
  k_scan_tiles<<<1, 1024, 0, s>>>(w, FT, max_pairs);
}

void launch_emit(const Work &w, int64_t N, int F, int T, cudaStream_t s) {
  if (N <= 0) return;
  k_emit<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(w, N, F, T);
}

}  // namespace rtg
