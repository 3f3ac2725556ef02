// Gaussian adding (Section 3.2, "Gaussians adding", Eq. 6): from a full-frame render of the
// map (colour, alpha = 1 - transmission, depth, index map) and the input frame (colour,
// depth), the pixels that get a new Gaussian:
//   M_s = {T_hat > delta_T or |D_hat - D| > delta_d}       new geometry: opaque Gaussian
//   M_c = {mean_c |C_hat - C| > delta_c, not in M_s}       colour error: transparent Gaussian,
//                                                          unless the hit Gaussian is unstable
// of which a uniform 5% is drawn.  The draw of pixel p of frame f is output number
// f * H * W + p of the SplitMix64 stream (Steele, Lea and Flood, 2014) seeded by the caller,
// kept iff its top 24 bits are below floor(rate * 2^24).  Each pixel draws first, so the
// ~95% of pixels not drawn read no image at all.  Pixels without a valid input depth are in
// neither mask.  The new Gaussians are written in (frame, pixel) order: per-pixel kinds and
// per-block counts, one scan, then each block writes at its base.
#include "kernels.cuh"

namespace rtg {

namespace {

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// 0: nothing, 1: opaque Gaussian (M_s), 2: transparent Gaussian (M_c, stable hit).  The
// independent loads of a drawn pixel are issued together (two dependent levels, then the
// stability flag), so the rare drawn pixels cost a few memory latencies, not a chain.
__device__ __forceinline__ int add_kind(const AddArgs &a, int f, int64_t p) {
  const int64_t HW = (int64_t)a.H * a.W, q = (int64_t)f * HW + p;
  if ((uint32_t)(splitmix64_at(a.seed, (uint64_t)q) >> 40) >= a.t24) return 0;
  const float D = a.depth[q], alpha = a.ralpha[q], Dh = a.rdepth[q];
  const int32_t idx = a.index[q];
  float rc[8], ic[8];
  const int C8 = a.C < 8 ? a.C : 8;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int64_t o = ((int64_t)f * a.C + c) * HW + p;
    rc[c] = c < C8 ? a.rcolor[o] : 0.f;
    ic[c] = c < C8 ? a.color[o] : 0.f;
  }
  if (!(D > 0.f)) return 0;
  const float T_hat = __fsub_rn(1.f, alpha);
  if (T_hat > a.dT || fabsf(__fsub_rn(Dh, D)) > a.dd) return 1;
  float err = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c)
    if (c < C8) err = __fadd_rn(err, fabsf(__fsub_rn(rc[c], ic[c])));
  for (int c = 8; c < a.C; ++c) {
    const int64_t o = ((int64_t)f * a.C + c) * HW + p;
    err = __fadd_rn(err, fabsf(__fsub_rn(a.rcolor[o], a.color[o])));
  }
  if (!(err > a.thr_c)) return 0;
  if (idx < 0 || (int64_t)idx >= a.n) return 0;
  return a.unstable[idx] == 0 ? 2 : 0;
}

}  // namespace

// Per pixel its kind (a byte, kept for the write pass), per block the number of new
// Gaussians.  Thread t of block b owns pixels b * kSelPerBlock + 4t .. + 3.
__global__ void __launch_bounds__(kSelThreads) k_add_count(AddArgs a, int nb) {
  grid_dep_wait();
  __shared__ int s_w[kSelThreads / 32];
  const int f = blockIdx.y;
  const int64_t HW = (int64_t)a.H * a.W, p0 = (int64_t)blockIdx.x * kSelPerBlock + 4 * threadIdx.x;
  uint8_t *__restrict__ kinds = a.kinds + (int64_t)f * HW;
  int cnt = 0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t p = p0 + u;
    if (p < HW) {
      const int k = add_kind(a, f, p);
      kinds[p] = (uint8_t)k;
      cnt += k != 0;
    }
  }
  cnt = block_sum_int(cnt, s_w);
  if (threadIdx.x == 0) a.cnt[(int64_t)f * nb + blockIdx.x] = (uint32_t)cnt;
}

// One CTA: exclusive scan of the per-block counts over all frames (frame-major), total out.
__global__ void __launch_bounds__(1024) k_add_scan(AddArgs a, int total_blocks) {
  grid_dep_wait();
  __shared__ unsigned long long s_w[32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int per = (total_blocks + 1023) / 1024;
  const int e0 = min(total_blocks, tid * per), e1 = min(total_blocks, e0 + per);
  unsigned long long mine = 0;
  for (int e = e0; e < e1; ++e) mine += a.cnt[e];
  unsigned long long inc = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) s_w[wid] = inc;
  __syncthreads();
  unsigned long long run = inc - mine;
  for (int q = 0; q < wid; ++q) run += s_w[q];
  for (int e = e0; e < e1; ++e) {
    const uint32_t c = a.cnt[e];
    a.cnt[e] = (uint32_t)run;
    run += c;
  }
  if (tid == 1023) *a.count_out = (long long)run;
}

// Each thread reads the kinds of its 4 pixels, takes its slots from a block scan, and writes
// the new Gaussians of those pixels (those below the capacity).
__global__ void __launch_bounds__(kSelThreads) k_add_write(AddArgs a, AddFrames fr, int nb) {
  grid_dep_wait();
  __shared__ uint32_t s_w[kSelThreads / 32];
  const int f = blockIdx.y, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t HW = (int64_t)a.H * a.W, p0 = (int64_t)blockIdx.x * kSelPerBlock + 4 * tid;
  const uint8_t *__restrict__ kinds = a.kinds + (int64_t)f * HW;
  int k4[4];
  uint32_t mine = 0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    k4[u] = p0 + u < HW ? kinds[p0 + u] : 0;
    mine += k4[u] != 0;
  }
  uint32_t inc = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) s_w[wid] = inc;
  __syncthreads();
  int64_t slot = (int64_t)a.cnt[(int64_t)f * nb + blockIdx.x] + (inc - mine);
  for (int q = 0; q < wid; ++q) slot += s_w[q];
  if (mine == 0u) return;
  const AddCam &cam = fr.cam[f];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (k4[u] == 0) continue;
    if (slot < a.capacity) {
      const int64_t p = p0 + u, q = (int64_t)f * HW + p;
      const int x = (int)(p % a.W), y = (int)(p / a.W);
      const float D = a.depth[q];
      const float cx_ = ((float)x - cam.cx) / cam.fx * D, cy_ = ((float)y - cam.cy) / cam.fy * D;
      a.pix_out[slot] = (int32_t)q;
      a.kind_out[slot] = (uint8_t)k4[u];
#pragma unroll
      for (int r = 0; r < 3; ++r)
        a.pos_out[3 * slot + r] =
            fmaf(cam.R[3 * r], cx_, fmaf(cam.R[3 * r + 1], cy_, fmaf(cam.R[3 * r + 2], D, cam.t[r])));
      for (int c = 0; c < a.C; ++c) a.col_out[slot * a.C + c] = a.color[((int64_t)f * a.C + c) * HW + p];
      a.op_out[slot] = k4[u] == 1 ? a.op_opaque : a.op_transparent;
    }
    ++slot;
  }
}

void launch_add_candidates(const AddArgs &a, const AddFrames &fr, int F, cudaStream_t s) {
  const int64_t HW = (int64_t)a.H * a.W;
  const int nb = (int)((HW + kSelPerBlock - 1) / kSelPerBlock);
  const dim3 grid((unsigned)nb, (unsigned)F);
  launch(k_add_count, grid, kSelThreads, 0, s, a, nb);
  launch(k_add_scan, 1, 1024, 0, s, a, nb * F);
  launch(k_add_write, grid, kSelThreads, 0, s, a, fr, nb);
}

}  // namespace rtg
