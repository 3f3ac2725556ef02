// Fusion and state management (Section 3.2, "Gaussian optimization", Eq. 9, and "State
// management"): elementwise and scatter kernels over the per-Gaussian arrays.
//   - confidence: eta_i += 1 for each optimised Gaussian whose colour gradient is non-zero;
//   - fusion after a window: G = (1 - w) G_prev + w G', w = (eta' - eta_start) / eta', in
//     float32 with one rounding per operation, for every stored parameter;
//   - error count: per frame, each stable Gaussian hit (index map) by a pixel whose colour
//     (mean over channels) or depth error is above its threshold gets one count;
//   - transitions: stable with e > delta_e -> unstable (eta, e reset); unstable with
//     eta > delta_eta -> stable (e reset); unstable with k - t0 > delta_t -> removed;
//   - pruning: an order-preserving compaction of every per-Gaussian array.
#include "kernels.cuh"

namespace rtg {

__global__ void __launch_bounds__(256) k_confidence(int64_t nu, int C, const int32_t *__restrict__ ids,
                                                    const float *__restrict__ g_colors, int32_t *__restrict__ eta) {
  grid_dep_wait();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nu; k += (int64_t)gridDim.x * blockDim.x) {
    bool upd = false;
    for (int c = 0; c < C; ++c) upd |= g_colors[k * C + c] != 0.f;
    if (upd) eta[ids[k]] += 1;  // ids are distinct: one thread per Gaussian
  }
}

__device__ __forceinline__ float blend(float a, float b, float one_w, float w) {
  return __fadd_rn(__fmul_rn(one_w, a), __fmul_rn(w, b));
}

__global__ void __launch_bounds__(256) k_fuse(int64_t nu, int C, const int32_t *__restrict__ ids,
                                              const int32_t *__restrict__ eta_start,
                                              const int32_t *__restrict__ eta_now, FuseArrays a) {
  grid_dep_wait();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nu; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = ids[k];
    const int32_t e1 = eta_now[i], e0 = eta_start[i];
    if (e1 <= 0) continue;  // never updated: G' = G_prev
    const float w = __fdiv_rn((float)(e1 - e0), (float)e1), one_w = __fsub_rn(1.f, w);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      a.means[3 * i + r] = blend(a.means[3 * i + r], a.u_means[3 * k + r], one_w, w);
      a.scales[3 * i + r] = blend(a.scales[3 * i + r], a.u_scales[3 * k + r], one_w, w);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) a.quats[4 * i + r] = blend(a.quats[4 * i + r], a.u_quats[4 * k + r], one_w, w);
    a.opacity[i] = blend(a.opacity[i], a.u_opacity[k], one_w, w);
    for (int c = 0; c < C; ++c) a.colors[(int64_t)C * i + c] = blend(a.colors[(int64_t)C * i + c], a.u_colors[(int64_t)C * k + c], one_w, w);
  }
}

// One bit per frame: pixels of frame f that err set bit f of their stable hit Gaussian.
__global__ void __launch_bounds__(256) k_error_mark(int F, int C, int64_t HW, const float *__restrict__ rcolor,
                                                    const float *__restrict__ rdepth,
                                                    const int32_t *__restrict__ index_map,
                                                    const float *__restrict__ color, const float *__restrict__ depth,
                                                    const uint8_t *__restrict__ unstable, int64_t n, float thr_c,
                                                    float dd, uint32_t *__restrict__ bits) {
  grid_dep_wait();
  const int64_t NP = (int64_t)F * HW;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < NP; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t idx = index_map[q];
    if (idx < 0 || (int64_t)idx >= n) continue;
    const int64_t f = q / HW, p = q - f * HW;
    const float D = depth[q];
    bool bad = D > 0.f && fabsf(__fsub_rn(rdepth[q], D)) > dd;
    if (!bad) {
      float err = 0.f;
      for (int c = 0; c < C; ++c) {
        const int64_t o = (f * C + c) * HW + p;
        err = __fadd_rn(err, fabsf(__fsub_rn(rcolor[o], color[o])));
      }
      bad = err > thr_c;
    }
    if (bad && unstable[idx] == 0) {
      const uint32_t bit = 1u << f;
      if ((bits[idx] & bit) == 0u) atomicOr(&bits[idx], bit);  // read first: most pixels repeat a bit
    }
  }
}

__global__ void __launch_bounds__(256) k_error_accum(int64_t n, uint32_t *__restrict__ bits, int32_t *__restrict__ err) {
  grid_dep_wait();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t b = bits[i];
    if (b) {
      err[i] += __popc(b);
      bits[i] = 0u;  // clear for the next call
    }
  }
}

__global__ void __launch_bounds__(256) k_update_states(int64_t n, int32_t frame, const int32_t *__restrict__ t0,
                                                       rtg_state_params p, uint8_t *__restrict__ unstable,
                                                       int32_t *__restrict__ eta, int32_t *__restrict__ err,
                                                       uint8_t *__restrict__ remove) {
  grid_dep_wait();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint8_t rm = 0;
    if (unstable[i] == 0) {
      if (err[i] > p.delta_e) {
        unstable[i] = 1;
        eta[i] = 0;
        err[i] = 0;
      }
    } else if (eta[i] > p.delta_eta) {
      unstable[i] = 0;
      err[i] = 0;
    } else if ((int64_t)frame - (int64_t)t0[i] > (int64_t)p.delta_t) {
      rm = 1;
    }
    remove[i] = rm;
  }
}

// Compaction: per-block kept counts (1024 Gaussians per block), one scan, then each block
// writes its kept rows at its base in order.  Lane L of warp w handles Gaussian
// chunk * 256 + 32 w + L, so a warp reads and writes consecutive rows.
constexpr int kCompactPer = 1024;

__global__ void __launch_bounds__(256) k_compact_count(int64_t n, const uint8_t *__restrict__ remove,
                                                       int32_t *__restrict__ cnt) {
  grid_dep_wait();
  __shared__ int s_w[8];
  const int64_t i0 = (int64_t)blockIdx.x * kCompactPer + threadIdx.x;
  int c = 0;
#pragma unroll
  for (int u = 0; u < kCompactPer / 256; ++u) {
    const int64_t i = i0 + u * 256;
    c += (i < n && remove[i] == 0) ? 1 : 0;
  }
  c = block_sum_int(c, s_w);
  if (threadIdx.x == 0) cnt[blockIdx.x] = c;
}

__global__ void __launch_bounds__(1024) k_compact_scan(int nb, int32_t *__restrict__ cnt, long long *count_out) {
  grid_dep_wait();
  __shared__ long long s_w[32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int per = (nb + 1023) / 1024;
  const int e0 = min(nb, tid * per), e1 = min(nb, e0 + per);
  long long mine = 0;
  for (int e = e0; e < e1; ++e) mine += cnt[e];
  long long inc = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const long long v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) s_w[wid] = inc;
  __syncthreads();
  long long run = inc - mine;
  for (int q = 0; q < wid; ++q) run += s_w[q];
  for (int e = e0; e < e1; ++e) {
    const int32_t c = cnt[e];
    cnt[e] = (int32_t)run;
    run += c;
  }
  if (tid == 1023) *count_out = run;
}

__global__ void __launch_bounds__(256) k_compact_write(int64_t n, int C, const uint8_t *__restrict__ remove,
                                                       const int32_t *__restrict__ base, rtg_map_arrays in,
                                                       rtg_map_arrays out) {
  grid_dep_wait();
  __shared__ int s_w[8];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  int64_t run = base[blockIdx.x];  // kept rows of earlier blocks and chunks
#pragma unroll 1
  for (int u = 0; u < kCompactPer / 256; ++u) {
    const int64_t i = (int64_t)blockIdx.x * kCompactPer + u * 256 + tid;
    const bool keep = i < n && remove[i] == 0;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) s_w[wid] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int c = s_w[q];
      before += q < wid ? c : 0;
      total += c;
    }
    __syncthreads();
    if (keep) {
      const int64_t j = run + before + __popc(bal & lanemask_lt());
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        out.means[3 * j + r] = in.means[3 * i + r];
        out.scales[3 * j + r] = in.scales[3 * i + r];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) out.quats[4 * j + r] = in.quats[4 * i + r];
      out.opacity[j] = in.opacity[i];
      for (int c = 0; c < C; ++c) out.colors[(int64_t)C * j + c] = in.colors[(int64_t)C * i + c];
      out.unstable[j] = in.unstable[i];
      out.eta[j] = in.eta[i];
      out.err[j] = in.err[i];
      out.t0[j] = in.t0[i];
    }
    run += total;
  }
}

static int elementwise_grid(const void *kernel, int64_t work) {
  const int wave = resident_grid(kernel, 256);
  const int64_t need = (work + 255) / 256;
  return (int)(need < wave ? (need > 0 ? need : 1) : wave);
}

void launch_confidence(int64_t nu, int C, const int32_t *ids, const float *g_colors, int32_t *eta, cudaStream_t s) {
  launch(k_confidence, elementwise_grid((const void *)k_confidence, nu), 256, 0, s, nu, C, ids, g_colors, eta);
}

void launch_fuse(int64_t nu, int C, const int32_t *ids, const int32_t *eta_start, const int32_t *eta_now,
                 const FuseArrays &a, cudaStream_t s) {
  launch(k_fuse, elementwise_grid((const void *)k_fuse, nu), 256, 0, s, nu, C, ids, eta_start, eta_now, a);
}

void launch_error_count(int F, int C, int64_t HW, const float *rcolor, const float *rdepth, const int32_t *index_map,
                        const float *color, const float *depth, const uint8_t *unstable, int64_t n, float thr_c,
                        float dd, uint32_t *bits, int32_t *err, cudaStream_t s) {
  launch(k_error_mark, elementwise_grid((const void *)k_error_mark, (int64_t)F * HW), 256, 0, s,
      F, C, HW, rcolor, rdepth, index_map, color, depth, unstable, n, thr_c, dd, bits);
  launch(k_error_accum, elementwise_grid((const void *)k_error_accum, n), 256, 0, s, n, bits, err);
}

void launch_update_states(int64_t n, int32_t frame, const int32_t *t0, const rtg_state_params &p, uint8_t *unstable,
                          int32_t *eta, int32_t *err, uint8_t *remove, cudaStream_t s) {
  launch(k_update_states, elementwise_grid((const void *)k_update_states, n), 256, 0, s, n, frame, t0, p, unstable, eta,
                                                                                     err, remove);
}

void launch_compact(int64_t n, int C, const uint8_t *remove, int32_t *block_cnt, const rtg_map_arrays &in,
                    const rtg_map_arrays &out, long long *count_out, cudaStream_t s) {
  const int nb = (int)((n + kCompactPer - 1) / kCompactPer);
  launch(k_compact_count, nb, 256, 0, s, n, remove, block_cnt);
  launch(k_compact_scan, 1, 1024, 0, s, nb, block_cnt, count_out);
  launch(k_compact_write, nb, 256, 0, s, n, C, remove, block_cnt, in, out);
}

}  // namespace rtg
