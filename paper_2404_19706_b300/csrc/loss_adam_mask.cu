// L1 losses (Section 3.2, Eq. 7/8), Adam on the unstable subset (Supplement C learning
// rates), unstable-subset gather/scatter, and the unstable-pixel mask (Supplement B,
// Eq. S2 plus the 50% tile rule).
#include <algorithm>

#include "kernels.cuh"
#include "project.cuh"

namespace rtg {

// --------------------------------------------------------------------------- L1 loss
// Reduction: |C - C_hat| over masked pixels and channels; |D - D_hat| over masked pixels
// with a rendered intersection (D_hat != -1) and a valid input depth (D > 0).  Block
// partials are summed in a fixed order by the last block, so the loss is deterministic.
__global__ void __launch_bounds__(256) k_loss_reduce(Work w, int F, int C, int H, int W,
                                                     const float *__restrict__ color,
                                                     const float *__restrict__ depth,
                                                     const float *__restrict__ tcolor,
                                                     const float *__restrict__ tdepth,
                                                     const uint8_t *__restrict__ mask, float w_c, float w_d,
                                                     float *__restrict__ loss_out) {
  grid_dep_wait();
  __shared__ float s_red[4][8];
  __shared__ bool s_last;
  const int64_t HW = (int64_t)H * W, NP = (int64_t)F * HW;
  float sc = 0.f, sd = 0.f, np = 0.f, nd = 0.f;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < NP; p += (int64_t)gridDim.x * blockDim.x) {
    if (mask != nullptr && mask[p] == 0) continue;
    const int64_t f = p / HW, q = p - f * HW;
    for (int c = 0; c < C; ++c) {
      const int64_t o = (f * C + c) * HW + q;
      sc += fabsf(color[o] - tcolor[o]);
    }
    np += 1.f;
    if (depth[p] != -1.f && tdepth[p] > 0.f) {
      sd += fabsf(depth[p] - tdepth[p]);
      nd += 1.f;
    }
  }
  float v[4] = {sc, sd, np, nd};
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0) s_red[k][wid] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    float t = 0.f;
    for (int k = 0; k < 8; ++k) t += s_red[threadIdx.x][k];
    w.loss_part[blockIdx.x * 4 + threadIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(w.loss_done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  // last block: every thread sums a strided share of the block partials (fixed order), then
  // a fixed-order reduction across the threads keeps the result deterministic
  __threadfence();
  __shared__ float s_tot[4][256];
  float t[4] = {0.f, 0.f, 0.f, 0.f};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < 4; ++k) t[k] += __ldcg(w.loss_part + b * 4 + k);
#pragma unroll
  for (int k = 0; k < 4; ++k) s_tot[k][threadIdx.x] = t[k];
  __syncthreads();
  for (int stride = 128; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride)
#pragma unroll
      for (int k = 0; k < 4; ++k) s_tot[k][threadIdx.x] += s_tot[k][threadIdx.x + stride];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const float sc = s_tot[0][0], sd = s_tot[1][0], np = s_tot[2][0], nd = s_tot[3][0];
    const float Lc = np > 0.f ? sc / (np * (float)C) : 0.f;
    const float Ld = nd > 0.f ? sd / nd : 0.f;
    loss_out[0] = w_c * Lc + w_d * Ld;
    loss_out[1] = Lc;
    loss_out[2] = Ld;
    w.loss_scal[4] = np > 0.f ? w_c / (np * (float)C) : 0.f;
    w.loss_scal[5] = nd > 0.f ? w_d / nd : 0.f;
    w.loss_scal[1] = Lc;
    w.loss_scal[2] = Ld;
    w.counters[kDepthPix] = (unsigned long long)nd;
    *w.loss_done = 0u;
  }
}

// The last fused L1 loss's pixel counts and sums, for a caller that splits one batch of
// keyframes over several GPUs: out = (P, P_d, sum |C_hat - C| over the P x C values,
// sum |D_hat - D| over the P_d depth pixels), as doubles (summed over ranks by the caller).
__global__ void k_loss_counts(Work w, int C, double *__restrict__ out) {
  grid_dep_wait();
  if (threadIdx.x != 0) return;
  const double np = (double)w.counters[kMaskedPix], nd = (double)w.counters[kDepthPix];
  out[0] = np;
  out[1] = nd;
  out[2] = (double)w.loss_scal[1] * np * (double)C;
  out[3] = (double)w.loss_scal[2] * nd;
}

// The backward's L1 gradient scales for the loss of the whole batch (Eq. 7 means over every
// rank's pixels): w_c / (P_total C) and w_d / P_d,total from the summed counts, and, with
// loss_out, that loss (L, L_color, L_depth) from the summed sums.
__global__ void k_set_loss_scales(Work w, int C, const double *__restrict__ tot, float w_c, float w_d,
                                  float *__restrict__ loss_out) {
  grid_dep_wait();
  if (threadIdx.x != 0) return;
  const double np = tot[0], nd = tot[1];
  w.loss_scal[4] = np > 0.0 ? (float)((double)w_c / (np * (double)C)) : 0.f;
  w.loss_scal[5] = nd > 0.0 ? (float)((double)w_d / nd) : 0.f;
  if (loss_out != nullptr) {
    const float Lc = np > 0.0 ? (float)(tot[2] / (np * (double)C)) : 0.f;
    const float Ld = nd > 0.0 ? (float)(tot[3] / nd) : 0.f;
    loss_out[0] = w_c * Lc + w_d * Ld;
    loss_out[1] = Lc;
    loss_out[2] = Ld;
  }
}

void launch_loss_counts(const Work &w, int C, double *out, cudaStream_t s) {
  launch(k_loss_counts, 1, 32, 0, s, w, C, out);
}

void launch_set_loss_scales(const Work &w, int C, const double *tot, float w_c, float w_d, float *loss_out,
                            cudaStream_t s) {
  launch(k_set_loss_scales, 1, 32, 0, s, w, C, tot, w_c, w_d, loss_out);
}

// Fused L1 (Eq. 7/8): sums the forward's per-(tile, 32-pixel group) partials in a fixed
// order (only groups that held masked pixels wrote them), then the loss and its gradient
// scales.  2^gshift groups per tile.  Block b sums a fixed range of tiles (Kahan per thread,
// fixed-order tree across threads); the last block to finish sums the block partials in
// block order, so the loss does not depend on scheduling.  The sums are FP32 (B300's FP64
// rate is a small fraction of its FP32 rate).
__global__ void __launch_bounds__(256) k_loss_finalize(Work w, int FT, int gshift, int C, float w_c, float w_d,
                                                       float *__restrict__ loss_out) {
  grid_dep_wait();
  __shared__ float s_t[3][256];
  __shared__ bool s_last;
  const int per = (FT + (int)gridDim.x - 1) / (int)gridDim.x;
  const int t0 = (int)blockIdx.x * per, t1 = min(FT, t0 + per);
  float t[3] = {0.f, 0.f, 0.f}, comp[3] = {0.f, 0.f, 0.f};
  for (int tile = t0 + (int)threadIdx.x; tile < t1; tile += (int)blockDim.x) {
    const int nw = (int)((w.tile_npix[tile] + 31u) / 32u);
    for (int k = 0; k < nw; ++k) {
      const float *lp = w.tile_loss + (((int64_t)tile << gshift) + k) * 4;
#pragma unroll
      for (int q = 0; q < 3; ++q) {  // Kahan summation
        const float y = lp[q] - comp[q];
        const float tt = t[q] + y;
        comp[q] = (tt - t[q]) - y;
        t[q] = tt;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) s_t[q][threadIdx.x] = t[q];
  __syncthreads();
  for (int stride = 128; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride)
#pragma unroll
      for (int q = 0; q < 3; ++q) s_t[q][threadIdx.x] += s_t[q][threadIdx.x + stride];
    __syncthreads();
  }
  if (threadIdx.x < 3) w.loss_part[blockIdx.x * 4 + threadIdx.x] = s_t[threadIdx.x][0];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(w.loss_done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  float a[3] = {0.f, 0.f, 0.f};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < 3; ++q) a[q] += __ldcg(w.loss_part + b * 4 + q);
#pragma unroll
  for (int q = 0; q < 3; ++q) s_t[q][threadIdx.x] = a[q];
  __syncthreads();
  for (int stride = 128; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride)
#pragma unroll
      for (int q = 0; q < 3; ++q) s_t[q][threadIdx.x] += s_t[q][threadIdx.x + stride];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const float np = (float)w.counters[kMaskedPix], nd = s_t[2][0];
    const float Lc = np > 0.f ? s_t[0][0] / (np * (float)C) : 0.f;
    const float Ld = nd > 0.f ? s_t[1][0] / nd : 0.f;
    loss_out[0] = w_c * Lc + w_d * Ld;
    loss_out[1] = Lc;
    loss_out[2] = Ld;
    w.loss_scal[4] = np > 0.f ? w_c / (np * (float)C) : 0.f;
    w.loss_scal[5] = nd > 0.f ? w_d / nd : 0.f;
    w.loss_scal[1] = Lc;
    w.loss_scal[2] = Ld;
    w.counters[kDepthPix] = (unsigned long long)nd;
    *w.loss_done = 0u;
  }
}

// --------------------------------------------------------------------------- L_reg
// Transparent-Gaussian regulariser (Section 3.2, the L_reg term of Eq. 8): w_reg times the
// mean squared difference of the position, raw quaternion and scale components of the
// optimised Gaussians with opacity < alpha_split from their values when added.  Per-block
// partial sums in a fixed grid, the last block (ticket) adds them in block order and
// stores the loss and the gradient factor 2 w_reg / (10 n_t); the second kernel adds the
// gradient.
// The transparent-Gaussian regulariser: every row's values are loaded with its opacity (no
// load waits on the opacity test), the block sums go through warp shuffles, and the last
// block sums the per-block partials with all its threads.
__device__ __forceinline__ float reg_d2(const RegArgs &a, int64_t k) {
  float d2 = 0.f;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float dm = a.means[3 * k + r] - a.means0[3 * k + r], ds = a.scales[3 * k + r] - a.scales0[3 * k + r];
    d2 = fmaf(dm, dm, fmaf(ds, ds, d2));
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const float dq = a.quats[4 * k + r] - a.quats0[4 * k + r];
    d2 = fmaf(dq, dq, d2);
  }
  return d2;
}

// Sums of two values over the block (result in every thread); s holds 2 x 8 floats.
__device__ __forceinline__ float2 block_sum2(float x, float y, float *s) {
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, o);
    y += __shfl_xor_sync(0xffffffffu, y, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    s[wid] = x;
    s[8 + wid] = y;
  }
  __syncthreads();
  float2 r = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    r.x += s[k];
    r.y += s[8 + k];
  }
  return r;
}

__global__ void __launch_bounds__(256) k_reg_reduce(RegArgs a, float *__restrict__ loss_out) {
  grid_dep_wait();
  __shared__ float s_w[16];
  __shared__ int s_last;
  float sum = 0.f, cnt = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  constexpr int U = 4;  // rows a thread has in flight
  for (int64_t k0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k0 < a.nu; k0 += U * stride) {
    bool t[U];
    float d2[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t k = k0 + u * stride;
      t[u] = k < a.nu && a.opacity[k] < a.alpha_split;
      d2[u] = k < a.nu ? reg_d2(a, k) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      sum += t[u] ? d2[u] : 0.f;
      cnt += t[u] ? 1.f : 0.f;
    }
  }
  const float2 blk = block_sum2(sum, cnt, s_w);
  if (threadIdx.x == 0) {
    a.part[2 * blockIdx.x] = blk.x;
    a.part[2 * blockIdx.x + 1] = blk.y;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(a.done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  float tot = 0.f, n = 0.f;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    tot += __ldcg(a.part + 2 * b);
    n += __ldcg(a.part + 2 * b + 1);
  }
  const float2 all = block_sum2(tot, n, s_w);
  if (threadIdx.x == 0) {
    const float denom = 10.f * all.y;
    *loss_out = all.y > 0.f ? a.w_reg * all.x / denom : 0.f;
    *a.scale = all.y > 0.f ? 2.f * a.w_reg / denom : 0.f;
    *a.done = 0u;
  }
}

__global__ void __launch_bounds__(256) k_reg_grad(RegArgs a) {
  grid_dep_wait();
  const float sc = *a.scale;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.nu; k += (int64_t)gridDim.x * blockDim.x) {
    const bool t = a.opacity[k] < a.alpha_split;
    float dm[3], ds[3], dq[4];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      dm[r] = a.means[3 * k + r] - a.means0[3 * k + r];
      ds[r] = a.scales[3 * k + r] - a.scales0[3 * k + r];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) dq[r] = a.quats[4 * k + r] - a.quats0[4 * k + r];
    if (!t) continue;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      a.g_means[3 * k + r] += sc * dm[r];
      a.g_scales[3 * k + r] += sc * ds[r];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) a.g_quats[4 * k + r] += sc * dq[r];
  }
}

void launch_transparent_reg(const RegArgs &a, float *loss_out, cudaStream_t s) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(kLossBlocks, (a.nu + 255) / 256));
  launch(k_reg_reduce, blocks, 256, 0, s, a, loss_out);
  // one row a thread: the rows' loads all start at once
  const int64_t rows = (a.nu + 255) / 256;
  launch(k_reg_grad, (unsigned)std::max<int64_t>(1, rows), 256, 0, s, a);
}

void launch_loss_finalize(const Work &w, int FT, int gshift, int C, float w_c, float w_d, float *loss_out,
                          cudaStream_t s) {
  const int blocks = std::max(1, std::min(kLossBlocks, (FT + 255) / 256));
  launch(k_loss_finalize, blocks, 256, 0, s, w, FT, gshift, C, w_c, w_d, loss_out);
}

__device__ __forceinline__ float signf_(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

__global__ void __launch_bounds__(256) k_loss_grad(Work w, int F, int C, int H, int W,
                                                   const float *__restrict__ color, const float *__restrict__ depth,
                                                   const float *__restrict__ tcolor,
                                                   const float *__restrict__ tdepth,
                                                   const uint8_t *__restrict__ mask, float *__restrict__ dL_dcolor,
                                                   float *__restrict__ dL_ddepth) {
  grid_dep_wait();
  const int64_t HW = (int64_t)H * W, NP = (int64_t)F * HW;
  const float s_c = w.loss_scal[4], s_d = w.loss_scal[5];
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < NP; p += (int64_t)gridDim.x * blockDim.x) {
    const bool m = mask == nullptr || mask[p] != 0;
    const int64_t f = p / HW, q = p - f * HW;
    for (int c = 0; c < C; ++c) {
      const int64_t o = (f * C + c) * HW + q;
      dL_dcolor[o] = m ? s_c * signf_(color[o] - tcolor[o]) : 0.f;
    }
    const bool vd = m && depth[p] != -1.f && tdepth[p] > 0.f;
    dL_ddepth[p] = vd ? s_d * signf_(depth[p] - tdepth[p]) : 0.f;
  }
}

// --------------------------------------------------------------------------- Adam
// Kingma & Ba, Algorithm 1, with bc1 = 1 / (1 - beta1^t) and bc2_sqrt = 1 / sqrt(1 - beta2^t).
__device__ __forceinline__ float adam_delta(float g, float &m, float &v, float lr, const rtg_adam_params &hp,
                                            float bc1, float bc2_sqrt) {
  m = fmaf(hp.beta1, m, (1.f - hp.beta1) * g);
  v = fmaf(hp.beta2, v, (1.f - hp.beta2) * g * g);
  return lr * (m * bc1) * __frcp_rn(fmaf(sqrtf(v), bc2_sqrt, hp.eps));
}

// Parameter groups of the compact unstable set (means, scales, quats, opacity, colours);
// m and v hold the groups one after another in this order.
struct AdamGroups {
  float *param[5];
  const float *grad[5];
  float lr[5];
  int64_t begin[6];  // element offsets of the groups in m / v; begin[5] = total
  int64_t quad[6];   // the groups' first quads (runs of 4 elements) in one sequence; quad[5] = total
  int vec[5];        // the group's four streams are 16-byte aligned: quads move as float4
  // colour group: values at row positions >= dc (dc > 0) use lr_rest (the SH coefficients
  // of degree >= 1); width = values per row
  float lr_rest;
  int width, dc;
};

// Adam is element-wise, so the kernel walks the parameter groups as one sequence of quads
// (4 consecutive elements of one group; a group's last quad may be short).  A thread takes
// kAdamRounds quads per round, a grid's width apart, and issues every load of the round
// (float4 per stream where the group is aligned) before it computes, so each thread has up
// to 8 vector loads in flight and every stream (param, grad, m, v) moves in coalesced
// 16-byte accesses.
constexpr int kAdamRounds = 2;

__device__ __forceinline__ float4 ld4(const float *p, int64_t e, int cnt, bool vec) {
  if (vec && cnt == 4) return *reinterpret_cast<const float4 *>(p + e);
  float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
  if (cnt > 0) r.x = p[e];
  if (cnt > 1) r.y = p[e + 1];
  if (cnt > 2) r.z = p[e + 2];
  if (cnt > 3) r.w = p[e + 3];
  return r;
}

__device__ __forceinline__ void st4(float *p, int64_t e, int cnt, bool vec, const float4 &r) {
  if (vec && cnt == 4) {
    *reinterpret_cast<float4 *>(p + e) = r;
    return;
  }
  if (cnt > 0) p[e] = r.x;
  if (cnt > 1) p[e + 1] = r.y;
  if (cnt > 2) p[e + 2] = r.z;
  if (cnt > 3) p[e + 3] = r.w;
}

// early: the kernel in front on the stream writes neither the parameters nor the moments
// (the projection backward, which writes the gradients): a thread's first round of
// parameter and moment loads, and the bias corrections, go out before the wait on that
// kernel, so they overlap its tail; the gradient loads come after it.
__global__ void __launch_bounds__(256) k_adam(AdamGroups G, float *__restrict__ m, float *__restrict__ v,
                                              rtg_adam_params hp, float bc1, float bc2_sqrt,
                                              int32_t *__restrict__ step_dev, int early) {
  bool waited = early == 0;
  if (waited) grid_dep_wait();
  // Device step counter: step_dev[0] completed steps, step_dev[1] a ticket.  Every block
  // takes t = step_dev[0] + 1 when it starts; the last block to finish stores t, after
  // every block has read the old value.
  if (step_dev != nullptr) {  // bias corrections of step t, once per block
    __shared__ float s_bc[2];
    if (threadIdx.x == 0) {
      const float t = (float)(step_dev[0] + 1);
      s_bc[0] = 1.f / (1.f - powf(hp.beta1, t));
      s_bc[1] = rsqrtf(1.f - powf(hp.beta2, t));
    }
    __syncthreads();
    bc1 = s_bc[0];
    bc2_sqrt = s_bc[1];
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, nq = G.quad[5];
  for (int64_t q0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q0 < nq; q0 += kAdamRounds * stride) {
    float4 x[kAdamRounds], g[kAdamRounds], mm[kAdamRounds], vv[kAdamRounds];
    int grp[kAdamRounds], cnt[kAdamRounds];
    int64_t e[kAdamRounds];
#pragma unroll
    for (int r = 0; r < kAdamRounds; ++r) {
      const int64_t q = q0 + r * stride;
      grp[r] = 0;
      cnt[r] = 0;
      e[r] = 0;
      if (q < nq) {
        int k = 0;
#pragma unroll
        for (int j = 1; j < 5; ++j) k += q >= G.quad[j] ? 1 : 0;
        grp[r] = k;
        e[r] = 4 * (q - G.quad[k]);
        const int64_t n = G.begin[k + 1] - G.begin[k];
        cnt[r] = (int)min((int64_t)4, n - e[r]);
      }
      const int k = grp[r];
      const bool vec = G.vec[k] != 0;
      x[r] = ld4(G.param[k], e[r], cnt[r], vec);
      mm[r] = ld4(m + G.begin[k], e[r], cnt[r], vec);
      vv[r] = ld4(v + G.begin[k], e[r], cnt[r], vec);
    }
    if (!waited) {
      grid_dep_wait();
      waited = true;
    }
#pragma unroll
    for (int r = 0; r < kAdamRounds; ++r) g[r] = ld4(G.grad[grp[r]], e[r], cnt[r], G.vec[grp[r]] != 0);
#pragma unroll
    for (int r = 0; r < kAdamRounds; ++r) {
      if (cnt[r] == 0) continue;
      const int k = grp[r];
      const float lr = G.lr[k];
      float xs[4] = {x[r].x, x[r].y, x[r].z, x[r].w}, gs[4] = {g[r].x, g[r].y, g[r].z, g[r].w};
      float ms[4] = {mm[r].x, mm[r].y, mm[r].z, mm[r].w}, vs[4] = {vv[r].x, vv[r].y, vv[r].z, vv[r].w};
      // the group is the same for (nearly) a whole warp, so these branches do not diverge
      if (k == 1) {  // theta = log s, dL/dtheta = s dL/ds, s <- s exp(-step)
#pragma unroll
        for (int u = 0; u < 4; ++u) xs[u] *= expf(-adam_delta(gs[u] * xs[u], ms[u], vs[u], lr, hp, bc1, bc2_sqrt));
      } else if (k == 4 && G.dc > 0) {  // lr_rest past the first dc values of a colour row
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t j = e[r] + u;
          const int pos = j < (1ll << 32) ? (int)((uint32_t)j % (uint32_t)G.width) : (int)(j % G.width);
          xs[u] -= adam_delta(gs[u], ms[u], vs[u], pos >= G.dc ? G.lr_rest : lr, hp, bc1, bc2_sqrt);
        }
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) xs[u] -= adam_delta(gs[u], ms[u], vs[u], lr, hp, bc1, bc2_sqrt);
      }
      const bool vec = G.vec[k] != 0;
      st4(G.param[k], e[r], cnt[r], vec, make_float4(xs[0], xs[1], xs[2], xs[3]));
      st4(m + G.begin[k], e[r], cnt[r], vec, make_float4(ms[0], ms[1], ms[2], ms[3]));
      st4(v + G.begin[k], e[r], cnt[r], vec, make_float4(vs[0], vs[1], vs[2], vs[3]));
    }
  }
  if (!waited) grid_dep_wait();  // a thread without quads still completes only after the kernel in front
  if (step_dev != nullptr) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned ticket = atomicAdd(reinterpret_cast<unsigned *>(step_dev + 1), 1u);
      if (ticket == gridDim.x - 1) {
        step_dev[0] += 1;
        step_dev[1] = 0;
      }
    }
  }
}

__global__ void k_gather(int64_t nu, int C, const int32_t *__restrict__ ids, const float *__restrict__ means,
                         const float *__restrict__ scales, const float *__restrict__ quats,
                         const float *__restrict__ opacity, const float *__restrict__ colors, float *__restrict__ um,
                         float *__restrict__ us, float *__restrict__ uq, float *__restrict__ uo,
                         float *__restrict__ uc) {
  grid_dep_wait();
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nu) return;
  const int64_t i = ids[k];
  for (int j = 0; j < 3; ++j) {
    um[3 * k + j] = means[3 * i + j];
    us[3 * k + j] = scales[3 * i + j];
  }
  for (int j = 0; j < 4; ++j) uq[4 * k + j] = quats[4 * i + j];
  uo[k] = opacity[i];
  for (int c = 0; c < C; ++c) uc[(int64_t)C * k + c] = colors[(int64_t)C * i + c];
}

__global__ void k_scatter(int64_t nu, int C, const int32_t *__restrict__ ids, const float *__restrict__ um,
                          const float *__restrict__ us, const float *__restrict__ uq, const float *__restrict__ uo,
                          const float *__restrict__ uc, float *__restrict__ means, float *__restrict__ scales,
                          float *__restrict__ quats, float *__restrict__ opacity, float *__restrict__ colors) {
  grid_dep_wait();
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nu) return;
  const int64_t i = ids[k];
  for (int j = 0; j < 3; ++j) {
    means[3 * i + j] = um[3 * k + j];
    scales[3 * i + j] = us[3 * k + j];
  }
  for (int j = 0; j < 4; ++j) quats[4 * i + j] = uq[4 * k + j];
  opacity[i] = uo[k];
  for (int c = 0; c < C; ++c) colors[(int64_t)C * i + c] = uc[(int64_t)C * k + c];
}

// --------------------------------------------------------------------------- unstable mask
// One CTA per 16x16 tile (the tile grid of the rule).  The unstable Gaussians were
// projected and bucketed into every tile their support box touches; a pixel is covered
// when one footprint reaches alpha_min there (T_unstable < 1 in Eq. S2), with the same
// projection and footprint expression as the forward.  Each warp owns an 8 x 4 pixel block
// (the tile taken in Z order) and walks the tile's bucket alone, in batches of 32 records of which it keeps only those
// whose support box reaches its pixel box (a conservative test), and stops as soon as all
// its pixels are covered.  The tile rule (Supplement B) is applied in the same kernel: a
// tile with fewer than `discard` of its in-image pixels covered is cleared.  Every
// in-image pixel of the mask is written.
// kMode = kCoverFusedSame (rtg_render_forward_masked, render tiles = 16 x 16): the tile's
// masked-pixel count and pixel list replace the coverage pass's, and the pair counters are
// cleared for the second binning.  kCoverFusedOther (other render tiles): only the staging
// counter is cleared; a tile-mask pass over the render grid follows.
template <int kMode>
__global__ void __launch_bounds__(kTilePix) k_mask_cover_tiles(Work w, Prm prm, int64_t N, int T, int H4,
                                                               uint8_t *__restrict__ mask) {
  grid_dep_wait();
  constexpr int NW = kTilePix / 32;
  __shared__ float4 s_rec[NW][2][32];
  __shared__ int s_wcnt[NW];
  if (w.counters[kSkip] != 0ull) return;
  const int tile = blockIdx.x;
  const int f = tile / T, lt = tile - f * T;
  const DevCam &cam = w.cams[f];
  const int tx = lt % cam.mtiles_x, ty = lt / cam.mtiles_x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int rpix = tile_order_pixel(tid, kTileShift, kTileShift);  // Z order: a warp owns an 8 x 4 block
  const int px = tx * kTile + (rpix & (kTile - 1)), py = ty * kTile + (rpix >> kTileShift);
  const bool in = px < cam.W && py < cam.H;
  const float fpx = (float)px, fpy = (float)py;
  const uint32_t off = w.tile_offset[tile];
  const uint32_t n = w.tile_offset[tile + 1] - off;
  const float4 *__restrict__ rec = w.rec_hot + (int64_t)f * N * H4;
  const float2 *__restrict__ box = w.rec_box + (int64_t)f * N;
  // the warp's pixel box (an 8 x 4 block; pixels outside the image are not in it)
  const int bx0 = __reduce_min_sync(0xffffffffu, in ? px : 0x7fffffff);
  const int bx1 = __reduce_max_sync(0xffffffffu, in ? px : -1);
  const int by0 = __reduce_min_sync(0xffffffffu, in ? py : 0x7fffffff);
  const int by1 = __reduce_max_sync(0xffffffffu, in ? py : -1);
  const float wcx = 0.5f * (float)(bx0 + bx1), whx = 0.5f * (float)(bx1 - bx0);
  const float wcy = 0.5f * (float)(by0 + by1), why = 0.5f * (float)(by1 - by0);
  bool cov = false;
  // Software pipeline over the batches of 32 records: while batch b is tested, the records
  // of batch b + 1 and the Gaussian indices of batch b + 2 are in flight, so a batch costs
  // about one L2 round trip instead of the chain index -> record -> record.
  auto gid_of = [&](uint32_t b0_) -> uint32_t {
    const uint32_t j = b0_ + lane;
    return j < n ? (uint32_t)w.keys[off + j] : 0xffffffffu;
  };
  auto fetch = [&](uint32_t gid, float4 &a0, float4 &a1, float2 &bb) {
    if (gid != 0xffffffffu) {
      bb = box[gid];
      a0 = rec[(int64_t)gid * H4];
      a1 = rec[(int64_t)gid * H4 + 1];
    }
  };
  float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
  float2 bb = make_float2(0.f, 0.f);
  uint32_t gcur = gid_of(0);
  uint32_t gnext = n > 32 ? gid_of(32) : 0xffffffffu;
  fetch(gcur, r0, r1, bb);
  for (uint32_t b0 = 0; b0 < n; b0 += 32) {
    if (__all_sync(0xffffffffu, cov || !in)) break;
    float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0;
    float2 nbb = make_float2(0.f, 0.f);
    fetch(gnext, n0, n1, nbb);
    const uint32_t gafter = b0 + 64 < n ? gid_of(b0 + 64) : 0xffffffffu;
    bool keep = gcur != 0xffffffffu && fabsf(r0.x - wcx) <= whx + bb.x && fabsf(r0.y - wcy) <= why + bb.y;
    if (keep) keep = reaches_box(r0, r1, (float)bx0, (float)bx1, (float)by0, (float)by1, prm.alpha_min);
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      const int slot = __popc(bal & lanemask_lt());
      s_rec[wid][0][slot] = r0;
      s_rec[wid][1][slot] = r1;
    }
    __syncwarp();
    if (in && !cov) {
      const int m = __popc(bal);
      auto alpha_of = [&](int k) {
        const float4 a = s_rec[wid][0][k], c = s_rec[wid][1][k];
        float dx, dy, t1, t2, g;
        return footprint(fpx, fpy, a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w, prm.f_max, dx, dy, t1, t2, g);
      };
      // two independent footprints per step
      for (int k = 0; k < m && !cov; k += 2)
        cov = alpha_of(k) >= prm.alpha_min || (k + 1 < m && alpha_of(k + 1) >= prm.alpha_min);
    }
    __syncwarp();
    r0 = n0;
    r1 = n1;
    bb = nbb;
    gcur = gnext;
    gnext = gafter;
  }
  const int n_in = __syncthreads_count(in);
  const int n_cov = __syncthreads_count(cov);
  const bool keep = !(prm.discard > 0.f) || (float)n_cov >= prm.discard * (float)n_in;
  if (in) mask[((int64_t)f * cam.H + py) * cam.W + px] = (cov && keep) ? 1 : 0;
  if (kMode == kCoverFusedSame) {  // compacted pixel list of the render tile (Z order)
    const bool act = in && cov && keep;
    const unsigned bal = __ballot_sync(0xffffffffu, act);
    if (lane == 0) s_wcnt[wid] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int k = 0; k < wid; ++k) before += s_wcnt[k];
    if (act) w.px_list[((int64_t)tile << (2 * kTileShift)) + before + __popc(bal & lanemask_lt())] = (uint8_t)rpix;
    if (tid == 0) {
      w.tile_npix[tile] = keep ? (uint32_t)n_cov : 0u;
      w.tile_count[tile] = 0u;
    }
  }
  if (kMode != kCoverPlain && tile == 0 && tid == 0) w.counters[kStaged] = 0ull;
}

void launch_l1_loss(const Work &w, int F, int C, int H, int W, const float *color, const float *depth,
                    const float *tcolor, const float *tdepth, const uint8_t *mask, float w_c, float w_d,
                    float *loss_out, float *dL_dcolor, float *dL_ddepth, cudaStream_t s) {
  launch(k_loss_reduce, kLossBlocks, 256, 0, s, w, F, C, H, W, color, depth, tcolor, tdepth, mask, w_c, w_d, loss_out);
  launch(k_loss_grad, kLossBlocks, 256, 0, s, w, F, C, H, W, color, depth, tcolor, tdepth, mask, dL_dcolor, dL_ddepth);
}

void launch_adam(int64_t nu, int C, float *means, float *scales, float *quats, float *opacity, float *colors,
                 const float *g_means, const float *g_scales, const float *g_quats, const float *g_opacity,
                 const float *g_colors, float *m, float *v, const rtg_adam_params &hp, float bc1, float bc2_sqrt,
                 int32_t *step_dev, cudaStream_t s, bool early) {
  if (nu <= 0) return;
  AdamGroups G;
  float *params[5] = {means, scales, quats, opacity, colors};
  const float *grads[5] = {g_means, g_scales, g_quats, g_opacity, g_colors};
  const float lrs[5] = {hp.lr_means, hp.lr_scales, hp.lr_quats, hp.lr_opacity, hp.lr_colors};
  const int64_t width[5] = {3, 3, 4, 1, C};
  G.begin[0] = 0;
  for (int k = 0; k < 5; ++k) {
    G.param[k] = params[k];
    G.grad[k] = grads[k];
    G.lr[k] = lrs[k];
    G.begin[k + 1] = G.begin[k] + nu * width[k];
  }
  G.lr_rest = hp.lr_colors_rest;
  G.width = C;
  G.dc = (hp.colors_dc > 0 && hp.colors_dc < C) ? hp.colors_dc : 0;
  G.quad[0] = 0;
  for (int k = 0; k < 5; ++k) {
    G.quad[k + 1] = G.quad[k] + (nu * width[k] + 3) / 4;
    const uintptr_t a = (uintptr_t)G.param[k] | (uintptr_t)G.grad[k] | (uintptr_t)(m + G.begin[k]) |
                        (uintptr_t)(v + G.begin[k]);
    G.vec[k] = (a & 15u) == 0u ? 1 : 0;
  }
  const int64_t rounds = (G.quad[5] + 256 * kAdamRounds - 1) / (256 * kAdamRounds);
  const unsigned blocks = (unsigned)std::min<int64_t>(rounds, (int64_t)resident_grid((const void *)k_adam, 256));
  launch(k_adam, blocks, 256, 0, s, G, m, v, hp, bc1, bc2_sqrt, step_dev, early ? 1 : 0);
}

void launch_gather(int64_t nu, int C, const int32_t *ids, const float *means, const float *scales,
                   const float *quats, const float *opacity, const float *colors, float *um, float *us, float *uq,
                   float *uo, float *uc, cudaStream_t s) {
  if (nu <= 0) return;
  launch(k_gather, (unsigned)((nu + 255) / 256), 256, 0, s, nu, C, ids, means, scales, quats, opacity, colors, um, us, uq,
                                                        uo, uc);
}

void launch_scatter(int64_t nu, int C, const int32_t *ids, const float *um, const float *us, const float *uq,
                    const float *uo, const float *uc, float *means, float *scales, float *quats, float *opacity,
                    float *colors, cudaStream_t s) {
  if (nu <= 0) return;
  launch(k_scatter, (unsigned)((nu + 255) / 256), 256, 0, s, nu, C, ids, um, us, uq, uo, uc, means, scales, quats,
                                                         opacity, colors);
}

void launch_mask_cover_tiles(const Work &w, const Prm &prm, int64_t N, int F, int T, int C, uint8_t *mask,
                             int mode, cudaStream_t s) {
  if (mode == kCoverFusedSame)
    launch(k_mask_cover_tiles<kCoverFusedSame>, F * T, kTilePix, 0, s, w, prm, N, T, hot4_of(C), mask);
  else if (mode == kCoverFusedOther)
    launch(k_mask_cover_tiles<kCoverFusedOther>, F * T, kTilePix, 0, s, w, prm, N, T, hot4_of(C), mask);
  else
    launch(k_mask_cover_tiles<kCoverPlain>, F * T, kTilePix, 0, s, w, prm, N, T, hot4_of(C), mask);
}

}  // namespace rtg
