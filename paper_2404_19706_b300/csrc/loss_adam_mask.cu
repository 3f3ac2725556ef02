// L1 losses (Section 3.2, Eq. 7/8), Adam on the unstable subset (Supplement C learning
// rates), unstable-subset gather/scatter, and the unstable-pixel mask (Supplement B,
// Eq. S2 plus the 50% tile rule).
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
  if (threadIdx.x == 0) {
    __threadfence();
    double t[4] = {0, 0, 0, 0};
    for (int b = 0; b < (int)gridDim.x; ++b)
      for (int k = 0; k < 4; ++k) t[k] += (double)((volatile float *)w.loss_part)[b * 4 + k];
    const double Lc = t[2] > 0 ? t[0] / (t[2] * C) : 0.0;
    const double Ld = t[3] > 0 ? t[1] / t[3] : 0.0;
    loss_out[0] = (float)(w_c * Lc + w_d * Ld);
    loss_out[1] = (float)Lc;
    loss_out[2] = (float)Ld;
    w.loss_scal[4] = t[2] > 0 ? (float)(w_c / (t[2] * C)) : 0.f;
    w.loss_scal[5] = t[3] > 0 ? (float)(w_d / t[3]) : 0.f;
    *w.loss_done = 0u;
  }
}

__device__ __forceinline__ float signf_(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

__global__ void __launch_bounds__(256) k_loss_grad(Work w, int F, int C, int H, int W,
                                                   const float *__restrict__ color, const float *__restrict__ depth,
                                                   const float *__restrict__ tcolor,
                                                   const float *__restrict__ tdepth,
                                                   const uint8_t *__restrict__ mask, float *__restrict__ dL_dcolor,
                                                   float *__restrict__ dL_ddepth) {
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
  return lr * (m * bc1) / (sqrtf(v) * bc2_sqrt + hp.eps);
}

__global__ void __launch_bounds__(256) k_adam(int64_t nu, int C, float *__restrict__ means, float *__restrict__ scales,
                                              float *__restrict__ quats, float *__restrict__ opacity,
                                              float *__restrict__ colors, const float *__restrict__ g_means,
                                              const float *__restrict__ g_scales, const float *__restrict__ g_quats,
                                              const float *__restrict__ g_opacity, const float *__restrict__ g_colors,
                                              float *__restrict__ m, float *__restrict__ v, rtg_adam_params hp,
                                              float bc1, float bc2_sqrt) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nu) return;
  const int D = 11 + C;
  float *mr = m + k * D, *vr = v + k * D;
  for (int j = 0; j < 3; ++j) {
    float mm = mr[j], vv = vr[j];
    means[3 * k + j] -= adam_delta(g_means[3 * k + j], mm, vv, hp.lr_means, hp, bc1, bc2_sqrt);
    mr[j] = mm;
    vr[j] = vv;
  }
  for (int j = 0; j < 3; ++j) {  // log-space scale: theta = log s, dL/dtheta = s dL/ds
    const float s = scales[3 * k + j];
    float mm = mr[3 + j], vv = vr[3 + j];
    const float step = adam_delta(g_scales[3 * k + j] * s, mm, vv, hp.lr_scales, hp, bc1, bc2_sqrt);
    scales[3 * k + j] = s * expf(-step);
    mr[3 + j] = mm;
    vr[3 + j] = vv;
  }
  for (int j = 0; j < 4; ++j) {
    float mm = mr[6 + j], vv = vr[6 + j];
    quats[4 * k + j] -= adam_delta(g_quats[4 * k + j], mm, vv, hp.lr_quats, hp, bc1, bc2_sqrt);
    mr[6 + j] = mm;
    vr[6 + j] = vv;
  }
  {
    float mm = mr[10], vv = vr[10];
    opacity[k] -= adam_delta(g_opacity[k], mm, vv, hp.lr_opacity, hp, bc1, bc2_sqrt);
    mr[10] = mm;
    vr[10] = vv;
  }
  for (int c = 0; c < C; ++c) {
    float mm = mr[11 + c], vv = vr[11 + c];
    colors[(int64_t)C * k + c] -= adam_delta(g_colors[(int64_t)C * k + c], mm, vv, hp.lr_colors, hp, bc1, bc2_sqrt);
    mr[11 + c] = mm;
    vr[11 + c] = vv;
  }
}

__global__ void k_gather(int64_t nu, int C, const int32_t *__restrict__ ids, const float *__restrict__ means,
                         const float *__restrict__ scales, const float *__restrict__ quats,
                         const float *__restrict__ opacity, const float *__restrict__ colors, float *__restrict__ um,
                         float *__restrict__ us, float *__restrict__ uq, float *__restrict__ uo,
                         float *__restrict__ uc) {
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
// Coverage: a pixel is covered when an unstable Gaussian's footprint reaches alpha_min
// there (T_unstable < 1 in Eq. S2).  The footprint is evaluated with the same
// projection and expression as the forward, over the Gaussian's support box.
__global__ void __launch_bounds__(256) k_mask_cover(GaussPtrs g, Work w, Prm prm, int F, uint8_t *__restrict__ mask) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n || g.unstable[i] == 0) return;
  GParams P;
  bool ok = load_params(g, w.rank, i, P);
  if (!ok) return;
  const float *cp = color_ptr(g, w.rank, i);
  for (int c = 0; c < g.C; ++c) ok = ok && isfinite(cp[c]);
  if (!ok) return;
  const float qn = sqrtf(P.q[0] * P.q[0] + P.q[1] * P.q[1] + P.q[2] * P.q[2] + P.q[3] * P.q[3]);
  float R[9];
  quat_to_rot(P.q[0] / qn, P.q[1] / qn, P.q[2] / qn, P.q[3] / qn, R);
  const int kmin = argmin3(P.s[0], P.s[1], P.s[2]);
  for (int f = 0; f < F; ++f) {
    const DevCam &cam = w.cams[f];
    Projected o;
    if (!project_gaussian(cam, prm, P, R, kmin, o)) continue;
    uint8_t *mf = mask + (int64_t)f * cam.H * cam.W;
    for (int y = o.y0; y <= o.y1; ++y)
      for (int x = o.x0; x <= o.x1; ++x) {
        float dx, dy, t1, t2, gg;
        const float fa = footprint((float)x, (float)y, o.mux.hi, o.muy.hi, o.mux.lo, o.muy.lo, o.u11, o.u12, o.u22,
                                   P.alpha, prm.f_max, dx, dy, t1, t2, gg);
        if (fa >= prm.alpha_min) mf[(int64_t)y * cam.W + x] = 1;
      }
  }
}

// Tile rule (Supplement B): clear every 16x16 tile in which fewer than `discard` of the
// in-image pixels are covered.
__global__ void __launch_bounds__(kTilePix) k_mask_tiles(Work w, Prm prm, int T, uint8_t *__restrict__ mask) {
  const int tile = blockIdx.x;
  const int f = tile / T, lt = tile - f * T;
  const DevCam &cam = w.cams[f];
  const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
  const int px = tx * kTile + (threadIdx.x & (kTile - 1)), py = ty * kTile + threadIdx.x / kTile;
  const bool in = px < cam.W && py < cam.H;
  const int64_t o = ((int64_t)f * cam.H + py) * cam.W + px;
  const bool cov = in && mask[o] != 0;
  const int n_in = __syncthreads_count(in);
  const int n_cov = __syncthreads_count(cov);
  if (prm.discard > 0.f && !((float)n_cov >= prm.discard * (float)n_in) && cov) mask[o] = 0;
}

void launch_l1_loss(const Work &w, int F, int C, int H, int W, const float *color, const float *depth,
                    const float *tcolor, const float *tdepth, const uint8_t *mask, float w_c, float w_d,
                    float *loss_out, float *dL_dcolor, float *dL_ddepth, cudaStream_t s) {
  k_loss_reduce<<<kLossBlocks, 256, 0, s>>>(w, F, C, H, W, color, depth, tcolor, tdepth, mask, w_c, w_d, loss_out);
  k_loss_grad<<<kLossBlocks, 256, 0, s>>>(w, F, C, H, W, color, depth, tcolor, tdepth, mask, dL_dcolor, dL_ddepth);
}

void launch_adam(int64_t nu, int C, float *means, float *scales, float *quats, float *opacity, float *colors,
                 const float *g_means, const float *g_scales, const float *g_quats, const float *g_opacity,
                 const float *g_colors, float *m, float *v, const rtg_adam_params &hp, float bc1, float bc2_sqrt,
                 cudaStream_t s) {
  if (nu <= 0) return;
  k_adam<<<(unsigned)((nu + 255) / 256), 256, 0, s>>>(nu, C, means, scales, quats, opacity, colors, g_means, g_scales,
                                                      g_quats, g_opacity, g_colors, m, v, hp, bc1, bc2_sqrt);
}

void launch_gather(int64_t nu, int C, const int32_t *ids, const float *means, const float *scales,
                   const float *quats, const float *opacity, const float *colors, float *um, float *us, float *uq,
                   float *uo, float *uc, cudaStream_t s) {
  if (nu <= 0) return;
  k_gather<<<(unsigned)((nu + 255) / 256), 256, 0, s>>>(nu, C, ids, means, scales, quats, opacity, colors, um, us, uq,
                                                        uo, uc);
}

void launch_scatter(int64_t nu, int C, const int32_t *ids, const float *um, const float *us, const float *uq,
                    const float *uo, const float *uc, float *means, float *scales, float *quats, float *opacity,
                    float *colors, cudaStream_t s) {
  if (nu <= 0) return;
  k_scatter<<<(unsigned)((nu + 255) / 256), 256, 0, s>>>(nu, C, ids, um, us, uq, uo, uc, means, scales, quats,
                                                         opacity, colors);
}

void launch_unstable_mask(const GaussPtrs &g, const Work &w, const Prm &prm, int F, int T, uint8_t *mask,
                          cudaStream_t s) {
  if (g.n > 0) k_mask_cover<<<(unsigned)((g.n + 255) / 256), 256, 0, s>>>(g, w, prm, F, mask);
  k_mask_tiles<<<F * T, kTilePix, 0, s>>>(w, prm, T, mask);
}

}  // namespace rtg
