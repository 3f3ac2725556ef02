// Forward compositing (Section 3.1): per 16x16 tile, the masked pixels composite the
// tile's front-to-back list — colour by alpha blending (Eq. 1) with the footprint of
// Eq. 2 and transmission of Eq. 3, stopping before a fragment that would take the
// transmission below t_eps — and take their depth from the first processed fragment
// with f > delta_alpha (the opaque-disc hit), through the ray/disc-plane intersection
// of Eq. 4 and the cases of Eq. 5.  The masked pixels of a tile are compacted onto the
// lowest threads, so warps without pixels skip the compositing loop (only pixels
// covered by unstable Gaussians are rendered, Supplement B).  After the compaction each
// warp works alone on its 32 pixels: it walks the tile's list in batches of 32 records,
// keeps only the records whose support box reaches the warp's pixel box (a conservative
// test, so the result is that of the per-pixel alpha_min test), and stops as soon as all
// its pixels have stopped.
#include "kernels.cuh"
#include "project.cuh"

namespace rtg {

template <int C>
__global__ void __launch_bounds__(kTilePix) k_forward(Work w, Prm prm, int64_t N, int T,
                                                      const uint8_t *__restrict__ mask, float *__restrict__ color,
                                                      float *__restrict__ depth, float *__restrict__ alpha,
                                                      int32_t *__restrict__ index_map,
                                                      const float *__restrict__ tcolor,
                                                      const float *__restrict__ tdepth) {
  constexpr int H4 = (C <= 4) ? 3 : 4;
  constexpr int NW = kTilePix / 32;
  __shared__ float4 s_rec[NW][H4][32];
  __shared__ uint32_t s_j[NW][32];
  __shared__ int s_pix[kTilePix];
  __shared__ int s_wcnt[NW];
  if (w.counters[kSkip] != 0ull) return;
  const int tile = blockIdx.x;
  if (w.tile_npix[tile] == 0u) return;
  const int f = tile / T, lt = tile - f * T;
  const DevCam &cam = w.cams[f];
  const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // compact the masked pixels of the tile onto threads 0..npix-1 (the only block barriers)
  {
    const int px = tx * kTile + (tid & (kTile - 1)), py = ty * kTile + tid / kTile;
    bool act = px < cam.W && py < cam.H;
    if (act && mask != nullptr) act = mask[((int64_t)f * cam.H + py) * cam.W + px] != 0;
    const unsigned bal = __ballot_sync(0xffffffffu, act);
    if (lane == 0) s_wcnt[wid] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int k = 0; k < wid; ++k) before += s_wcnt[k];
    if (act) s_pix[before + __popc(bal & lanemask_lt())] = tid;
    __syncthreads();
  }
  // From here on every warp works alone on its 32 compacted pixels.
  const int npix = (int)w.tile_npix[tile];
  if (wid * 32 >= npix) return;
  const bool has = tid < npix;
  const int my = has ? s_pix[tid] : 0;
  const int px = tx * kTile + (my & (kTile - 1)), py = ty * kTile + my / kTile;
  const float fpx = (float)px, fpy = (float)py;
  // bounding box of the warp's pixels: records whose support box misses it are skipped
  const int bx0 = __reduce_min_sync(0xffffffffu, has ? px : 0x7fffffff);
  const int bx1 = __reduce_max_sync(0xffffffffu, has ? px : -1);
  const int by0 = __reduce_min_sync(0xffffffffu, has ? py : 0x7fffffff);
  const int by1 = __reduce_max_sync(0xffffffffu, has ? py : -1);
  const float wcx = 0.5f * (float)(bx0 + bx1), whx = 0.5f * (float)(bx1 - bx0);
  const float wcy = 0.5f * (float)(by0 + by1), why = 0.5f * (float)(by1 - by0);
  const uint32_t off = w.tile_offset[tile];
  const uint32_t n = w.tile_offset[tile + 1] - off;
  const float4 *__restrict__ rec = w.rec_hot + (int64_t)f * N * H4;
  const float2 *__restrict__ box = w.rec_box + (int64_t)f * N;

  float T_ = 1.f;
  float acc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] = 0.f;
  uint32_t last = 0, nfrag = 0;
  int hit_j = -1;
  bool done = !has;
  // the records of batch b0 are fetched while batch b0 - 32 is composited
  float4 r[H4];
  float2 bb = make_float2(0.f, 0.f);
  bool valid = lane < (int)n;
  if (valid) {
    const uint32_t gid = w.sorted[off + lane];
#pragma unroll
    for (int k = 0; k < H4; ++k) r[k] = rec[(int64_t)gid * H4 + k];
    bb = box[gid];
  }
  for (uint32_t b0 = 0; b0 < n; b0 += 32) {
    if (__all_sync(0xffffffffu, done)) break;
    const uint32_t j = b0 + lane;
    const uint32_t jn = j + 32;
    const bool vnext = jn < n;
    float4 rn[H4];
    float2 bn = make_float2(0.f, 0.f);
    if (vnext) {
      const uint32_t gid = w.sorted[off + jn];
#pragma unroll
      for (int k = 0; k < H4; ++k) rn[k] = rec[(int64_t)gid * H4 + k];
      bn = box[gid];
    }
    // keep the records whose support box reaches the warp's pixel box, in list order
    const bool keep = valid && fabsf(r[0].x - wcx) <= whx + bb.x && fabsf(r[0].y - wcy) <= why + bb.y;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      const int slot = __popc(bal & lanemask_lt());
#pragma unroll
      for (int k = 0; k < H4; ++k) s_rec[wid][k][slot] = r[k];
      s_j[wid][slot] = j;
    }
    __syncwarp();
    if (!done) {
      const int cnt = __popc(bal);
      for (int k = 0; k < cnt; ++k) {
        const float4 r0 = s_rec[wid][0][k], r1 = s_rec[wid][1][k];
        float dx, dy, t1, t2, g;
        const float fa = footprint(fpx, fpy, r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, prm.f_max, dx, dy, t1,
                                   t2, g);
        if (fa < prm.alpha_min) continue;
        const float Tn = T_ * (1.f - fa);
        if (Tn < prm.t_eps) {
          done = true;
          break;
        }
        const float wgt = fa * T_;
        const float4 c0 = s_rec[wid][2][k];
        float cw[8] = {c0.x, c0.y, c0.z, c0.w, 0.f, 0.f, 0.f, 0.f};
        if (H4 == 4) {
          const float4 c1 = s_rec[wid][3 % H4][k];
          cw[4] = c1.x; cw[5] = c1.y; cw[6] = c1.z; cw[7] = c1.w;
        }
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] = fmaf(cw[c], wgt, acc[c]);
        const uint32_t jj = s_j[wid][k];
        if (hit_j < 0 && fa > prm.delta_alpha) hit_j = (int)jj;
        T_ = Tn;
        last = jj + 1;
        ++nfrag;
      }
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < H4; ++k) r[k] = rn[k];
    bb = bn;
    valid = vnext;
  }
  float lc = 0.f, ld = 0.f, nd = 0.f;
  if (has) {
    const int64_t HW = (int64_t)cam.H * cam.W;
    const int64_t pix = (int64_t)f * HW + (int64_t)py * cam.W + px;
#pragma unroll
    for (int c = 0; c < C; ++c) color[((int64_t)f * C + c) * HW + (int64_t)py * cam.W + px] = acc[c];
    alpha[pix] = 1.f - T_;
    int hit_gid = -1;
    float D = -1.f;
    if (hit_j >= 0) {
      hit_gid = (int)w.sorted[off + hit_j];
      const float4 c0 = w.rec_cold[((int64_t)f * N + hit_gid) * 2];
      const float4 c1 = w.rec_cold[((int64_t)f * N + hit_gid) * 2 + 1];
      const float ux = (fpx - cam.cx) / cam.fx, uy = (fpy - cam.cy) / cam.fy;
      const float den = fmaf(c0.x, ux, fmaf(c0.y, uy, c0.z));
      const float nu = sqrtf(fmaf(ux, ux, fmaf(uy, uy, 1.f)));
      D = (fabsf(den) >= prm.cos_max * nu) ? c0.w / den : c1.x;
    }
    depth[pix] = D;
    if (index_map != nullptr) index_map[pix] = hit_gid;
    w.px_T[pix] = T_;
    w.px_last[pix] = last;
    w.px_hit[pix] = hit_gid;
    if (tcolor != nullptr) {  // fused L1 terms of this pixel (Eq. 7)
#pragma unroll
      for (int c = 0; c < C; ++c)
        lc += fabsf(acc[c] - tcolor[((int64_t)f * C + c) * HW + (int64_t)py * cam.W + px]);
      const float td = tdepth[pix];
      if (D != -1.f && td > 0.f) {
        ld = fabsf(D - td);
        nd = 1.f;
      }
    }
  }
  if (tcolor != nullptr) {  // fixed-order per-warp partials, summed by k_loss_finalize
    for (int o = 16; o > 0; o >>= 1) {
      lc += __shfl_xor_sync(0xffffffffu, lc, o);
      ld += __shfl_xor_sync(0xffffffffu, ld, o);
      nd += __shfl_xor_sync(0xffffffffu, nd, o);
    }
    if (lane == 0) {
      float *lp = w.tile_loss + ((int64_t)tile * (kTilePix / 32) + wid) * 4;
      lp[0] = lc;
      lp[1] = ld;
      lp[2] = nd;
    }
  }
  // fragment counter: one atomic per warp
  const unsigned fr = __reduce_add_sync(0xffffffffu, nfrag);
  if (lane == 0 && fr) atomicAdd(w.counters + kFragments, (unsigned long long)fr);
}

void launch_forward(int C, const Work &w, const Prm &prm, int64_t N, int F, int T, const uint8_t *mask, float *color,
                    float *depth, float *alpha, int32_t *index_map, const float *tcolor, const float *tdepth,
                    cudaStream_t s) {
  if (C == 3)
    k_forward<3><<<F * T, kTilePix, 0, s>>>(w, prm, N, T, mask, color, depth, alpha, index_map, tcolor, tdepth);
  else
    k_forward<8><<<F * T, kTilePix, 0, s>>>(w, prm, N, T, mask, color, depth, alpha, index_map, tcolor, tdepth);
}

}  // namespace rtg
