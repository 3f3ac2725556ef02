// Backward pass of the masked render (Section 3.1: the depth is a linear function of the
// Gaussian's position and rotation, so the whole render is differentiable; Section 3.2:
// only the unstable Gaussians are optimised).
//
// k_backward replays each masked pixel's composited fragments back to front, recovering
// the transmission by division (T_j = T_{j+1} / (1 - f_j)) instead of storing it, and
// accumulates, for unstable Gaussians only, the screen-space gradients
//   dC/dc_j = f_j T_j,   dC/df_j = c_j T_j - S_j / (1 - f_j),   S_j = sum_{i>j} c_i f_i T_i
// (no background term), chained through f = min(f_max, alpha 2^-q), q = |U (u - mu)|^2.
// The depth depends on f only through the choice of the hit fragment, so it adds no
// gradient to f; its gradient goes to the hit Gaussian's plane record (d0, n_c) or to
// its centre depth.  Each warp works alone on the forward's 32-pixel groups and skips the
// records the forward's culling tests (support box, footprint ellipse) reject; sums over the
// warp are formed by a halving reduce-scatter and added with vector atomics.  The two
// schedules of the forward (CTA per tile, persistent warps over the item queue) apply.
//
// k_project_backward chains those screen-space gradients to position, linear scale,
// raw quaternion, opacity and colour through Sigma_2D = J W R S^2 R^T W^T J^T + lowpass I,
// the conic inverse, the perspective centre, the plane offset d0 = p_c . n_c and the
// normal n_c = W R e_k.
#include "kernels.cuh"
#include "project.cuh"

namespace rtg {

// Per-warp shared memory of the backward compositing.  The replay runs with one pixel a lane
// (the transmission and the colour behind a fragment are per-pixel recurrences), but the
// gradient rows are sums over pixels for one record: so the replay leaves, for each unstable
// record of the batch it meets with at least one active pixel, the pixel's blend weight f T
// and dL/dalpha in a pending slot, and at the end of the batch (or when the slots are full)
// the warp sums the pending rows with one record a lane, over that record's active pixels
// only (flush_rows).
__host__ __device__ constexpr int bwd_slots(int C, int B) { return (C > 4 && B > 32) ? 16 : 32; }

template <int C, int B>
struct BwdWarpSmem {
  static constexpr int H4 = (C <= 4) ? 3 : 4;
  static constexpr int kSlots = bwd_slots(C, B);
  float4 rec[H4][B];        // the batch's kept records, in list order
  int2 jr[B];               // their list position and unstable rank
  float2 wg[kSlots][33];    // pending record x pixel: (f T, dL/dalpha); rows padded by one
  float2 px[32];            // the group's pixel centres
  float dc[C][32];          // the group's dL/dcolour, per channel
};

template <int C, int B>
constexpr size_t bwd_smem_bytes() { return 8 * sizeof(BwdWarpSmem<C, B>); }

// Adds the gradient rows of pending records [0, n) to grad2d, lane s taking slot s: staged
// record slot_k (a slot of sm.rec) whose active pixels are the bits of slot_m.  With
// G = dL/dalpha of a fragment (zero where the footprint is clamped at f_max, f = alpha 2^-q)
// and t = U d, q = |t|^2:
//   dL/dmu    = 2 alpha ln2 (u11 sum G t1,  u12 sum G t1 + u22 sum G t2)
//   dL/dconic = -alpha ln2 kQScale2 (sum G dx^2, 2 sum G dx dy, sum G dy^2)
//   dL/dalpha = sum G,   dL/dc = sum f T dL/dC,
// each sum over the record's active pixels.  A row takes ceil((6 + C) / 4) vector atomics
// (the depth slots get zeros).
template <int C, int B>
__device__ __forceinline__ void flush_rows(const BwdWarpSmem<C, B> &sm, int n, int slot_k, unsigned slot_m,
                                           float *__restrict__ g2base) {
  constexpr int NV = 6 + C, G2 = (C <= 5) ? 16 : 20;
  const int lane = threadIdx.x & 31;
  if (lane >= n) return;
  const float4 a0 = sm.rec[0][slot_k], a1 = sm.rec[1][slot_k];
  const int rank = sm.jr[slot_k].y;
  float acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.f;
  unsigned m = slot_m;
  while (m) {
    const int p = __ffs(m) - 1;
    m &= m - 1u;
    const float2 w_ = sm.wg[lane][p];
    const float2 pp = sm.px[p];
    const float dx = (pp.x - a0.x) - a0.z, dy = (pp.y - a0.y) - a0.w;
    const float t1 = fmaf(a1.x, dx, a1.y * dy), t2 = a1.z * dy;
    const float G = w_.y, Gx = G * dx;
    acc[0] = fmaf(G, t1, acc[0]);
    acc[1] = fmaf(G, t2, acc[1]);
    acc[2] = fmaf(Gx, dx, acc[2]);
    acc[3] = fmaf(Gx, dy, acc[3]);
    acc[4] = fmaf(G * dy, dy, acc[4]);
    acc[5] += G;
#pragma unroll
    for (int c = 0; c < C; ++c) acc[6 + c] = fmaf(w_.x, sm.dc[c][p], acc[6 + c]);
  }
  const float al = a1.w * kLn2, c2 = 2.f * al, kc = -al * kQScale2;
  float v[4 * ((NV + 3) / 4)];
  v[0] = c2 * a1.x * acc[0];
  v[1] = c2 * fmaf(a1.y, acc[0], a1.z * acc[1]);
  v[2] = kc * acc[2];
  v[3] = 2.f * kc * acc[3];
  v[4] = kc * acc[4];
#pragma unroll
  for (int q = 5; q < NV; ++q) v[q] = acc[q];
#pragma unroll
  for (int q = NV; q < 4 * ((NV + 3) / 4); ++q) v[q] = 0.f;
  float4 *row = reinterpret_cast<float4 *>(g2base + (int64_t)rank * G2);
#pragma unroll
  for (int q = 0; q < (NV + 3) / 4; ++q) atomicAdd(row + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
}

// A lane's pixel of group `grp` of render tile `tile` (the forward's pixel grouping) and its
// loss gradients, with the group's pixel centres and colour gradients stored in s_px / s_dc
// for the row sums (the depth gradient goes to the hit Gaussian in bwd_depth_grad).
template <int C>
struct BwdPixel {
  bool has;
  int f, px, py;
  float fpx, fpy;
  uint32_t off, last;
  float T_;
  float dC[C];
  float *g2base;
  int hit;     // the pixel's hit Gaussian (-1: none)
  float dLdD;  // the loss gradient of its depth
};

// With `state` (the composited-lane backward of a fused-loss forward) the lane's pixel, T,
// last entry, hit and L1 signs come from the forward's group state in one load; otherwise
// from the tile's pixel list and the per-pixel arrays.
template <int C>
__device__ __forceinline__ void bwd_pixel_prologue(const Work &w, const Prm &prm, int64_t N, int T, int tile, int grp,
                                                   const float *__restrict__ dL_dcolor,
                                                   const float *__restrict__ dL_ddepth, const L1Fused &l1,
                                                   float2 *s_px, float (*s_dc)[32], BwdPixel<C> &o,
                                                   bool state = false) {
  constexpr int G2 = (C <= 5) ? 16 : 20;
  const int lane = threadIdx.x & 31;
  const int f = tile / T, lt = tile - f * T;
  const DevCam &cam = w.cams[f];
  const int tws = cam.tws, ths = cam.ths;
  float T_ = 1.f, dLdD = 0.f;
  uint32_t last = 0;
  int hit = -1;
#pragma unroll
  for (int c = 0; c < C; ++c) o.dC[c] = 0.f;
  if (state) {
    // the tile's list offset (the unit's first list read needs it) is loaded with the group
    // state, not after the shared-memory writes below
    const uint32_t toff = w.tile_offset[tile];
    const int64_t gslot = (((int64_t)tile << (tws + ths - 5)) + grp) * 32 + lane;
    const uint4 st = w.gstate[gslot];
    const uint32_t sg = w.gsign[gslot];
    const bool has = st.x != 0xffffffffu;
    const int px = has ? (int)(st.x & 0xffffu) : 0, py = has ? (int)(st.x >> 16) : 0;
    if (has) {
      T_ = __uint_as_float(st.y);
      last = st.z;
      hit = (int)st.w;
      const float sc = w.loss_scal[4], sd = w.loss_scal[5];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const uint32_t code = (sg >> (2 * c)) & 3u;
        o.dC[c] = code == 1u ? sc : (code == 2u ? -sc : 0.f);
      }
      const uint32_t code = (sg >> (2 * C)) & 3u;
      dLdD = code == 1u ? sd : (code == 2u ? -sd : 0.f);
    }
    s_px[lane] = make_float2((float)px, (float)py);
#pragma unroll
    for (int c = 0; c < C; ++c) s_dc[c][lane] = o.dC[c];
    o.has = has;
    o.f = f;
    o.px = px;
    o.py = py;
    o.fpx = (float)px;
    o.fpy = (float)py;
    o.off = toff;
    o.last = last;
    o.T_ = T_;
    o.g2base = w.grad2d + (int64_t)f * N * G2;
    o.hit = hit;
    o.dLdD = dLdD;
    return;
  }
  const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
  const int q = grp * 32 + lane;
  const bool has = q < (int)w.tile_npix[tile];
  const int my = has ? (int)w.px_list[((int64_t)tile << (tws + ths)) + q] : 0;
  const int px = (tx << tws) + (my & ((1 << tws) - 1)), py = (ty << ths) + (my >> tws);
  const float fpx = (float)px, fpy = (float)py;
  const int64_t HW = (int64_t)cam.H * cam.W;
  const int64_t pix = (int64_t)f * HW + (int64_t)py * cam.W + px;
  if (has) {
    T_ = w.px_T[pix];
    last = w.px_last[pix];
    hit = w.px_hit[pix];
    if (l1.tcolor != nullptr) {  // gradient of the fused L1 loss, formed here (sign(0) = 0)
      const float sc = w.loss_scal[4], sd = w.loss_scal[5];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int64_t oc = ((int64_t)f * C + c) * HW + (int64_t)py * cam.W + px;
        const float d = l1.color[oc] - l1.tcolor[oc];
        o.dC[c] = d > 0.f ? sc : (d < 0.f ? -sc : 0.f);
      }
      const float Dh = l1.depth[pix], td = l1.tdepth[pix];
      const float d = Dh - td;
      dLdD = (Dh != -1.f && td > 0.f) ? (d > 0.f ? sd : (d < 0.f ? -sd : 0.f)) : 0.f;
    } else {
#pragma unroll
      for (int c = 0; c < C; ++c) o.dC[c] = dL_dcolor[((int64_t)f * C + c) * HW + (int64_t)py * cam.W + px];
      dLdD = dL_ddepth[pix];
    }
  }
  float *__restrict__ g2base = w.grad2d + (int64_t)f * N * G2;
  s_px[lane] = make_float2(fpx, fpy);
#pragma unroll
  for (int c = 0; c < C; ++c) s_dc[c][lane] = o.dC[c];

  o.has = has;
  o.f = f;
  o.px = px;
  o.py = py;
  o.fpx = fpx;
  o.fpy = fpy;
  o.off = w.tile_offset[tile];
  o.last = last;
  o.T_ = T_;
  o.g2base = g2base;
  o.hit = hit;
  o.dLdD = dLdD;
}

// The depth gradient of a group's pixels to their hit Gaussians' plane records or centre
// depths (Eq. 4/5; the depth depends on f only through the choice of the hit), added by
// each pixel's lane.  Called by the whole warp after its list walk, so the walk's first
// loads are not queued behind this one's.
template <int C>
__device__ __forceinline__ void bwd_depth_grad(const Work &w, const Prm &prm, int64_t N, const BwdPixel<C> &o) {
  constexpr int G2 = (C <= 5) ? 16 : 20;
  const int f = o.f, hit = o.hit;
  const bool has = o.has;
  const float fpx = o.fpx, fpy = o.fpy, dLdD = o.dLdD;
  const DevCam &cam = w.cams[f];
  float *__restrict__ g2base = o.g2base;
  {
    int key = -1;
    float gd0 = 0.f, gn0 = 0.f, gn1 = 0.f, gn2 = 0.f, gz = 0.f;
    if (has && hit >= 0 && dLdD != 0.f) {
      const float4 c0 = w.rec_cold[((int64_t)f * N + hit) * 2];
      const float4 c1 = w.rec_cold[((int64_t)f * N + hit) * 2 + 1];
      const int rk = __float_as_int(c1.y);
      if (rk >= 0) {
        key = rk;
        const float ux = (fpx - cam.cx) / cam.fx, uy = (fpy - cam.cy) / cam.fy;
        const float den = fmaf(c0.x, ux, fmaf(c0.y, uy, c0.z));
        const float nu = sqrtf(fmaf(ux, ux, fmaf(uy, uy, 1.f)));
        if (fabsf(den) >= prm.cos_max * nu) {
          // D = d0 / (n_c . u~): dD/dd0 = 1/den, dD/dn_c = -d0 u~ / den^2
          const float id = 1.f / den;
          gd0 = dLdD * id;
          const float s = -dLdD * c0.w * id * id;
          gn0 = s * ux;
          gn1 = s * uy;
          gn2 = s;
        } else {
          gz = dLdD;
        }
      }
    }
    // each lane adds its own terms (fire-and-forget atomics, no return awaited): a group's
    // pixels mostly hit many distinct Gaussians, and aggregating lanes per Gaussian first
    // (five warp sums per distinct one) cost more than it saved
    if (key >= 0) {
      float *row = g2base + (int64_t)key * G2;
      if (gz != 0.f) {
        atomicAdd(row + g2_z(C), gz);
      } else {
        atomicAdd(row + g2_d0(C), gd0);
        atomicAdd(row + g2_nc(C) + 0, gn0);
        atomicAdd(row + g2_nc(C) + 1, gn1);
        atomicAdd(row + g2_nc(C) + 2, gn2);
      }
    }
  }
}

// Replays the pixels of group `grp` of render tile `tile` (the forward's pixel grouping)
// back to front, walking the tile's list with the forward's culling (no composited-lane
// masks: a forward narrowed to a pixel subset).  Called by a whole warp; sm is the warp's
// own shared memory.
template <int C, int B>
__device__ __forceinline__ void backward_group(const Work &w, const Prm &prm, int64_t N, int T, int tile, int grp,
                                               BwdWarpSmem<C, B> &sm, const float *__restrict__ dL_dcolor,
                                               const float *__restrict__ dL_ddepth, const L1Fused &l1) {
  constexpr int H4 = (C <= 4) ? 3 : 4;
  constexpr int R = B / 32;
  const int lane = threadIdx.x & 31;
  BwdPixel<C> pxs;
  bwd_pixel_prologue<C>(w, prm, N, T, tile, grp, dL_dcolor, dL_ddepth, l1, sm.px, sm.dc, pxs);
  const bool has = pxs.has;
  const int f = pxs.f, px = pxs.px, py = pxs.py;
  const float fpx = pxs.fpx, fpy = pxs.fpy;
  const uint32_t off = pxs.off, last = pxs.last;
  float T_ = pxs.T_;
  float dC[C];
#pragma unroll
  for (int c = 0; c < C; ++c) dC[c] = pxs.dC[c];
  float *__restrict__ g2base = pxs.g2base;

  // bounding box of the warp's pixels (records whose support misses it were skipped by the
  // forward's identical test and contribute nothing here)
  const int bx0 = __reduce_min_sync(0xffffffffu, has ? px : 0x7fffffff);
  const int bx1 = __reduce_max_sync(0xffffffffu, has ? px : -1);
  const int by0 = __reduce_min_sync(0xffffffffu, has ? py : 0x7fffffff);
  const int by1 = __reduce_max_sync(0xffffffffu, has ? py : -1);
  const float wcx = 0.5f * (float)(bx0 + bx1), whx = 0.5f * (float)(bx1 - bx0);
  const float wcy = 0.5f * (float)(by0 + by1), why = 0.5f * (float)(by1 - by0);
  const float wbx0 = (float)bx0, wbx1 = (float)bx1, wby0 = (float)by0, wby1 = (float)by1;
  const uint32_t maxlast = __reduce_max_sync(0xffffffffu, last);
  const float4 *__restrict__ rec = w.rec_hot + (int64_t)f * N * H4;
  const float2 *__restrict__ box = w.rec_box + (int64_t)f * N;
  float S[C];
#pragma unroll
  for (int c = 0; c < C; ++c) S[c] = 0.f;
  constexpr int kSlots = bwd_slots(C, B);
  int nslot = 0;          // pending records of the batch (warp-uniform)
  int slot_k = 0;         // lane s: the staged record of pending slot s
  unsigned slot_m = 0u;   // lane s: its active pixels

  // batches of B records run back to front; the records of the next (earlier) batch are
  // fetched while the current one is replayed
  auto fetch = [&](int b_end_, float4 (&rr)[R][H4], float2 (&bx)[R], int (&rank_)[R], bool (&v_)[R]) {
    const int b_beg_ = max(0, b_end_ - B);
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int jq = b_beg_ + u * 32 + lane;
      v_[u] = jq < b_end_;
      bx[u] = make_float2(0.f, 0.f);
      rank_[u] = -1;
      if (v_[u]) {
        const uint32_t gid = w.sorted[off + jq];
#pragma unroll
        for (int k = 0; k < H4; ++k) rr[u][k] = rec[(int64_t)gid * H4 + k];
        bx[u] = box[gid];
        rank_[u] =
            (H4 == 3) ? __float_as_int(rr[u][2].w) : __float_as_int(w.rec_cold[((int64_t)f * N + gid) * 2 + 1].y);
      }
    }
  };
  // One fragment, back to front: its transmission by division, dL/df from the colour behind
  // it, and for an unstable record a pending slot with (f T, dL/dalpha) per pixel.  A record
  // no pixel of the group composited (outside its support, or past the early stop) is
  // skipped as a whole.
  auto replay = [&](int k, float fa, float g) {
    const int2 jr = sm.jr[k];
    const bool act = has && (uint32_t)jr.x < last && fa >= prm.alpha_min;
    if (!__any_sync(0xffffffffu, act)) return;
    float wgt = 0.f, G = 0.f;
    if (act) {
      const float iom = __fdividef(1.f, 1.f - fa);  // 1 - f >= 1 - f_max: a normal divisor
      T_ = T_ * iom;  // transmission in front of this fragment
      wgt = fa * T_;
      const float4 c0 = sm.rec[2][k];
      float cw[8] = {c0.x, c0.y, c0.z, c0.w, 0.f, 0.f, 0.f, 0.f};
      if (H4 == 4) {
        const float4 c1 = sm.rec[3 % H4][k];
        cw[4] = c1.x; cw[5] = c1.y; cw[6] = c1.z; cw[7] = c1.w;
      }
      float dLdf = 0.f;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        dLdf = fmaf(dC[c], fmaf(cw[c], T_, -S[c] * iom), dLdf);
        S[c] = fmaf(cw[c], wgt, S[c]);
      }
      if (sm.rec[1][k].w * g < prm.f_max) G = dLdf * g;  // unclamped branch of min(f_max, alpha g)
    }
    if (jr.y >= 0) {  // warp-uniform: the record is unstable
      sm.wg[nslot][lane] = make_float2(wgt, G);
      const unsigned am = __ballot_sync(0xffffffffu, act);
      slot_k = lane == nslot ? k : slot_k;
      slot_m = lane == nslot ? am : slot_m;
      if (++nslot == kSlots) {
        __syncwarp();
        flush_rows<C, B>(sm, nslot, slot_k, slot_m, g2base);
        __syncwarp();
        nslot = 0;
      }
    }
  };
  float4 r[R][H4];
  float2 bb[R];
  int rk[R];
  bool valid[R];
  fetch((int)maxlast, r, bb, rk, valid);
  for (int b_end = (int)maxlast; b_end > 0; b_end -= B) {
    const int b_beg = max(0, b_end - B);
    float4 rn[R][H4];
    float2 bn[R];
    int rkn[R];
    bool vnext[R];
    fetch(b_beg, rn, bn, rkn, vnext);
    int cnt = 0;
    __syncwarp();  // the previous batch's staged records are no longer read
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const bool keep = valid[u] && fabsf(r[u][0].x - wcx) <= whx + bb[u].x &&
                        fabsf(r[u][0].y - wcy) <= why + bb[u].y &&
                        reaches_box(r[u][0], r[u][1], wbx0, wbx1, wby0, wby1, prm.alpha_min);
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int slot = cnt + __popc(bal & lanemask_lt());
#pragma unroll
        for (int k = 0; k < H4; ++k) sm.rec[k][slot] = r[u][k];
        sm.jr[slot] = make_int2(b_beg + u * 32 + lane, rk[u]);
      }
      cnt += __popc(bal);
    }
    __syncwarp();
    // records back to front, footprints two at a time (they are independent; the
    // recurrences then take the two fragments in order)
    int k = cnt - 1;
    for (; k >= 1; k -= 2) {
      const float4 a0 = sm.rec[0][k], a1 = sm.rec[1][k], b0 = sm.rec[0][k - 1], b1 = sm.rec[1][k - 1];
      float dxA, dyA, t1A, t2A, gA, dxB, dyB, t1B, t2B, gB;
      const float faA = footprint(fpx, fpy, a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, prm.f_max, dxA, dyA, t1A,
                                  t2A, gA);
      const float faB = footprint(fpx, fpy, b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w, prm.f_max, dxB, dyB, t1B,
                                  t2B, gB);
      replay(k, faA, gA);
      replay(k - 1, faB, gB);
    }
    if (k == 0) {
      const float4 a0 = sm.rec[0][0], a1 = sm.rec[1][0];
      float dxA, dyA, t1A, t2A, gA;
      const float faA = footprint(fpx, fpy, a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, prm.f_max, dxA, dyA, t1A,
                                  t2A, gA);
      replay(0, faA, gA);
    }
    if (nslot > 0) {  // the batch's staging is rewritten next: its pending rows go now
      __syncwarp();
      flush_rows<C, B>(sm, nslot, slot_k, slot_m, g2base);
      nslot = 0;
    }
#pragma unroll
    for (int u = 0; u < R; ++u) {
#pragma unroll
      for (int k2 = 0; k2 < H4; ++k2) r[u][k2] = rn[u][k2];
      bb[u] = bn[u];
      rk[u] = rkn[u];
      valid[u] = vnext[u];
    }
  }
  bwd_depth_grad<C>(w, prm, N, pxs);
  __syncwarp();  // the next group rewrites the warp's pixel arrays
}

// ---- backward with the forward's composited-lane masks
// The forward left, for each entry j of a tile's list and each 32-pixel group g, the mask of
// the lanes that composited entry j, at fmask[(off + j) * groups + g].  The backward then
// walks the list in batches of 32 entries back to front, stages only the entries some lane
// composited, and each lane replays its own fragments only (its bit of each staged mask),
// so no lane steps through fragments it did not composite.  The unstable records' rows are
// then summed over their composited pixels, 32 / nu lanes a record (rounded down to a power
// of two), and added to the 2D gradient rows with one atomic per four values.
template <int C>
struct BwdFlSmem {
  static constexpr int H4 = (C <= 4) ? 3 : 4;
  float4 rec[H4][32];    // records of the batch's composited entries, at their batch position
  int2 jr[32];           // their list position and unstable rank
  uint32_t am[32];       // their composited lanes
  uint8_t us[32];        // batch position -> row slot of an unstable record
  uint8_t uk[32];        // row slot -> batch position
  float2 wg[32][33];     // row slot x pixel: (f T, dL/dalpha); zero where not composited
  float2 px[32];
  float dc[C][32];
};

template <int C>
constexpr size_t bwd_fl_smem_bytes() { return 8 * sizeof(BwdFlSmem<C>); }

// seg >= 0: only segment `seg` of the list (entries [seg kSeg, seg kSeg + kSeg), the last
// segment to the end), each lane starting from the forward's checkpoint at the segment's
// back end; seg < 0: the whole list.
template <int C>
__device__ __forceinline__ void backward_group_fl(const Work &w, const Prm &prm, int64_t N, int T, int tile, int grp,
                                                  int seg, BwdFlSmem<C> &sm, const uint32_t *__restrict__ fmask,
                                                  const float *__restrict__ dL_dcolor,
                                                  const float *__restrict__ dL_ddepth, const L1Fused &l1) {
  constexpr int H4 = (C <= 4) ? 3 : 4;
  constexpr int NV = 6 + C, G2 = (C <= 5) ? 16 : 20;
  const int lane = threadIdx.x & 31;
  BwdPixel<C> pxs;
  bwd_pixel_prologue<C>(w, prm, N, T, tile, grp, dL_dcolor, dL_ddepth, l1, sm.px, sm.dc, pxs, l1.tcolor != nullptr);
  const float fpx = pxs.fpx, fpy = pxs.fpy;
  const uint32_t off = pxs.off;
  const int f = pxs.f;
  float T_ = pxs.T_;
  float dC[C];
#pragma unroll
  for (int c = 0; c < C; ++c) dC[c] = pxs.dC[c];
  float *__restrict__ g2base = pxs.g2base;
  const DevCam &cam = w.cams[f];
  const int ngrp = 1 << (cam.tws + cam.ths - 5);
  const uint32_t maxlast = __reduce_max_sync(0xffffffffu, pxs.last);
  const float4 *__restrict__ rec = w.rec_hot + (int64_t)f * N * H4;
  float S[C];
#pragma unroll
  for (int c = 0; c < C; ++c) S[c] = 0.f;
  // the entries [lo, hi) replayed here
  int lo = 0, hi = (int)maxlast;
  if (seg >= 0) {
    lo = seg * kSeg;
    if (seg < kSegMax - 1) hi = min(hi, lo + kSeg);
    hi = max(hi, lo);
    if (pxs.last > (uint32_t)hi) {
      // the lane composited entries behind the segment: the transmission in front of entry
      // hi and the colour behind it (final colour - colour in front) from the checkpoints
      constexpr int CK4 = (C + 4) / 4;
      const int64_t pix = (int64_t)f * cam.H * cam.W + (int64_t)pxs.py * cam.W + pxs.px;
      const float4 *ck = w.ckpt + ((int64_t)seg * w.px_cap + pix) * CK4;
      const float4 *fin = w.ckpt + ((int64_t)(kSegMax - 1) * w.px_cap + pix) * CK4;
      float vs[4 * CK4], vf[4 * CK4];
#pragma unroll
      for (int k = 0; k < CK4; ++k) {
        const float4 a = ck[k], b = fin[k];
        vs[4 * k] = a.x; vs[4 * k + 1] = a.y; vs[4 * k + 2] = a.z; vs[4 * k + 3] = a.w;
        vf[4 * k] = b.x; vf[4 * k + 1] = b.y; vf[4 * k + 2] = b.z; vf[4 * k + 3] = b.w;
      }
      T_ = vs[0];
#pragma unroll
      for (int c = 0; c < C; ++c) S[c] = vf[1 + c] - vs[1 + c];
    }
  }

  // entry b_end - 32 + lane of the list: its mask and Gaussian id (fetched two batches
  // ahead), then, when some lane composited it, its record and unstable rank (one batch
  // ahead), so each batch's replay covers one load latency instead of a chain of three
  auto fetch_idx = [&](int b_end_, uint32_t &am_, uint32_t &gid_) {
    const int jq = b_end_ - 32 + lane;
    am_ = 0u;
    gid_ = 0u;
    if (jq >= lo) {
      am_ = fmask[(int64_t)(off + (uint32_t)jq) * ngrp + grp];
      gid_ = w.sorted[off + jq];
    }
  };
  auto fetch_rec = [&](uint32_t am_, uint32_t gid_, float4 (&rr)[H4], int &rank_) {
    rank_ = -1;
    if (am_ != 0u) {
#pragma unroll
      for (int k = 0; k < H4; ++k) rr[k] = rec[(int64_t)gid_ * H4 + k];
      rank_ = (H4 == 3) ? __float_as_int(rr[2].w) : __float_as_int(w.rec_cold[((int64_t)f * N + gid_) * 2 + 1].y);
    }
  };
  uint32_t am = 0u, gid = 0u, am1 = 0u, gid1 = 0u, nsteps = 0u;
  float4 r[H4];
  int rk = -1;
  fetch_idx(hi, am, gid);
  if (hi > lo + 32) fetch_idx(hi - 32, am1, gid1);
  fetch_rec(am, gid, r, rk);
  for (int b_end = hi; b_end > lo; b_end -= 32) {
    const uint32_t amn = am1;
    float4 rn[H4];
    int rkn = -1;
    fetch_rec(am1, gid1, rn, rkn);
    uint32_t am2 = 0u, gid2 = 0u;
    if (b_end > lo + 64) fetch_idx(b_end - 64, am2, gid2);
    // stage the composited entries at their batch position (entry b_end - 32 + k at k),
    // numbering the unstable ones in list order; this lane's fragments in the batch are
    // bit k = its bit of entry k's mask, a bit transpose of the lanes' masks.  (The row
    // slots need no clearing: the row sums read slot (u, p) only for pixels p that
    // composited record u, and lane p's replay writes exactly those.)
    const unsigned ubal = __ballot_sync(0xffffffffu, am != 0u && rk >= 0);
    const int nu = __popc(ubal);
    uint32_t mine = bit_transpose32(am, lane);
    if (am != 0u) {
#pragma unroll
      for (int k = 0; k < H4; ++k) sm.rec[k][lane] = r[k];
      sm.jr[lane] = make_int2(b_end - 32 + lane, rk);
      sm.am[lane] = am;
      if (rk >= 0) {
        const int u = __popc(ubal & lanemask_lt());
        sm.us[lane] = (uint8_t)u;
        sm.uk[u] = (uint8_t)lane;
      }
    }
    __syncwarp();
    nsteps += __reduce_max_sync(0xffffffffu, (unsigned)__popc(mine));
    // back to front over this lane's own fragments: the transmission in front of each by
    // division, dL/df from the colour behind it, and for an unstable record (f T, dL/dalpha)
    // a fragment replayed as invalid (past this lane's last one) leaves T and S as they are
    auto replay = [&](int k, float fa, float g, float alpha, bool valid) {
      const float iom = valid ? __fdividef(1.f, 1.f - fa) : 1.f;  // 1 - f >= 1 - f_max: a normal divisor
      T_ = T_ * iom;
      const float wgt = fa * T_;
      const float4 c0 = sm.rec[2][k];
      float cw[8] = {c0.x, c0.y, c0.z, c0.w, 0.f, 0.f, 0.f, 0.f};
      if (H4 == 4) {
        const float4 c1 = sm.rec[3 % H4][k];
        cw[4] = c1.x; cw[5] = c1.y; cw[6] = c1.z; cw[7] = c1.w;
      }
      float dLdf = 0.f;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        dLdf = fmaf(dC[c], fmaf(cw[c], T_, -S[c] * iom), dLdf);
        const float Sn = fmaf(cw[c], wgt, S[c]);
        S[c] = valid ? Sn : S[c];
      }
      if (valid && sm.jr[k].y >= 0) {
        const float G = alpha * g < prm.f_max ? dLdf * g : 0.f;  // unclamped branch of min(f_max, alpha g)
        sm.wg[sm.us[k]][lane] = make_float2(wgt, G);
      }
    };
    // two fragments a round in one block of straight-line code (a missing second one
    // replays as invalid, not branched around), so the compiler overlaps their loads and
    // footprints; the recurrences then take them in order
    while (mine) {
      const int kA = 31 - __clz(mine);
      mine ^= 1u << kA;
      const bool vB = mine != 0u;
      const int kB = vB ? 31 - __clz(mine) : kA;
      mine ^= vB ? (1u << kB) : 0u;
      const float4 a0 = sm.rec[0][kA], a1 = sm.rec[1][kA], b0 = sm.rec[0][kB], b1 = sm.rec[1][kB];
      float dx, dy, t1, t2, gA, gB;
      const float faA = footprint(fpx, fpy, a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, prm.f_max, dx, dy, t1,
                                  t2, gA);
      const float faB = footprint(fpx, fpy, b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w, prm.f_max, dx, dy, t1,
                                  t2, gB);
      replay(kA, faA, gA, a1.w, true);
      replay(kB, faB, gB, b1.w, vB);
    }
    __syncwarp();
    // the rows of the unstable records: L lanes a record (L = 32 / nu rounded down to a
    // power of two), each lane over every L-th pixel of the record's composited ones, the
    // L partial rows then summed across the lanes
    if (nu > 0) {
      const int lg = 5 - (32 - __clz(nu - 1));  // L = 2^lg: nu <= 32 / L
      const int u = lane >> lg, sub = lane & ((1 << lg) - 1);
      // pixels p = sub (mod L)
      const unsigned pat = lg == 0 ? 0xffffffffu : lg == 1 ? 0x55555555u : lg == 2 ? 0x11111111u
                         : lg == 3 ? 0x01010101u : lg == 4 ? 0x00010001u : 0x00000001u;
      float acc[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] = 0.f;
      float4 a1 = make_float4(0.f, 0.f, 0.f, 0.f);
      int rank = 0;
      if (u < nu) {
        const int k = sm.uk[u];
        const float4 a0 = sm.rec[0][k];
        a1 = sm.rec[1][k];
        rank = sm.jr[k].y;
        unsigned m = sm.am[k] & (pat << sub);
        // four pixels an iteration, their loads issued together (a missing one adds zeros)
        while (m) {
          int pq[4];
          bool ok[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            ok[q] = m != 0u;
            pq[q] = ok[q] ? __ffs(m) - 1 : 0;
            m &= m - 1u;
          }
          float2 wq[4], ppq[4];
          float dq[4][C];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            wq[q] = sm.wg[u][pq[q]];
            ppq[q] = sm.px[pq[q]];
#pragma unroll
            for (int c = 0; c < C; ++c) dq[q][c] = sm.dc[c][pq[q]];
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float dx = (ppq[q].x - a0.x) - a0.z, dy = (ppq[q].y - a0.y) - a0.w;
            const float t1 = fmaf(a1.x, dx, a1.y * dy), t2 = a1.z * dy;
            const float G = ok[q] ? wq[q].y : 0.f, wx = ok[q] ? wq[q].x : 0.f, Gx = G * dx;
            acc[0] = fmaf(G, t1, acc[0]);
            acc[1] = fmaf(G, t2, acc[1]);
            acc[2] = fmaf(Gx, dx, acc[2]);
            acc[3] = fmaf(Gx, dy, acc[3]);
            acc[4] = fmaf(G * dy, dy, acc[4]);
            acc[5] += G;
#pragma unroll
            for (int c = 0; c < C; ++c) acc[6 + c] = fmaf(wx, dq[q][c], acc[6 + c]);
          }
        }
      }
      for (int o = (1 << lg) >> 1; o > 0; o >>= 1) {
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
      }
      if (u < nu && sub == 0) {
        const float al = a1.w * kLn2, c2 = 2.f * al, kc = -al * kQScale2;
        float v[4 * ((NV + 3) / 4)];
        v[0] = c2 * a1.x * acc[0];
        v[1] = c2 * fmaf(a1.y, acc[0], a1.z * acc[1]);
        v[2] = kc * acc[2];
        v[3] = 2.f * kc * acc[3];
        v[4] = kc * acc[4];
#pragma unroll
        for (int qv = 5; qv < NV; ++qv) v[qv] = acc[qv];
#pragma unroll
        for (int qv = NV; qv < 4 * ((NV + 3) / 4); ++qv) v[qv] = 0.f;
        float4 *row = reinterpret_cast<float4 *>(g2base + (int64_t)rank * G2);
#pragma unroll
        for (int qv = 0; qv < (NV + 3) / 4; ++qv)
          atomicAdd(row + qv, make_float4(v[4 * qv], v[4 * qv + 1], v[4 * qv + 2], v[4 * qv + 3]));
      }
    }
    __syncwarp();  // the next batch rewrites the staging
    am = amn;
    rk = rkn;
#pragma unroll
    for (int k = 0; k < H4; ++k) r[k] = rn[k];
    am1 = am2;
    gid1 = gid2;
  }
  if (lane == 0 && nsteps) atomicAdd(w.counters + kBwdSteps, (unsigned long long)nsteps);
  if (seg <= 0) bwd_depth_grad<C>(w, prm, N, pxs);
  __syncwarp();  // the next group rewrites the warp's pixel arrays
}

struct BwdIn {
  const float *dL_dcolor, *dL_ddepth;
  L1Fused l1;
  const uint32_t *fmask;  // the forward's composited-lane masks (nullptr: walk with the culling)
  int segments;           // non-zero: the forward queued its segments (persistent schedule)
};

// Schedule 0: CTA `tile` with one warp per 32-pixel group of the tile's pixel list.
template <int C, int B>
__global__ void __launch_bounds__(kMaxTilePix, 2) k_backward(Work w, Prm prm, int64_t N, int T, BwdIn in) {
  grid_dep_wait();
  extern __shared__ float4 bwd_dyn_smem[];
  if (w.counters[kSkip] != 0ull) return;
  const int tile = blockIdx.x, wid = threadIdx.x >> 5;
  if (wid * 32 >= (int)w.tile_npix[tile]) return;
  BwdWarpSmem<C, B> *sm = reinterpret_cast<BwdWarpSmem<C, B> *>(bwd_dyn_smem) + wid;
  backward_group<C, B>(w, prm, N, T, tile, wid, *sm, in.dL_dcolor, in.dL_ddepth, in.l1);
}

// Schedule 1: persistent warps over the forward's item queue (its own counter).
template <int C, int B>
__global__ void __launch_bounds__(256, 2) k_backward_queue(Work w, Prm prm, int64_t N, int T, BwdIn in, int spread) {
  grid_dep_wait();
  extern __shared__ float4 bwd_dyn_smem[];
  if (w.counters[kSkip] != 0ull) return;
  const uint32_t nitems = (uint32_t)w.counters[kItems];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  BwdWarpSmem<C, B> *sm = reinterpret_cast<BwdWarpSmem<C, B> *>(bwd_dyn_smem) + wid;
  const uint32_t nwarps = gridDim.x * 8u;
  uint32_t it = first_item(w, wid, spread);
  while (it < nitems) {
    const uint32_t item = w.items[it];
    backward_group<C, B>(w, prm, N, T, (int)(item >> 3), (int)(item & 7u), *sm, in.dL_dcolor, in.dL_ddepth, in.l1);
    uint32_t nx = 0;
    if (lane == 0) nx = nwarps + (uint32_t)atomicAdd(w.counters + kQBwd, 1ull);
    it = __shfl_sync(0xffffffffu, nx, 0);
  }
}

// Schedule 0 and 1 with the forward's composited-lane masks.
template <int C>
__global__ void __launch_bounds__(kMaxTilePix, 2) k_backward_fl(Work w, Prm prm, int64_t N, int T, BwdIn in) {
  grid_dep_wait();
  extern __shared__ float4 bwd_dyn_smem[];
  if (w.counters[kSkip] != 0ull) return;
  const int tile = blockIdx.x, wid = threadIdx.x >> 5;
  if (wid * 32 >= (int)w.tile_npix[tile]) return;
  BwdFlSmem<C> *sm = reinterpret_cast<BwdFlSmem<C> *>(bwd_dyn_smem) + wid;
  backward_group_fl<C>(w, prm, N, T, tile, wid, -1, *sm, in.fmask, in.dL_dcolor, in.dL_ddepth, in.l1);
}

template <int C>
__global__ void __launch_bounds__(256, 2) k_backward_fl_queue(Work w, Prm prm, int64_t N, int T, BwdIn in,
                                                              int spread) {
  grid_dep_wait();
  extern __shared__ float4 bwd_dyn_smem[];
  if (w.counters[kSkip] != 0ull) return;
  const uint32_t nitems = (uint32_t)w.counters[kItems];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  BwdFlSmem<C> *sm = reinterpret_cast<BwdFlSmem<C> *>(bwd_dyn_smem) + wid;
  const uint32_t nwarps = gridDim.x * 8u;
  uint32_t it = first_item(w, wid, spread);
  while (it < nitems) {
    const uint32_t item = w.items[it];
    backward_group_fl<C>(w, prm, N, T, (int)(item >> 3), (int)(item & 7u), -1, *sm, in.fmask, in.dL_dcolor,
                         in.dL_ddepth, in.l1);
    uint32_t nx = 0;
    if (lane == 0) nx = nwarps + (uint32_t)atomicAdd(w.counters + kQBwd, 1ull);
    it = __shfl_sync(0xffffffffu, nx, 0);
  }
}

// Schedule 1 over the forward's queued segments: the bins in decreasing cost, each a warp's
// (group, segment) unit.  A warp's first unit is static (warp k of CTA b takes unit
// k * grid + b, spreading the costliest units over the SMs); later ones come from the
// shared counter.  kW warps a CTA (8, or 10 for calls of many tiles, see the launcher).
template <int C, int kW>
__global__ void __launch_bounds__(32 * kW, 2) k_backward_seg_queue(Work w, Prm prm, int64_t N, int T, BwdIn in) {
  grid_dep_wait();
  extern __shared__ float4 bwd_dyn_smem[];
  if (w.counters[kSkip] != 0ull) return;
  uint32_t cnt[kSegBins], total = 0;
#pragma unroll
  for (int b = 0; b < kSegBins; ++b) {
    const unsigned long long c = w.counters[kBSeg0 + b * kCounterStride];
    cnt[b] = (uint32_t)(c < (unsigned long long)w.bseg_cap ? c : (unsigned long long)w.bseg_cap);
    total += cnt[b];
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  BwdFlSmem<C> *sm = reinterpret_cast<BwdFlSmem<C> *>(bwd_dyn_smem) + wid;
  const uint32_t nwarps = gridDim.x * (uint32_t)kW;
  uint32_t t = (uint32_t)wid * gridDim.x + blockIdx.x;
  while (t < total) {
    uint32_t r = t;
    int b = 0;
#pragma unroll
    for (int k = 0; k < kSegBins - 1; ++k)
      if (b == k && r >= cnt[k]) {
        r -= cnt[k];
        b = k + 1;
      }
    const uint32_t code = w.bseg[(int64_t)b * w.bseg_cap + r];
    backward_group_fl<C>(w, prm, N, T, (int)(code >> 6), (int)(code & 7u), (int)((code >> 3) & 7u), *sm, in.fmask,
                         in.dL_dcolor, in.dL_ddepth, in.l1);
    uint32_t nx = 0;
    if (lane == 0) nx = nwarps + (uint32_t)atomicAdd(w.counters + kQBwd, 1ull);
    t = __shfl_sync(0xffffffffu, nx, 0);
  }
}

// --------------------------------------------------------------------------- 2D -> 3D
// The persistent backward's queue counter is cleared here (this kernel always follows the
// backward), so a second backward of the same forward finds the queue full again.
template <int C>
__device__ __forceinline__ void project_backward_one(const GaussPtrs &g, const Work &w, const Prm &prm, int F,
                                                     int64_t N, int64_t k, int64_t i, float *__restrict__ g_means,
                                                     float *__restrict__ g_scales, float *__restrict__ g_quats,
                                                     float *__restrict__ g_opacity, float *__restrict__ g_colors,
                                                     int accumulate) {
  constexpr int G2 = (C <= 5) ? 16 : 20;
  GParams P;
  const bool ok = load_params(g, w.rank, i, P);
  float gp[3] = {0, 0, 0}, gs[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0}, ga = 0.f, gc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) gc[c] = 0.f;
  // SH colour: k_sh_backward writes the coefficient gradients and adds the position term
  const bool sh = C == 3 && g.sh_degree > 0;
  if (ok) {
    const float qn = sqrtf(P.q[0] * P.q[0] + P.q[1] * P.q[1] + P.q[2] * P.q[2] + P.q[3] * P.q[3]);
    const float qw = P.q[0] / qn, qx = P.q[1] / qn, qy = P.q[2] / qn, qz = P.q[3] / qn;
    float R[9];
    quat_to_rot(qw, qx, qy, qz, R);
    const int kmin = argmin3(P.s[0], P.s[1], P.s[2]);
    float gR[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int f = 0; f < F; ++f) {
      if (w.ntiles[(int64_t)f * N + i] == 0u) continue;
      const DevCam &cam = w.cams[f];
      const float *row = w.grad2d + ((int64_t)f * N + k) * G2;
      const float gmx = row[kG2Mu], gmy = row[kG2Mu + 1];
      const float gA = row[kG2Conic], gB = row[kG2Conic + 1], gCc = row[kG2Conic + 2];
      ga += row[kG2Alpha];
#pragma unroll
      for (int c = 0; c < C; ++c) gc[c] += row[kG2Col + c];

      const float gd0 = row[g2_d0(C)], gn[3] = {row[g2_nc(C)], row[g2_nc(C) + 1], row[g2_nc(C) + 2]};
      const float gz = row[g2_z(C)];

      // forward quantities (FP32 recomputation)
      const float d[3] = {P.p[0] - cam.t[0], P.p[1] - cam.t[1], P.p[2] - cam.t[2]};
      float pc[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) pc[r] = cam.R[r] * d[0] + cam.R[3 + r] * d[1] + cam.R[6 + r] * d[2];
      float A[9];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) A[3 * r + c] = cam.R[r] * R[c] + cam.R[3 + r] * R[3 + c] + cam.R[6 + r] * R[6 + c];
      const float X = pc[0], Y = pc[1], Z = pc[2], iz = 1.f / Z;
      const float j00 = cam.fx * iz, j02 = -cam.fx * X * iz * iz, j11 = cam.fy * iz, j12 = -cam.fy * Y * iz * iz;
      // Sigma_c = A S^2 A^T (camera-frame covariance); cov = J Sigma_c J^T + lowpass I
      float Sc[9];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float acc = 0.f;
#pragma unroll
          for (int m = 0; m < 3; ++m) acc += A[3 * r + m] * P.s[m] * P.s[m] * A[3 * c + m];
          Sc[3 * r + c] = acc;
        }
      const float J[6] = {j00, 0.f, j02, 0.f, j11, j12};
      float JS[6];  // J Sigma_c (2x3)
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) JS[3 * r + c] = J[3 * r] * Sc[c] + J[3 * r + 1] * Sc[3 + c] + J[3 * r + 2] * Sc[6 + c];
      const float a = JS[0] * J[0] + JS[1] * J[1] + JS[2] * J[2] + prm.lowpass;
      const float b = JS[0] * J[3] + JS[1] * J[4] + JS[2] * J[5];
      const float cc = JS[3] * J[3] + JS[4] * J[4] + JS[5] * J[5] + prm.lowpass;
      const float det = a * cc - b * b;
      const float id2 = 1.f / (det * det);
      // conic (a', b', c') = (c, -b, a) / det  ->  gradient w.r.t. (a, b, c) of Sigma_2D
      const float ga_ = (-cc * cc * gA + b * cc * gB - b * b * gCc) * id2;
      const float gb_ = (2.f * b * cc * gA - (a * cc + b * b) * gB + 2.f * a * b * gCc) * id2;
      const float gc_ = (-b * b * gA + a * b * gB - a * a * gCc) * id2;
      // symmetric matrix gradient G = [[ga, gb/2], [gb/2, gc]]
      const float G[4] = {ga_, 0.5f * gb_, 0.5f * gb_, gc_};
      // dL/dSigma_c = J^T G J ; dL/dJ = 2 G J Sigma_c
      float GJ[6];
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) GJ[3 * r + c] = G[2 * r] * J[c] + G[2 * r + 1] * J[3 + c];
      float gSc[9];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) gSc[3 * r + c] = J[r] * GJ[c] + J[3 + r] * GJ[3 + c];
      float gJ[6];
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          gJ[3 * r + c] = 2.f * (GJ[3 * r] * Sc[c] + GJ[3 * r + 1] * Sc[3 + c] + GJ[3 * r + 2] * Sc[6 + c]);
      // camera-frame centre: J entries, mu, depth terms
      float gpc[3];
      gpc[0] = gJ[2] * (-cam.fx * iz * iz) + gmx * cam.fx * iz;
      gpc[1] = gJ[5] * (-cam.fy * iz * iz) + gmy * cam.fy * iz;
      gpc[2] = gJ[0] * (-cam.fx * iz * iz) + gJ[2] * (2.f * cam.fx * X * iz * iz * iz) +
               gJ[4] * (-cam.fy * iz * iz) + gJ[5] * (2.f * cam.fy * Y * iz * iz * iz) -
               (gmx * cam.fx * X + gmy * cam.fy * Y) * iz * iz + gz;
      float nc[3];  // column kmin of A, by selects (a run-time index would put A in local memory)
#pragma unroll
      for (int r = 0; r < 3; ++r) nc[r] = kmin == 0 ? A[3 * r] : (kmin == 1 ? A[3 * r + 1] : A[3 * r + 2]);
#pragma unroll
      for (int r = 0; r < 3; ++r) gpc[r] += gd0 * nc[r];
      float gnc[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) gnc[r] = gd0 * pc[r] + gn[r];
      // p_c = W (p - t)  ->  dL/dp = W^T dL/dp_c = R_g dL/dp_c
#pragma unroll
      for (int r = 0; r < 3; ++r) gp[r] += cam.R[3 * r] * gpc[0] + cam.R[3 * r + 1] * gpc[1] + cam.R[3 * r + 2] * gpc[2];
      // Sigma_c = W Sigma W^T -> dL/dSigma = W^T gSc W ; Sigma = R S^2 R^T
      float gS[9];  // dL/dSigma (world), = R_g gSc R_g^T
      {
        float tmp[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c)
            tmp[3 * r + c] = cam.R[3 * r] * gSc[c] + cam.R[3 * r + 1] * gSc[3 + c] + cam.R[3 * r + 2] * gSc[6 + c];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c)
            gS[3 * r + c] = tmp[3 * r] * cam.R[3 * c] + tmp[3 * r + 1] * cam.R[3 * c + 1] + tmp[3 * r + 2] * cam.R[3 * c + 2];
      }
      // dL/dR += 2 gS R D (D = diag s^2), dL/ds_m += 2 s_m (R^T gS R)_mm
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float gSR = gS[3 * r] * R[c] + gS[3 * r + 1] * R[3 + c] + gS[3 * r + 2] * R[6 + c];
          gR[3 * r + c] += 2.f * gSR * P.s[c] * P.s[c];
        }
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        float acc = 0.f;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c) acc += R[3 * r + m] * gS[3 * r + c] * R[3 * c + m];
        gs[m] += 2.f * P.s[m] * acc;
      }
      // n_c = W R e_k -> dL/dR[:, k] += W^T dL/dn_c = R_g dL/dn_c
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float v = cam.R[3 * r] * gnc[0] + cam.R[3 * r + 1] * gnc[1] + cam.R[3 * r + 2] * gnc[2];
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (kmin == c) gR[3 * r + c] += v;
      }
    }
    // R(q) -> unit quaternion -> raw quaternion
    const float G01 = gR[1], G02 = gR[2], G10 = gR[3], G12 = gR[5], G20 = gR[6], G21 = gR[7];
    const float G00 = gR[0], G11 = gR[4], G22 = gR[8];
    float gqn[4];
    gqn[0] = 2.f * (-qz * G01 + qy * G02 + qz * G10 - qx * G12 - qy * G20 + qx * G21);
    gqn[1] = 2.f * (qy * G01 + qz * G02 + qy * G10 - 2.f * qx * G11 - qw * G12 + qz * G20 + qw * G21 - 2.f * qx * G22);
    gqn[2] = 2.f * (-2.f * qy * G00 + qx * G01 + qw * G02 + qx * G10 + qz * G12 - qw * G20 + qz * G21 - 2.f * qy * G22);
    gqn[3] = 2.f * (-2.f * qz * G00 - qw * G01 + qx * G02 + qw * G10 - 2.f * qz * G11 + qy * G12 + qx * G20 + qy * G21);
    const float qh[4] = {qw, qx, qy, qz};
    const float dotq = qh[0] * gqn[0] + qh[1] * gqn[1] + qh[2] * gqn[2] + qh[3] * gqn[3];
#pragma unroll
    for (int m = 0; m < 4; ++m) gq[m] = (gqn[m] - qh[m] * dotq) / qn;
  }
  if (accumulate) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      gp[r] += g_means[3 * k + r];
      gs[r] += g_scales[3 * k + r];
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) gq[m] += g_quats[4 * k + m];
    ga += g_opacity[k];
    if (!sh)
#pragma unroll
      for (int c = 0; c < C; ++c) gc[c] += g_colors[(int64_t)C * k + c];
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    g_means[3 * k + r] = gp[r];
    g_scales[3 * k + r] = gs[r];
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) g_quats[4 * k + m] = gq[m];
  g_opacity[k] = ga;
  if (!sh)
#pragma unroll
    for (int c = 0; c < C; ++c) g_colors[(int64_t)C * k + c] = gc[c];
}

// Most unstable Gaussians of a masked step have no row in any frame (outside every frame's
// masked tiles).  So each CTA takes kPbRounds rounds of the grid-stride walk over the compact
// indices at once: a light pass checks them with all their loads in flight, writes the zero
// gradients of those without a row (unless accumulating) and lists the others in shared
// memory; then the CTA's threads run the chain rule over that list only.  The rounds stay
// interleaved over the grid as in a plain grid-stride loop, and when most entries have rows
// (every Gaussian seen in several keyframes) each thread keeps its own, as that loop would.
constexpr int kPbRounds = 4;

template <int C>
__global__ void __launch_bounds__(256) k_project_backward(GaussPtrs g, Work w, Prm prm, int F,
                                                          float *__restrict__ g_means, float *__restrict__ g_scales,
                                                          float *__restrict__ g_quats, float *__restrict__ g_opacity,
                                                          float *__restrict__ g_colors, int accumulate) {
  // The light pass reads only the unstable list and the projection's visibility flags and
  // writes only gradient rows, none of which the compositing backward in front of this
  // kernel touches, so a CTA runs it before waiting on that kernel (its CTAs get an SM as
  // the backward's retire); the chain rule, which reads the 2D rows, comes after the wait.
  __shared__ int s_k[256 * kPbRounds], s_i[256 * kPbRounds];
  __shared__ int s_n;
  const int64_t nu = (int64_t)w.counters[kNumUnstable];
  const int64_t N = g.n;
  const bool sh = C == 3 && g.sh_degree > 0;  // k_sh_backward writes the colour rows
  bool waited = false;
  auto wait_backward = [&]() {
    grid_dep_wait();
    waited = true;
    if (blockIdx.x == 0 && threadIdx.x == 0) w.counters[kQBwd] = 0ull;
  };
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // the grid-stride rounds, grouped evenly: no CTA ends with a short group while others still
  // run a full one
  const int64_t rounds = (nu + stride - 1) / stride;
  const int64_t groups = (rounds + kPbRounds - 1) / kPbRounds;
  const int64_t per = groups > 0 ? (rounds + groups - 1) / groups : 0;
  for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x; r0 < nu; r0 += per * stride) {
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    int64_t ii[kPbRounds];
    unsigned mine = 0u;  // bit u: round u's entry has a row
#pragma unroll
    for (int u = 0; u < kPbRounds; ++u) {
      const int64_t k = r0 + u * stride + threadIdx.x;
      ii[u] = (u < per && k < nu) ? (int64_t)w.ids[k] : -1;
    }
#pragma unroll
    for (int u = 0; u < kPbRounds; ++u) {
      const int64_t k = r0 + u * stride + threadIdx.x;
      if (ii[u] < 0) continue;
      uint32_t any = 0u;  // every frame's flag is loaded (no early exit), so the loads overlap
      for (int f = 0; f < F; ++f) any |= w.ntiles[(int64_t)f * N + ii[u]];
      if (any != 0u) {
        mine |= 1u << u;
        const int slot = atomicAdd(&s_n, 1);
        s_k[slot] = (int)k;
        s_i[slot] = (int)ii[u];
      } else if (!accumulate) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          g_means[3 * k + r] = 0.f;
          g_scales[3 * k + r] = 0.f;
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) g_quats[4 * k + m] = 0.f;
        g_opacity[k] = 0.f;
        if (!sh)
#pragma unroll
          for (int c = 0; c < C; ++c) g_colors[(int64_t)C * k + c] = 0.f;
      }
    }
    __syncthreads();
    if (!waited) wait_backward();
    const int nv = s_n;
    if (2 * nv > (int)per * (int)blockDim.x) {
      // dense (most Gaussians seen): each thread keeps its own entries, as a plain
      // grid-stride loop would, instead of a list whose last pass leaves most lanes idle
#pragma unroll 1
      for (int u = 0; u < kPbRounds; ++u)
        if ((mine >> u) & 1u)
          project_backward_one<C>(g, w, prm, F, N, r0 + u * stride + threadIdx.x, ii[u], g_means, g_scales,
                                  g_quats, g_opacity, g_colors, accumulate);
    } else {
      for (int j = threadIdx.x; j < nv; j += blockDim.x)
        project_backward_one<C>(g, w, prm, F, N, s_k[j], s_i[j], g_means, g_scales, g_quats, g_opacity, g_colors,
                                accumulate);
    }
    __syncthreads();
  }
  if (!waited) wait_backward();  // a CTA without entries still completes only after the backward
}

// SH colour backward (Section 3.1 colour from the view direction): 4 lanes per optimised
// Gaussian, lane t owning SH coefficients 4t .. 4t+3, so a group reads and writes its
// coefficient row (3 (d+1)^2 floats) contiguously.  Per frame that sees the Gaussian, from
// that frame's colour gradient g_c (the screen-space row): dL/dSH[k] += g_c Y_k(r), and the
// position gets (I - r r^T) / |p - t| sum_k (g_c . SH[k]) grad Y_k, added to g_means.
__global__ void __launch_bounds__(256) k_sh_backward(GaussPtrs g, Work w, int F, float *__restrict__ g_means,
                                                     float *__restrict__ g_colors, int accumulate) {
  grid_dep_wait();
  constexpr int G2 = 16;  // C = 3
  constexpr int kChunk = 1024;  // unstable Gaussians a CTA sorts out at once
  __shared__ int s_k[kChunk], s_i[kChunk];
  __shared__ int s_n;
  const int64_t nu = (int64_t)w.counters[kNumUnstable];
  const int64_t N = g.n;
  const int lane = threadIdx.x & 31, t = lane & 3, q0 = lane & ~3;
  const unsigned gmask = 0xfu << q0;  // the 4 lanes of a Gaussian
  const int deg = g.sh_degree, K = (deg + 1) * (deg + 1), width = 3 * K;
  // Most unstable Gaussians have no row in any frame.  A CTA takes a contiguous chunk of
  // compact indices: it zeroes the chunk's coefficient rows with coalesced stores (unless
  // accumulating) and lists the Gaussians with a row, then 4 lanes per listed Gaussian run
  // the chain rule, so the heavy code runs on full warps.
  for (int64_t c0 = (int64_t)blockIdx.x * kChunk; c0 < nu; c0 += (int64_t)gridDim.x * kChunk) {
    const int64_t c1 = c0 + kChunk < nu ? c0 + kChunk : nu;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    for (int64_t kk = c0 + threadIdx.x; kk < c1; kk += blockDim.x) {
      const int64_t i = w.ids[kk];
      uint32_t any = 0u;  // all frames' flags are loaded (no early exit), so the loads overlap
      for (int f = 0; f < F; ++f) any |= w.ntiles[(int64_t)f * N + i];
      if (any != 0u) {
        const int slot = atomicAdd(&s_n, 1);
        s_k[slot] = (int)kk;
        s_i[slot] = (int)i;
      }
    }
    if (!accumulate) {
      float *z = g_colors + (int64_t)width * c0;
      const int64_t nz = (int64_t)width * (c1 - c0);
      for (int64_t e = threadIdx.x; e < nz; e += blockDim.x) z[e] = 0.f;
    }
    __syncthreads();
    const int nv = s_n;
    for (int j0 = 0; j0 < nv; j0 += (int)blockDim.x / 4) {
      const int jv = j0 + ((int)threadIdx.x >> 2);
      if (jv >= nv) continue;  // whole groups of 4 lanes skip together
      const int64_t kk = s_k[jv], i = s_i[jv];
      float *out = g_colors + (int64_t)width * kk;
      const int r = (g.u_means != nullptr) ? w.rank[i] : -1;
      const float *pm = r >= 0 ? g.u_means + 3 * (int64_t)r : g.means + 3 * i;
      const float p[3] = {pm[0], pm[1], pm[2]};
      const float *coef = color_ptr(g, w.rank, i);
      float c[4][3], acc[4][3];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = 4 * t + j;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          c[j][cc] = k < K ? coef[3 * k + cc] : 0.f;
          acc[j][cc] = 0.f;
        }
      }
      float gpos[3] = {0.f, 0.f, 0.f};
      for (int f = 0; f < F; ++f) {
        if (w.ntiles[(int64_t)f * N + i] == 0u) continue;  // the same for the 4 lanes
        const float *row = w.grad2d + ((int64_t)f * N + kk) * G2 + kG2Col;
        const float gc0 = row[0], gc1 = row[1], gc2 = row[2];
        const DevCam &cam = w.cams[f];
        const float dx = p[0] - cam.t[0], dy = p[1] - cam.t[1], dz = p[2] - cam.t[2];
        const float il = 1.f / sqrtf(dx * dx + dy * dy + dz * dz);
        const float x = dx * il, y = dy * il, z = dz * il;
        float Y[kShMax];
        sh_basis(deg, x, y, z, Y);
        float st[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float yk = 0.f;
#pragma unroll
          for (int q = 0; q < kShMax; ++q) yk = q == 4 * t + j ? Y[q] : yk;
          acc[j][0] = fmaf(gc0, yk, acc[j][0]);
          acc[j][1] = fmaf(gc1, yk, acc[j][1]);
          acc[j][2] = fmaf(gc2, yk, acc[j][2]);
          st[j] = gc0 * c[j][0] + gc1 * c[j][1] + gc2 * c[j][2];
        }
        float sk[kShMax];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int j = 0; j < 4; ++j) sk[4 * q + j] = __shfl_sync(gmask, st[j], q0 + q);
        float gx, gy, gz;
        sh_dir_grad(deg, x, y, z, sk, gx, gy, gz);
        const float dot = gx * x + gy * y + gz * z;
        gpos[0] += (gx - dot * x) * il;
        gpos[1] += (gy - dot * y) * il;
        gpos[2] += (gz - dot * z) * il;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = 4 * t + j;
        if (k < K)
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) out[3 * k + cc] = accumulate ? out[3 * k + cc] + acc[j][cc] : acc[j][cc];
      }
      if (t == 0) {
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) g_means[3 * kk + cc] += gpos[cc];
      }
    }
    __syncthreads();
  }
}

template <int C>
static void launch_backward_fl(const Work &w, const Prm &prm, int64_t N, int F, int T, const Tuning &tn,
                               const BwdIn &in, cudaStream_t s) {
  if (tn.schedule == 1 && in.segments) {
    // A call of many tiles (batched keyframes) has many short units against the warps: the
    // kernel is bound by throughput there, and ten warps a CTA (two CTAs an SM still fit at
    // C = 3: at most 88 registers, 221 KB of shared memory) hide more latency (eight
    // batched 1200x680 keyframes: backward 0.750 -> 0.699 ms).  A single frame's step is bound by its longest units
    // instead, and eight warps were as fast or faster there.
    bool ten = false;
    if constexpr (C == 3) ten = (int64_t)F * T > kScanSingleMax;
    if constexpr (C == 3) {
      if (ten) {
        launch(k_backward_seg_queue<C, 10>, tn.num_sms * tn.ctas_per_sm, 320, 10 * sizeof(BwdFlSmem<C>), s, w, prm,
               N, T, in);
        return;
      }
    }
    launch(k_backward_seg_queue<C, 8>, tn.num_sms * tn.ctas_per_sm, 256, bwd_fl_smem_bytes<C>(), s, w, prm, N, T, in);
  } else if (tn.schedule == 1)
    launch(k_backward_fl_queue<C>, tn.num_sms * tn.ctas_per_sm, 256, bwd_fl_smem_bytes<C>(), s, w, prm, N, T, in,
           tn.ctas_per_sm <= 2 ? 1 : 0);
  else
    launch(k_backward_fl<C>, F * T, 1 << (tn.tws + tn.ths),
           (size_t)((1 << (tn.tws + tn.ths)) / 32) * sizeof(BwdFlSmem<C>), s, w, prm, N, T, in);
}

template <int C, int B>
static void launch_backward_cb(const Work &w, const Prm &prm, int64_t N, int F, int T, const Tuning &tn,
                               const BwdIn &in, cudaStream_t s) {
  if (tn.schedule == 1)
    launch(k_backward_queue<C, B>, tn.num_sms * tn.ctas_per_sm, 256, bwd_smem_bytes<C, B>(), s, w, prm, N, T, in,
           tn.ctas_per_sm <= 2 ? 1 : 0);
  else
    launch(k_backward<C, B>, F * T, 1 << (tn.tws + tn.ths),
           (size_t)((1 << (tn.tws + tn.ths)) / 32) * sizeof(BwdWarpSmem<C, B>), s, w, prm, N, T, in);
}

template <int C, int B>
static void set_backward_attributes() {
  cudaFuncSetAttribute(k_backward_queue<C, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)bwd_smem_bytes<C, B>());
  cudaFuncSetAttribute(k_backward<C, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem_bytes<C, B>());
}

void init_backward_attributes() {
  cudaFuncSetAttribute(k_backward_fl_queue<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)bwd_fl_smem_bytes<3>());
  cudaFuncSetAttribute(k_backward_fl<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_fl_smem_bytes<3>());
  cudaFuncSetAttribute(k_backward_fl_queue<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)bwd_fl_smem_bytes<8>());
  cudaFuncSetAttribute(k_backward_fl<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_fl_smem_bytes<8>());
  cudaFuncSetAttribute(k_backward_seg_queue<3, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)bwd_fl_smem_bytes<3>());
  cudaFuncSetAttribute(k_backward_seg_queue<3, 10>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(10 * sizeof(BwdFlSmem<3>)));
  cudaFuncSetAttribute(k_backward_seg_queue<8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)bwd_fl_smem_bytes<8>());
  set_backward_attributes<3, 32>();
  set_backward_attributes<3, 64>();
  set_backward_attributes<8, 32>();
  set_backward_attributes<8, 64>();
}

void launch_backward(int C, const Work &w, const Prm &prm, int64_t N, int F, int T, const Tuning &tn,
                     const float *dL_dcolor, const float *dL_ddepth, const L1Fused &l1, const uint32_t *fmask,
                     bool segments, cudaStream_t s) {
  const BwdIn in{dL_dcolor, dL_ddepth, l1, fmask, (fmask != nullptr && segments) ? 1 : 0};
  if (fmask != nullptr) {
    if (C == 3) launch_backward_fl<3>(w, prm, N, F, T, tn, in, s);
    else launch_backward_fl<8>(w, prm, N, F, T, tn, in, s);
    return;
  }
  if (C == 3) {
    if (tn.batch == 64) launch_backward_cb<3, 64>(w, prm, N, F, T, tn, in, s);
    else launch_backward_cb<3, 32>(w, prm, N, F, T, tn, in, s);
  } else {
    if (tn.batch == 64) launch_backward_cb<8, 64>(w, prm, N, F, T, tn, in, s);
    else launch_backward_cb<8, 32>(w, prm, N, F, T, tn, in, s);
  }
}

void launch_project_backward(const GaussPtrs &g, const Work &w, const Prm &prm, int F, float *g_means,
                             float *g_scales, float *g_quats, float *g_opacity, float *g_colors, bool accumulate,
                             cudaStream_t s) {
  if (g.n <= 0) return;
  const int acc = accumulate ? 1 : 0;
  if (g.C == 3) {
    launch(k_project_backward<3>, resident_grid((const void *)k_project_backward<3>, 256), 256, 0, s,
        g, w, prm, F, g_means, g_scales, g_quats, g_opacity, g_colors, acc);
    if (g.sh_degree > 0)
      launch(k_sh_backward, resident_grid((const void *)k_sh_backward, 256), 256, 0, s, g, w, F, g_means, g_colors, acc);
  }
  else
    launch(k_project_backward<8>, resident_grid((const void *)k_project_backward<8>, 256), 256, 0, s,
        g, w, prm, F, g_means, g_scales, g_quats, g_opacity,
                                                         g_colors, acc);
}

}  // namespace rtg
