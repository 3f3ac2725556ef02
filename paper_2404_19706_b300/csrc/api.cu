// Host side of the C ABI declared in include/rtg.h: context and workspace, argument
// validation, and the kernel launch sequences of each entry point.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "kernels.cuh"

using namespace rtg;

// Open optimisation window: the call that projected the stable Gaussians (rtg_window_begin)
struct Window {
  bool open;
  int F;
  rtg_camera cams[RTG_MAX_FRAMES];
  rtg_render_params prm;
  rtg_gaussians g;
  cudaStream_t stream;
  // sorted per-tile lists of the stable Gaussians over whole frames, for one render grid
  bool lists;
  int lists_tws, lists_ths;
};

struct rtg_ctx {
  rtg_capacity cap;
  int device;
  char *slab;
  size_t bytes;
  Work w;
  uint32_t *status_host;
  uint32_t *winst_host;  // status word of the window's list build (host-mapped)
  uint32_t *winst_dev;
  uint32_t *win_scount, *win_soff;  // [F*T + 1] cached stable list length and offset per tile
  unsigned long long *win_skeys;    // [pairs] cached stable keys, each tile's list sorted
  char err[512];
  // state of the last forward, consumed by the backward
  bool has_fwd;
  Work w_fwd;  // the forward's view of the workspace (rank / ids may be the caller's)
  GaussPtrs g;
  Prm prm;
  int F, W, H, T, C;
  L1Fused l1;  // targets of the last rtg_render_forward_l1 (tcolor == nullptr otherwise)
  cudaStream_t last_stream;
  Tuning tune;      // launch configuration of the next forward
  Tuning tune_fwd;  // ... and of the last one, which its backward follows
  bool bwd_done;    // a backward of the last forward has run (its 2D gradient rows are used)
  bool fmask_ok;    // the last forward's composited-lane masks are intact (no binning since)
  bool narrowed;    // rtg_narrow_pixels reduced the last forward's pixel set
  SelBufs sel;      // scratch of rtg_select_top_error (ticket set per call)
  uint32_t *gauss_bits;  // [max_gaussians] per-frame error bits of rtg_error_count (kept zero)
  Window win;
  // tracing: (start, end) event pairs of the kernels launched while profiling is on
  bool prof;
  struct ProfRec *recs;
  int nrec, caprec;
};

// Kernel kinds reported by the tracing interface (one launcher each).
enum ProfKind {
  kPTileMask, kPUnstableIndex, kPProject, kPScanTiles, kPEmit, kPSortTiles, kPForward, kPL1Loss, kPBackward,
  kPProjectBackward, kPUnstableMask, kPBin, kPSelect, kPNarrow, kPAdd, kPErrorCount, kPCompact, kPDecode,
  kPNumKinds
};
static const char *kProfNames[kPNumKinds] = {"tile_mask", "unstable_index", "project", "scan_tiles",
                                             "emit", "sort_tiles", "forward", "l1_loss",
                                             "backward", "project_backward", "unstable_mask", "bin",
                                             "select_top_error", "narrow_pixels", "add_candidates",
                                             "error_count", "compact_gaussians", "decode"};
constexpr int kProfMaxRecords = 1 << 16;

struct ProfRec {
  cudaEvent_t a, b;
  int kind;
};

namespace {
// Brackets the launches of one kernel kind.  Sets the calling thread's launch-overlap flag
// from the context's tuning (off while tracing, so that each kind's events time its own
// kernels) and restores it afterwards; with tracing on, records the launches between
// construction and destruction under `kind`.
struct ProfScope {
  rtg_ctx *c;
  int idx;
  cudaStream_t s;
  bool prev_overlap;
  ProfScope(rtg_ctx *ctx, int kind, cudaStream_t st) : c(ctx), idx(-1), s(st), prev_overlap(launch_overlap()) {
    set_launch_overlap(c != nullptr && c->tune.overlap != 0 && !c->prof);
    if (c == nullptr || !c->prof) return;
    if (c->nrec == c->caprec) {
      if (c->caprec >= kProfMaxRecords) return;
      const int nc = c->caprec ? 2 * c->caprec : 256;
      ProfRec *r = (ProfRec *)realloc(c->recs, sizeof(ProfRec) * nc);
      if (r == nullptr) return;
      for (int k = c->caprec; k < nc; ++k) {
        cudaEventCreate(&r[k].a);
        cudaEventCreate(&r[k].b);
      }
      c->recs = r;
      c->caprec = nc;
    }
    idx = c->nrec++;
    c->recs[idx].kind = kind;
    cudaEventRecord(c->recs[idx].a, s);
  }
  ~ProfScope() {
    if (idx >= 0) cudaEventRecord(c->recs[idx].b, s);
    set_launch_overlap(prev_overlap);
  }
};
}  // namespace

namespace {

const char *kNoCtx = "rtg: NULL context";

rtg_status fail(rtg_ctx *ctx, rtg_status st, const char *fmt, ...) {
  if (ctx != nullptr) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

rtg_status check_launch(rtg_ctx *ctx, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, RTG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return RTG_OK;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t cams, counters, rank, ids, block_cnt, cand, rec_hot, rec_cold, rec_box, ntiles, tile_npix, tile_count, tile_offset, tile_order,
      tile_cursor, keys, keys_alt, stage, sorted, px_T, px_last, px_hit, grad2d, loss_part, loss_scal, loss_done, tile_loss,
      px_list, items, scand, win_scount, win_soff, win_skeys, scan_part, scan_hist, sel_keys, sel_small, sel_state,
      sel_tie, gauss_bits, loss_acc, ckpt, bseg, gstate, gsign, total;
};

bool capacity_ok(const rtg_capacity *c) {
  return c != nullptr && c->max_gaussians >= 0 && c->max_frames >= 1 && c->max_frames <= RTG_MAX_FRAMES &&
         c->max_width >= 1 && c->max_height >= 1 && (c->max_channels == 3 || c->max_channels == 8) &&
         c->max_pairs >= 1 && c->max_pairs <= 0xffffffffLL && c->max_width <= 32768 && c->max_height <= 32768 &&
         (int64_t)c->max_frames * ((c->max_width + 7) / 8) * ((c->max_height + 7) / 8) <=
             (int64_t)1024 * kScanBlockTiles &&
         (int64_t)c->max_frames * c->max_gaussians < 0xffffffffLL;
}

Layout layout_of(const rtg_capacity *c) {
  const size_t N = (size_t)(c->max_gaussians > 0 ? c->max_gaussians : 1);
  const size_t Fm = (size_t)c->max_frames;
  // tile arrays for the finest tiling (8 x 8); pixel lists, work items and loss partials
  // for the padded image of any tiling (tiles of at most 32 x 16 pixels)
  const size_t tiles = (size_t)((c->max_width + 7) / 8) * (size_t)((c->max_height + 7) / 8);
  const size_t FT = Fm * tiles;
  const size_t padded = Fm * (size_t)(c->max_width + 31) * (size_t)(c->max_height + 15);
  const size_t groups = padded / 32 + 1;
  const size_t P = Fm * (size_t)c->max_width * (size_t)c->max_height;
  const size_t K = (size_t)c->max_pairs;
  const size_t H4 = (size_t)hot4_of(c->max_channels), G2 = (size_t)g2_of(c->max_channels);
  Layout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o += align256(bytes);
    return at;
  };
  L.cams = take(Fm * sizeof(DevCam));
  L.counters = take(kNumCounters * sizeof(unsigned long long));
  L.rank = take(N * 4);
  L.ids = take(N * 4);
  L.block_cnt = take((N / kScanBlock + 2) * 4);
  L.cand = take(Fm * N * 4);
  L.rec_hot = take(Fm * N * H4 * 16);
  L.rec_cold = take(Fm * N * 32);
  L.rec_box = take(Fm * N * 8);
  L.ntiles = take(Fm * N * 4);
  L.tile_npix = take((FT + 1) * 4);
  L.tile_count = take((FT + 1) * 4);
  L.tile_offset = take((FT + 1) * 4);
  L.tile_order = take((FT + 1) * 4);
  L.tile_cursor = take((FT + 1) * 4);
  L.keys = take(K * 8);
  L.keys_alt = take(K * 8);
  L.stage = take(K * 16);
  L.sorted = take(K * 4);
  L.px_T = take(P * 4);
  L.px_last = take(P * 4);
  L.px_hit = take(P * 4);
  L.grad2d = take(Fm * N * G2 * 4);
  L.loss_part = take(kLossBlocks * 4 * 4);
  L.loss_scal = take(8 * 4);
  L.loss_done = take(4);
  L.tile_loss = take(groups * 4 * 4);
  L.px_list = take(padded);
  L.items = take(groups * 4);
  L.scand = take(Fm * N * 4);
  L.win_scount = take((FT + 1) * 4);
  L.win_soff = take((FT + 1) * 4);
  L.win_skeys = take(K * 8);
  const size_t scan_blocks = (FT + kScanBlockTiles - 1) / kScanBlockTiles + 1;
  L.scan_part = take(scan_blocks * 4 * 8);
  L.scan_hist = take(scan_blocks * kQueueClasses * 4);
  const size_t sel_blocks = ((size_t)c->max_width * (size_t)c->max_height + kSelPerBlock - 1) / kSelPerBlock;
  L.sel_keys = take(P * 4);
  L.sel_small = take(sel_scratch_words((int)Fm) * 4);
  L.sel_state = take(Fm * 2 * 4);
  L.sel_tie = take(Fm * sel_blocks * 4);
  L.gauss_bits = take(N * 4);
  L.loss_acc = take(4 * 8);
  L.ckpt = take((size_t)kSegMax * P * (size_t)ck4_of(c->max_channels) * 16);
  L.bseg = take((size_t)kSegBins * groups * kSegMax * 4);
  L.gstate = take(groups * 32 * 16);
  L.gsign = take(groups * 32 * 4);
  L.total = o;
  return L;
}

rtg_status make_frames(rtg_ctx *ctx, const rtg_camera *cams, int F, const rtg_render_params *prm, FrameSet &fs) {
  if (cams == nullptr) return fail(ctx, RTG_ERR_ARG, "cams is NULL");
  if (F < 1 || F > ctx->cap.max_frames) return fail(ctx, RTG_ERR_ARG, "F=%d outside [1, %d]", F, ctx->cap.max_frames);
  memset(&fs, 0, sizeof(fs));
  fs.F = F;
  for (int f = 0; f < F; ++f) {
    const rtg_camera &c = cams[f];
    if (c.width != cams[0].width || c.height != cams[0].height)
      return fail(ctx, RTG_ERR_ARG, "all cameras of a call must share width and height");
    if (c.width < 1 || c.height < 1 || c.width > ctx->cap.max_width || c.height > ctx->cap.max_height)
      return fail(ctx, RTG_ERR_ARG, "image %dx%d outside capacity %dx%d", c.width, c.height, ctx->cap.max_width,
                  ctx->cap.max_height);
    if (!(c.fx > 0.f) || !(c.fy > 0.f) || !isfinite(c.cx) || !isfinite(c.cy))
      return fail(ctx, RTG_ERR_ARG, "camera %d: focal lengths must be positive and finite", f);
    DevCam &d = fs.cam[f];
    d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
    d.W = c.width; d.H = c.height;
    for (int k = 0; k < 9; ++k) d.R[k] = c.R[k];
    for (int k = 0; k < 3; ++k) d.t[k] = c.t[k];
    d.lim_x = prm->guard_band * (0.5f * (float)c.width) / c.fx;
    d.lim_y = prm->guard_band * (0.5f * (float)c.height) / c.fy;
    d.tws = ctx->tune.tws;
    d.ths = ctx->tune.ths;
    d.tiles_x = (c.width + (1 << d.tws) - 1) >> d.tws;
    d.tiles_y = (c.height + (1 << d.ths) - 1) >> d.ths;
    d.mtiles_x = (c.width + kTile - 1) / kTile;
    d.mtiles_y = (c.height + kTile - 1) / kTile;
  }
  return RTG_OK;
}

int log2_exact(int v) {
  for (int k = 0; k < 31; ++k)
    if (v == (1 << k)) return k;
  return -1;
}

// True when a call renders exactly what the open window projected: the same cameras,
// render parameters, Gaussian arrays and precomputed unstable index.
bool window_matches(const rtg_ctx *ctx, const rtg_camera *cams, int F, const rtg_gaussians *g,
                    const rtg_render_params *p) {
  const Window &w = ctx->win;
  if (!w.open || F != w.F || g == nullptr || p == nullptr || cams == nullptr) return false;
  if (memcmp(cams, w.cams, sizeof(rtg_camera) * (size_t)F) != 0) return false;
  if (memcmp(p, &w.prm, sizeof(rtg_render_params)) != 0) return false;
  const rtg_gaussians &a = w.g;
  return g->n == a.n && g->channels == a.channels && g->means == a.means && g->scales == a.scales &&
         g->quats == a.quats && g->opacity == a.opacity && g->colors == a.colors && g->unstable == a.unstable &&
         g->u_means == a.u_means && g->u_scales == a.u_scales && g->u_quats == a.u_quats &&
         g->u_opacity == a.u_opacity && g->u_colors == a.u_colors && g->rank_map == a.rank_map &&
         g->unstable_ids == a.unstable_ids && g->n_unstable == a.n_unstable;
}

// rtg_tuning -> Tuning, or false if the setting is not one the library implements
bool make_tuning(const rtg_tuning *t, int num_sms, Tuning &o) {
  if (t == nullptr) return false;
  const int tws = log2_exact(t->tile_w), ths = log2_exact(t->tile_h);
  if (tws < 3 || tws > 5 || ths < 3 || ths > 4 || tws + ths > 8) return false;
  if (t->batch != 32 && t->batch != 64) return false;
  if (t->schedule != 0 && t->schedule != 1) return false;
  if (t->persist_ctas_per_sm < 1 || t->persist_ctas_per_sm > 8) return false;
  if (t->sort_digit_bits != 4 && t->sort_digit_bits != 8) return false;
  if (t->sort_rank_max < 0 || t->sort_rank_max > kSortCap) return false;
  if (t->overlap != 0 && t->overlap != 1) return false;
  o.tws = tws;
  o.ths = ths;
  o.batch = t->batch;
  o.schedule = t->schedule;
  o.ctas_per_sm = t->persist_ctas_per_sm;
  o.sort_bits = t->sort_digit_bits;
  o.sort_rank_max = t->sort_rank_max;
  o.overlap = t->overlap;
  o.num_sms = num_sms;
  return true;
}

rtg_status make_gauss(rtg_ctx *ctx, const rtg_gaussians *g, GaussPtrs &gp) {
  if (g == nullptr) return fail(ctx, RTG_ERR_ARG, "gaussians is NULL");
  if (g->n < 0 || g->n > ctx->cap.max_gaussians)
    return fail(ctx, RTG_ERR_ARG, "n=%lld outside [0, %lld]", (long long)g->n, (long long)ctx->cap.max_gaussians);
  if (g->n > 0x7fffffffLL) return fail(ctx, RTG_ERR_UNSUPPORTED, "n above 2^31-1");
  if (g->channels != 3 && g->channels != 8) return fail(ctx, RTG_ERR_UNSUPPORTED, "channels must be 3 or 8");
  if (g->channels > ctx->cap.max_channels) return fail(ctx, RTG_ERR_ARG, "channels above capacity");
  if (g->sh_degree < 0 || g->sh_degree > 3) return fail(ctx, RTG_ERR_UNSUPPORTED, "sh_degree must be 0..3");
  if (g->sh_degree > 0 && g->channels != 3) return fail(ctx, RTG_ERR_ARG, "SH colour needs channels = 3");
  if (g->n > 0 && (!g->means || !g->scales || !g->quats || !g->opacity || !g->colors || !g->unstable))
    return fail(ctx, RTG_ERR_ARG, "a Gaussian array is NULL");
  const bool any_u = g->u_means || g->u_scales || g->u_quats || g->u_opacity || g->u_colors;
  const bool all_u = g->u_means && g->u_scales && g->u_quats && g->u_opacity && g->u_colors;
  if (any_u && !all_u) return fail(ctx, RTG_ERR_ARG, "set all five compact u_* arrays or none");
  gp.means = g->means; gp.scales = g->scales; gp.quats = g->quats; gp.opacity = g->opacity; gp.colors = g->colors;
  gp.unstable = g->unstable;
  gp.u_means = g->u_means; gp.u_scales = g->u_scales; gp.u_quats = g->u_quats; gp.u_opacity = g->u_opacity;
  gp.u_colors = g->u_colors;
  gp.n = g->n;
  gp.C = g->channels;
  gp.sh_degree = g->sh_degree;
  gp.col_stride = g->sh_degree > 0 ? 3 * (g->sh_degree + 1) * (g->sh_degree + 1) : g->channels;
  gp.rank_map = g->rank_map;
  gp.unstable_ids = g->unstable_ids;
  gp.n_unstable = g->rank_map ? g->n_unstable : 0;
  if (g->rank_map != nullptr &&
      (g->n_unstable < 0 || g->n_unstable > g->n || (g->n_unstable > 0 && g->unstable_ids == nullptr)))
    return fail(ctx, RTG_ERR_ARG, "precomputed unstable index: bad n_unstable or NULL unstable_ids");
  return RTG_OK;
}

rtg_status make_prm(rtg_ctx *ctx, const rtg_render_params *p, Prm &o) {
  if (p == nullptr) return fail(ctx, RTG_ERR_ARG, "params is NULL");
  if (!(p->alpha_min > 0.f) || !(p->f_max > p->alpha_min) || !(p->f_max < 1.f) || !(p->t_eps > 0.f) ||
      !(p->delta_alpha > 0.f) || !(p->lowpass >= 0.f) || !(p->guard_band > 0.f) || !(p->near_z > 0.f) ||
      !(p->tile_discard_frac >= 0.f) || !(p->tile_discard_frac <= 1.f) || !(p->cos_max_angle >= 0.f))
    return fail(ctx, RTG_ERR_ARG, "render params out of range");
  o.near_z = p->near_z; o.alpha_min = p->alpha_min; o.f_max = p->f_max; o.t_eps = p->t_eps;
  o.delta_alpha = p->delta_alpha; o.cos_max = p->cos_max_angle; o.lowpass = p->lowpass; o.guard = p->guard_band;
  o.discard = p->tile_discard_frac;
  return RTG_OK;
}

// rank[i] / ids[k] of the unstable subset, and its count in counters[kNumUnstable]
rtg_status rank_pass(rtg_ctx *ctx, const uint8_t *unstable, int64_t n, int32_t *rank, int32_t *ids,
                     unsigned long long *nu_counter, int64_t *nu_out, cudaStream_t s) {
  {
    ProfScope ps(ctx, kPUnstableIndex, s);
    launch_rank(unstable, n, ctx->w.block_cnt, rank, ids, nu_counter, nu_out, s);
  }
  return check_launch(ctx, "unstable index");
}

__global__ void k_debug_extract(Work w, int64_t N, int F, int32_t *rect, uint32_t *zbits) {
  grid_dep_wait();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * F) return;
  const float4 c1 = w.rec_cold[i * 2 + 1];
  const bool vis = w.ntiles[i] != 0u;
  const uint32_t lo = __float_as_uint(c1.z), hi = __float_as_uint(c1.w);
  if (rect != nullptr) {  // pixel rect -> render tiles
    const DevCam &cam = w.cams[i / N];
    rect[4 * i + 0] = vis ? (int32_t)(lo & 0xffffu) >> cam.tws : -1;
    rect[4 * i + 1] = vis ? (int32_t)(lo >> 16) >> cam.ths : -1;
    rect[4 * i + 2] = vis ? (int32_t)(hi & 0xffffu) >> cam.tws : -1;
    rect[4 * i + 3] = vis ? (int32_t)(hi >> 16) >> cam.ths : -1;
  }
  if (zbits != nullptr) zbits[i] = vis ? __float_as_uint(c1.x) : 0u;
}

// Sorted per-tile lists of the open window's stable Gaussians over whole frames, for the
// render grid of ctx->tune: bins the cached stable projections into every tile, sorts each
// tile, and keeps the sorted keys with each tile's count and offset.  A window forward then
// bins and sorts only the unstable pairs and merges them with these lists per masked tile.
// Synchronises the window's stream; if the lists do not fit in the pair capacity the window
// keeps only its projections (and every forward bins the stable Gaussians itself).
rtg_status build_window_lists(rtg_ctx *ctx) {
  Window &win = ctx->win;
  win.lists = false;
  ctx->fmask_ok = false;  // the list build bins over the last forward's composited-lane masks
  Prm P;
  rtg_status st = make_prm(ctx, &win.prm, P);
  if (st != RTG_OK) return st;
  FrameSet fs;
  if ((st = make_frames(ctx, win.cams, win.F, &win.prm, fs)) != RTG_OK) return st;
  GaussPtrs gp;
  if ((st = make_gauss(ctx, &win.g, gp)) != RTG_OK) return st;
  const Tuning tn = ctx->tune;
  const DevCam &c0 = fs.cam[0];
  const int T = c0.tiles_x * c0.tiles_y, FT = win.F * T;
  cudaStream_t s = win.stream;
  Work w = ctx->w;
  w.rank = const_cast<int32_t *>(gp.rank_map);
  w.ids = const_cast<int32_t *>(gp.unstable_ids);
  w.status = ctx->winst_dev;  // an overflow here must not mark the caller's status
  *(volatile uint32_t *)ctx->winst_host = 0u;
  launch_tile_mask(fs, w, nullptr, T, c0.tiles_x, tn.tws, tn.ths, true, false, (long long)gp.n_unstable, s);
  launch_bin(w, gp.n, T, ctx->cap.max_pairs, false, true, s);
  launch_scan_tiles(w, FT, ctx->cap.max_pairs, -1, nullptr, s, true);
  launch_sort_tiles(w, FT, tn.sort_bits, tn.sort_rank_max, StableLists{nullptr, nullptr, nullptr}, ctx->win_skeys,
                    tn.tws + tn.ths <= 6, nullptr, s);
  cudaMemcpyAsync(ctx->win_scount, w.tile_count, (size_t)FT * 4, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(ctx->win_soff, w.tile_offset, (size_t)FT * 4, cudaMemcpyDeviceToDevice, s);
  if ((st = check_launch(ctx, "window lists")) != RTG_OK) return st;
  if (cudaStreamSynchronize(s) != cudaSuccess) return check_launch(ctx, "window lists");
  if (*(volatile uint32_t *)ctx->winst_host != 0u) {
    *(volatile uint32_t *)ctx->winst_host = 0u;
    return RTG_OK;  // did not fit: projections only
  }
  win.lists = true;
  win.lists_tws = tn.tws;
  win.lists_ths = tn.ths;
  return RTG_OK;
}

}  // namespace

extern "C" {

rtg_status rtg_workspace_size(const rtg_capacity *cap, size_t *bytes) {
  if (!capacity_ok(cap) || bytes == nullptr) return RTG_ERR_ARG;
  *bytes = layout_of(cap).total;
  return RTG_OK;
}

rtg_status rtg_create(rtg_ctx **out, const rtg_capacity *cap) {
  if (out == nullptr) return RTG_ERR_ARG;
  *out = nullptr;
  if (!capacity_ok(cap)) return RTG_ERR_ARG;
  rtg_ctx *ctx = (rtg_ctx *)calloc(1, sizeof(rtg_ctx));
  if (ctx == nullptr) return RTG_ERR_CUDA;
  ctx->cap = *cap;
  cudaGetDevice(&ctx->device);
  const Layout L = layout_of(cap);
  ctx->bytes = L.total;
  if (cudaMalloc((void **)&ctx->slab, L.total) != cudaSuccess) {
    cudaGetLastError();
    free(ctx);
    return RTG_ERR_CUDA;
  }
  if (cudaHostAlloc((void **)&ctx->status_host, 4, cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(ctx->slab);
    free(ctx);
    return RTG_ERR_CUDA;
  }
  *ctx->status_host = 0u;
  uint32_t *status_dev = nullptr;
  cudaHostGetDevicePointer((void **)&status_dev, ctx->status_host, 0);
  if (cudaHostAlloc((void **)&ctx->winst_host, 4, cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(ctx->status_host);
    cudaFree(ctx->slab);
    free(ctx);
    return RTG_ERR_CUDA;
  }
  *ctx->winst_host = 0u;
  cudaHostGetDevicePointer((void **)&ctx->winst_dev, ctx->winst_host, 0);
  char *b = ctx->slab;
  Work &w = ctx->w;
  w.cams = (DevCam *)(b + L.cams);
  w.counters = (unsigned long long *)(b + L.counters);
  w.rank = (int32_t *)(b + L.rank);
  w.ids = (int32_t *)(b + L.ids);
  w.block_cnt = (int32_t *)(b + L.block_cnt);
  w.cand = (uint32_t *)(b + L.cand);
  w.rec_hot = (float4 *)(b + L.rec_hot);
  w.rec_cold = (float4 *)(b + L.rec_cold);
  w.rec_box = (float2 *)(b + L.rec_box);
  w.ntiles = (uint32_t *)(b + L.ntiles);
  w.tile_npix = (uint32_t *)(b + L.tile_npix);
  w.tile_count = (uint32_t *)(b + L.tile_count);
  w.tile_offset = (uint32_t *)(b + L.tile_offset);
  w.tile_order = (uint32_t *)(b + L.tile_order);
  w.tile_cursor = (uint32_t *)(b + L.tile_cursor);
  w.keys = (unsigned long long *)(b + L.keys);
  w.keys_alt = (unsigned long long *)(b + L.keys_alt);
  w.stage = (uint4 *)(b + L.stage);
  w.sorted = (uint32_t *)(b + L.sorted);
  w.px_T = (float *)(b + L.px_T);
  w.px_last = (uint32_t *)(b + L.px_last);
  w.px_hit = (int32_t *)(b + L.px_hit);
  w.grad2d = (float *)(b + L.grad2d);
  w.loss_part = (float *)(b + L.loss_part);
  w.loss_scal = (float *)(b + L.loss_scal);
  w.loss_done = (uint32_t *)(b + L.loss_done);
  w.loss_acc = (double *)(b + L.loss_acc);
  w.tile_loss = (float *)(b + L.tile_loss);
  w.px_list = (uint8_t *)(b + L.px_list);
  w.items = (uint32_t *)(b + L.items);
  w.scand = (uint32_t *)(b + L.scand);
  ctx->win_scount = (uint32_t *)(b + L.win_scount);
  ctx->win_soff = (uint32_t *)(b + L.win_soff);
  ctx->win_skeys = (unsigned long long *)(b + L.win_skeys);
  w.scan_part = (unsigned long long *)(b + L.scan_part);
  w.scan_hist = (uint32_t *)(b + L.scan_hist);
  w.status = status_dev;
  w.ckpt = (float4 *)(b + L.ckpt);
  w.bseg = (uint32_t *)(b + L.bseg);
  w.gstate = (uint4 *)(b + L.gstate);
  w.gsign = (uint32_t *)(b + L.gsign);
  w.px_cap = (int64_t)ctx->cap.max_frames * ctx->cap.max_width * ctx->cap.max_height;
  {
    const size_t padded = (size_t)ctx->cap.max_frames * (size_t)(ctx->cap.max_width + 31) *
                          (size_t)(ctx->cap.max_height + 15);
    w.bseg_cap = (int64_t)(padded / 32 + 1) * kSegMax;
  }
  ctx->sel.keys = (uint32_t *)(b + L.sel_keys);
  ctx->sel.hist = (uint32_t *)(b + L.sel_small);
  ctx->sel.state = (uint32_t *)(b + L.sel_state);
  ctx->sel.tie = (uint32_t *)(b + L.sel_tie);
  ctx->gauss_bits = (uint32_t *)(b + L.gauss_bits);
  {
    int sms = 148;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || sms < 1) {
      cudaGetLastError();
      sms = 148;
    }
    const rtg_tuning def = {16, 16, 32, 0, 4, 8, 0, 1};
    make_tuning(&def, sms, ctx->tune);
    ctx->tune_fwd = ctx->tune;
  }
  // zero the small bookkeeping region once (counters, loss ticket)
  cudaMemset(ctx->slab + L.counters, 0, kNumCounters * sizeof(unsigned long long));
  ctx->win.open = false;
  cudaMemset(ctx->slab + L.loss_done, 0, 4);
  cudaMemset(ctx->slab + L.loss_acc, 0, 4 * 8);
  cudaMemset(ctx->slab + L.gauss_bits, 0, (size_t)(cap->max_gaussians > 0 ? cap->max_gaussians : 1) * 4);
  init_sort_attributes();
  init_backward_attributes();
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(ctx->status_host);
    cudaFree(ctx->slab);
    free(ctx);
    return RTG_ERR_CUDA;
  }
  snprintf(ctx->err, sizeof(ctx->err), "ok");
  *out = ctx;
  return RTG_OK;
}

rtg_status rtg_destroy(rtg_ctx *ctx) {
  if (ctx == nullptr) return RTG_OK;
  cudaDeviceSynchronize();
  for (int k = 0; k < ctx->caprec; ++k) {
    cudaEventDestroy(ctx->recs[k].a);
    cudaEventDestroy(ctx->recs[k].b);
  }
  free(ctx->recs);
  cudaFree(ctx->slab);
  cudaFreeHost(ctx->status_host);
  cudaFreeHost(ctx->winst_host);
  free(ctx);
  return RTG_OK;
}

rtg_status rtg_set_tuning(rtg_ctx *ctx, const rtg_tuning *t) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  Tuning o;
  if (!make_tuning(t, ctx->tune.num_sms, o)) return fail(ctx, RTG_ERR_ARG, "set_tuning: unsupported setting");
  const bool grid_changed = o.tws != ctx->tune.tws || o.ths != ctx->tune.ths;
  ctx->tune = o;
  // the window's cached stable lists belong to one render grid (and sort arrangement)
  if (ctx->win.open && (grid_changed || !ctx->win.lists)) return build_window_lists(ctx);
  return RTG_OK;
}

rtg_status rtg_get_tuning(rtg_ctx *ctx, rtg_tuning *out) {
  if (ctx == nullptr || out == nullptr) return RTG_ERR_ARG;
  const Tuning &t = ctx->tune;
  out->tile_w = 1 << t.tws;
  out->tile_h = 1 << t.ths;
  out->batch = t.batch;
  out->schedule = t.schedule;
  out->persist_ctas_per_sm = t.ctas_per_sm;
  out->sort_digit_bits = t.sort_bits;
  out->sort_rank_max = t.sort_rank_max;
  out->overlap = t.overlap;
  return RTG_OK;
}

rtg_status rtg_profile_enable(rtg_ctx *ctx, int32_t on) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  ctx->prof = on != 0;
  return RTG_OK;
}

int32_t rtg_profile_kinds(void) { return kPNumKinds; }

const char *rtg_profile_kind_name(int32_t kind) {
  return (kind >= 0 && kind < kPNumKinds) ? kProfNames[kind] : "";
}

rtg_status rtg_profile_read(rtg_ctx *ctx, int64_t *launches, double *total_ms, int32_t n_kinds) {
  if (ctx == nullptr || launches == nullptr || total_ms == nullptr || n_kinds < kPNumKinds)
    return RTG_ERR_ARG;
  for (int k = 0; k < kPNumKinds; ++k) {
    launches[k] = 0;
    total_ms[k] = 0.0;
  }
  for (int r = 0; r < ctx->nrec; ++r) {
    if (cudaEventSynchronize(ctx->recs[r].b) != cudaSuccess) {
      cudaError_t e = cudaGetLastError();
      return fail(ctx, RTG_ERR_CUDA, "profile_read: %s", cudaGetErrorString(e));
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->recs[r].a, ctx->recs[r].b) == cudaSuccess) {
      launches[ctx->recs[r].kind] += 1;
      total_ms[ctx->recs[r].kind] += ms;
    } else {
      cudaGetLastError();
    }
  }
  ctx->nrec = 0;
  return RTG_OK;
}

const char *rtg_last_error(rtg_ctx *ctx) { return ctx == nullptr ? kNoCtx : ctx->err; }

rtg_status rtg_get_status(rtg_ctx *ctx) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  return (rtg_status)(int32_t)(*(volatile uint32_t *)ctx->status_host);
}

rtg_status rtg_reset_status(rtg_ctx *ctx) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  *(volatile uint32_t *)ctx->status_host = 0u;
  return RTG_OK;
}

}  // extern "C"

// A sensor frame decoded into the targets at the start of a forward (rtg_render_forward_l1_frame).
struct FrameIn {
  const uint8_t *rgb;
  const uint16_t *depth;
  float scale;
};

static rtg_status forward_impl(rtg_ctx *ctx, const rtg_camera *cams, int32_t F, const rtg_gaussians *g,
                               const uint8_t *mask, uint8_t *mask_out, const rtg_render_params *prm, float *color,
                               float *depth,
                               float *alpha, int32_t *index_map, const float *tcolor, const float *tdepth, float w_c,
                               float w_d, float *loss_out, void *stream, const FrameIn *frame = nullptr) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  ctx->has_fwd = false;
  Prm P;
  rtg_status st = make_prm(ctx, prm, P);
  if (st != RTG_OK) return st;
  FrameSet fs;
  if ((st = make_frames(ctx, cams, F, prm, fs)) != RTG_OK) return st;
  GaussPtrs gp;
  if ((st = make_gauss(ctx, g, gp)) != RTG_OK) return st;
  if (color == nullptr || depth == nullptr || alpha == nullptr) return fail(ctx, RTG_ERR_ARG, "output is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const Tuning tn = ctx->tune;
  const DevCam &c0 = fs.cam[0];
  const int T = c0.tiles_x * c0.tiles_y;   // render tiles per frame
  const int TM = c0.mtiles_x * c0.mtiles_y;  // 16 x 16 mask-rule tiles per frame
  const int FT = F * T;
  const bool same_grid = tn.tws == kTileShift && tn.ths == kTileShift;
  const int64_t n = gp.n;
  const long long nu_preset = gp.rank_map ? (long long)gp.n_unstable : -1ll;
  // with a matching open window only the unstable Gaussians are projected; any other
  // forward rewrites the records the window keeps, so it closes the window
  const bool win = window_matches(ctx, cams, F, g, prm);
  if (!win) ctx->win.open = false;
  const int cull = win ? kCullUnstable : kCullAll;
  // with the window's sorted stable lists only the unstable pairs are binned and sorted
  const bool lists = win && ctx->win.lists && ctx->win.lists_tws == tn.tws && ctx->win.lists_ths == tn.ths;
  const StableLists sl = lists ? StableLists{ctx->win_skeys, ctx->win_soff, ctx->win_scount}
                               : StableLists{nullptr, nullptr, nullptr};
  Work w = ctx->w;
  if (gp.rank_map != nullptr) {
    w.rank = const_cast<int32_t *>(gp.rank_map);
    w.ids = const_cast<int32_t *>(gp.unstable_ids);
  }
  if (mask_out != nullptr) {
    // unstable mask in the same pass: bin the unstable Gaussians into every 16 x 16 tile,
    // test coverage and the tile rule, then bin everything into the surviving render tiles
    {
      ProfScope ps(ctx, kPTileMask, s);
      launch_tile_mask(fs, w, nullptr, TM, c0.mtiles_x, kTileShift, kTileShift, true, false, nu_preset, s);
    }
    if (gp.rank_map == nullptr)
      if ((st = rank_pass(ctx, gp.unstable, n, w.rank, w.ids, w.counters, nullptr, s)) != RTG_OK) return st;
    {
      ProfScope ps(ctx, kPProject, s);
      launch_project(gp, w, P, F, TM, kProjFused, cull, ctx->cap.max_pairs, s);
    }
    {
      ProfScope ps(ctx, kPUnstableMask, s);  // coverage pass: scan, scatter, cover + tile rule
      launch_scan_tiles(w, F * TM, ctx->cap.max_pairs, -1, nullptr, s, true);
      launch_mask_cover_tiles(w, P, n, F, TM, gp.C, mask_out, same_grid ? kCoverFusedSame : kCoverFusedOther, s);
      if (!same_grid)
        launch_tile_mask(fs, w, mask_out, T, c0.tiles_x, tn.tws, tn.ths, false, true, -1ll, s);
    }
    {
      ProfScope ps(ctx, kPBin, s);
      launch_bin(w, n, T, ctx->cap.max_pairs, true, win && !lists, s);
    }
  } else {
    if (frame != nullptr) {
      ProfScope ps(ctx, kPDecode, s);
      launch_decode_rgbd(F, c0.H, c0.W, frame->rgb, frame->depth, frame->scale, const_cast<float *>(tcolor),
                         const_cast<float *>(tdepth), s);
    }
    {
      ProfScope ps(ctx, kPTileMask, s);
      // after the call's own decode, the pass runs whole before waiting on it
      launch_tile_mask(fs, w, mask, T, c0.tiles_x, tn.tws, tn.ths, true, true, nu_preset, s, frame != nullptr);
    }
    if (gp.rank_map == nullptr)
      if ((st = rank_pass(ctx, gp.unstable, n, w.rank, w.ids, w.counters, nullptr, s)) != RTG_OK) return st;
    {
      ProfScope ps(ctx, kPProject, s);
      launch_project(gp, w, P, F, T, kProjForward, cull, ctx->cap.max_pairs, s);
    }
    if (win && !lists) {
      ProfScope ps(ctx, kPBin, s);
      launch_bin(w, n, T, ctx->cap.max_pairs, false, true, s);
    }
  }
  {
    ProfScope ps(ctx, kPScanTiles, s);  // with the scatter into the buckets (k_emit above 8,192 tiles)
    launch_scan_tiles(w, FT, ctx->cap.max_pairs, tn.schedule == 1 ? tn.gshift() : -1, sl.count, s, true);
  }
  {
    ProfScope ps(ctx, kPSortTiles, s);
    // the persistent schedule's single-CTA scan also lists the tiles with keys, longest first
    launch_sort_tiles(w, FT, tn.sort_bits, tn.sort_rank_max, sl, nullptr, tn.tws + tn.ths <= 6,
                      tn.schedule == 1 && FT <= kScanSingleMax ? w.tile_order : nullptr, s);
  }
  {
    ProfScope ps(ctx, kPForward, s);
    // the persistent schedule finalizes the fused L1 in its last CTA
    const bool fused_loss = tcolor != nullptr && tn.schedule == 1;
    // the composited-lane masks go over the call's bucket keys and staging, free after the sort
    launch_forward(gp.C, w, P, n, F, T, tn, color, depth, alpha, index_map, tcolor, tdepth,
                   fused_loss ? loss_out : nullptr, w_c, w_d, reinterpret_cast<uint32_t *>(w.keys), s);
  }
  if (tcolor != nullptr && tn.schedule != 1) {
    ProfScope ps(ctx, kPL1Loss, s);
    launch_loss_finalize(w, FT, tn.gshift(), gp.C, w_c, w_d, loss_out, s);
  }
  if ((st = check_launch(ctx, "render_forward")) != RTG_OK) return st;
  ctx->has_fwd = true;
  ctx->fmask_ok = true;
  ctx->w_fwd = w;
  ctx->g = gp;
  ctx->prm = P;
  ctx->F = F;
  ctx->W = fs.cam[0].W;
  ctx->H = fs.cam[0].H;
  ctx->T = T;
  ctx->C = gp.C;
  ctx->l1 = L1Fused{tcolor, tdepth, color, depth};
  ctx->tune_fwd = tn;
  ctx->bwd_done = false;
  ctx->narrowed = false;
  ctx->last_stream = s;
  return RTG_OK;
}

// The last forward's composited-lane masks, when its backward can use them: not after the
// forward was narrowed to a pixel subset (its pixel groups changed), nor after a call that
// binned again (the masks share the bucket keys' memory).
static const uint32_t *fwd_masks(const rtg_ctx *ctx) {
  return (ctx->fmask_ok && !ctx->narrowed) ? reinterpret_cast<const uint32_t *>(ctx->w_fwd.keys) : nullptr;
}

// The forward's projection zeroes the 2D gradient rows its backward accumulates into; a
// second backward of the same forward clears them itself first.
static rtg_status prepare_backward(rtg_ctx *ctx, cudaStream_t s) {
  if (ctx->bwd_done) {
    const size_t bytes = (size_t)ctx->F * (size_t)ctx->g.n * (size_t)g2_of(ctx->C) * sizeof(float);
    if (bytes > 0 && cudaMemsetAsync(ctx->w_fwd.grad2d, 0, bytes, s) != cudaSuccess)
      return check_launch(ctx, "clear 2D gradients");
  }
  ctx->bwd_done = true;
  return RTG_OK;
}

extern "C" {

rtg_status rtg_window_begin(rtg_ctx *ctx, const rtg_camera *cams, int32_t F, const rtg_gaussians *g,
                            const rtg_render_params *prm, void *stream) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  ctx->win.open = false;
  Prm P;
  rtg_status st = make_prm(ctx, prm, P);
  if (st != RTG_OK) return st;
  FrameSet fs;
  if ((st = make_frames(ctx, cams, F, prm, fs)) != RTG_OK) return st;
  GaussPtrs gp;
  if ((st = make_gauss(ctx, g, gp)) != RTG_OK) return st;
  if (gp.rank_map == nullptr) return fail(ctx, RTG_ERR_ARG, "window_begin needs the precomputed unstable index");
  cudaStream_t s = (cudaStream_t)stream;
  ctx->has_fwd = false;  // the window pass reuses the forward's workspace
  Work w = ctx->w;
  w.rank = const_cast<int32_t *>(gp.rank_map);
  w.ids = const_cast<int32_t *>(gp.unstable_ids);
  const DevCam &c0 = fs.cam[0];
  {
    ProfScope ps(ctx, kPProject, s);
    launch_tile_mask(fs, w, nullptr, c0.mtiles_x * c0.mtiles_y, c0.mtiles_x, kTileShift, kTileShift, true, false,
                     (long long)gp.n_unstable, s);
    launch_window_reset(w, s);
    launch_project(gp, w, P, F, c0.mtiles_x * c0.mtiles_y, kProjWindow, kCullStable, ctx->cap.max_pairs, s);
  }
  if ((st = check_launch(ctx, "window_begin")) != RTG_OK) return st;
  Window &win = ctx->win;
  win.F = F;
  memcpy(win.cams, cams, sizeof(rtg_camera) * (size_t)F);
  win.prm = *prm;
  win.g = *g;
  win.stream = s;
  win.open = true;
  ctx->last_stream = s;
  st = build_window_lists(ctx);
  if (st != RTG_OK) win.open = false;
  return st;
}

rtg_status rtg_window_end(rtg_ctx *ctx) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  ctx->win.open = false;
  return RTG_OK;
}

int32_t rtg_window_is_open(rtg_ctx *ctx) { return (ctx != nullptr && ctx->win.open) ? 1 : 0; }

rtg_status rtg_render_forward(rtg_ctx *ctx, const rtg_camera *cams, int32_t F, const rtg_gaussians *g,
                              const uint8_t *mask, const rtg_render_params *prm, float *color, float *depth,
                              float *alpha, int32_t *index_map, void *stream) {
  return forward_impl(ctx, cams, F, g, mask, nullptr, prm, color, depth, alpha, index_map, nullptr, nullptr, 0.f,
                      0.f, nullptr, stream);
}

rtg_status rtg_render_forward_l1(rtg_ctx *ctx, const rtg_camera *cams, int32_t F, const rtg_gaussians *g,
                                 const uint8_t *mask, const rtg_render_params *prm, const float *target_color,
                                 const float *target_depth, float w_color, float w_depth, float *color, float *depth,
                                 float *alpha, int32_t *index_map, float *loss_out, void *stream) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  if (target_color == nullptr || target_depth == nullptr || loss_out == nullptr)
    return fail(ctx, RTG_ERR_ARG, "render_forward_l1: NULL target or loss_out");
  return forward_impl(ctx, cams, F, g, mask, nullptr, prm, color, depth, alpha, index_map, target_color,
                      target_depth, w_color, w_depth, loss_out, stream);
}

rtg_status rtg_render_forward_l1_frame(rtg_ctx *ctx, const rtg_camera *cams, int32_t F, const rtg_gaussians *g,
                                       const uint8_t *mask, const rtg_render_params *prm, const uint8_t *rgb,
                                       const uint16_t *depth16, float depth_scale, float *target_color,
                                       float *target_depth, float w_color, float w_depth, float *color, float *depth,
                                       float *alpha, int32_t *index_map, float *loss_out, void *stream) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  if (rgb == nullptr || depth16 == nullptr || !(depth_scale > 0.f) || !isfinite(depth_scale))
    return fail(ctx, RTG_ERR_ARG, "render_forward_l1_frame: NULL frame or bad depth scale");
  if (target_color == nullptr || target_depth == nullptr || loss_out == nullptr)
    return fail(ctx, RTG_ERR_ARG, "render_forward_l1_frame: give the target planes and loss_out");
  if (g == nullptr || g->channels != 3 || g->sh_degree != 0)
    return fail(ctx, RTG_ERR_ARG, "render_forward_l1_frame: the sensor frame has 3 colour channels");
  const FrameIn fr{rgb, depth16, depth_scale};
  return forward_impl(ctx, cams, F, g, mask, nullptr, prm, color, depth, alpha, index_map, target_color, target_depth,
                      w_color, w_depth, loss_out, stream, &fr);
}

rtg_status rtg_render_forward_masked(rtg_ctx *ctx, const rtg_camera *cams, int32_t F, const rtg_gaussians *g,
                                     const rtg_render_params *prm, uint8_t *mask_out, const float *target_color,
                                     const float *target_depth, float w_color, float w_depth, float *color,
                                     float *depth, float *alpha, int32_t *index_map, float *loss_out, void *stream) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  if (mask_out == nullptr) return fail(ctx, RTG_ERR_ARG, "render_forward_masked: mask_out is NULL");
  if ((target_color == nullptr) != (target_depth == nullptr) || (target_color != nullptr && loss_out == nullptr))
    return fail(ctx, RTG_ERR_ARG, "render_forward_masked: give both targets and loss_out, or none");
  return forward_impl(ctx, cams, F, g, nullptr, mask_out, prm, color, depth, alpha, index_map, target_color,
                      target_depth, w_color, w_depth, loss_out, stream);
}

rtg_status rtg_render_backward_l1(rtg_ctx *ctx, float *g_means, float *g_scales, float *g_quats, float *g_opacity,
                                  float *g_colors, int32_t accumulate, void *stream) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  if (!ctx->has_fwd || ctx->l1.tcolor == nullptr)
    return fail(ctx, RTG_ERR_STATE, ctx->has_fwd && ctx->narrowed
                                        ? "render_backward_l1 after narrow_pixels without targets"
                                        : "render_backward_l1 without a preceding render_forward_l1");
  if (!g_means || !g_scales || !g_quats || !g_opacity || !g_colors)
    return fail(ctx, RTG_ERR_ARG, "gradient output is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = ctx->g.n;
  rtg_status st = prepare_backward(ctx, s);
  if (st != RTG_OK) return st;
  {
    ProfScope ps(ctx, kPBackward, s);
    launch_backward(ctx->C, ctx->w_fwd, ctx->prm, n, ctx->F, ctx->T, ctx->tune_fwd, nullptr, nullptr, ctx->l1,
                    fwd_masks(ctx), true, s);
  }
  {
    ProfScope ps(ctx, kPProjectBackward, s);
    launch_project_backward(ctx->g, ctx->w_fwd, ctx->prm, ctx->F, g_means, g_scales, g_quats, g_opacity, g_colors,
                            accumulate != 0, s);
  }
  ctx->last_stream = s;
  return check_launch(ctx, "render_backward_l1");
}

rtg_status rtg_loss_counts(rtg_ctx *ctx, double *counts_out, void *stream) {
  if (ctx == nullptr || counts_out == nullptr) return RTG_ERR_ARG;
  if (!ctx->has_fwd || ctx->l1.tcolor == nullptr)
    return fail(ctx, RTG_ERR_STATE, "loss_counts without a preceding forward with targets");
  cudaStream_t s = (cudaStream_t)stream;
  launch_loss_counts(ctx->w_fwd, ctx->C, counts_out, s);
  ctx->last_stream = s;
  return check_launch(ctx, "loss_counts");
}

rtg_status rtg_set_loss_scales(rtg_ctx *ctx, const double *totals, float w_color, float w_depth, float *loss_out,
                               void *stream) {
  if (ctx == nullptr || totals == nullptr) return RTG_ERR_ARG;
  if (!ctx->has_fwd || ctx->l1.tcolor == nullptr)
    return fail(ctx, RTG_ERR_STATE, "set_loss_scales without a preceding forward with targets");
  if (!(w_color >= 0.f) || !(w_depth >= 0.f)) return fail(ctx, RTG_ERR_ARG, "loss weights must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  launch_set_loss_scales(ctx->w_fwd, ctx->C, totals, w_color, w_depth, loss_out, s);
  ctx->last_stream = s;
  return check_launch(ctx, "set_loss_scales");
}

rtg_status rtg_render_backward(rtg_ctx *ctx, const float *dL_dcolor, const float *dL_ddepth, float *g_means,
                               float *g_scales, float *g_quats, float *g_opacity, float *g_colors,
                               int32_t accumulate, void *stream) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  if (!ctx->has_fwd) return fail(ctx, RTG_ERR_STATE, "render_backward without a preceding render_forward");
  if (dL_dcolor == nullptr || dL_ddepth == nullptr) return fail(ctx, RTG_ERR_ARG, "image gradient is NULL");
  if (!g_means || !g_scales || !g_quats || !g_opacity || !g_colors)
    return fail(ctx, RTG_ERR_ARG, "gradient output is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = ctx->g.n;
  rtg_status st = prepare_backward(ctx, s);
  if (st != RTG_OK) return st;
  {
    ProfScope ps(ctx, kPBackward, s);
    launch_backward(ctx->C, ctx->w_fwd, ctx->prm, n, ctx->F, ctx->T, ctx->tune_fwd, dL_dcolor, dL_ddepth,
                    L1Fused{nullptr, nullptr, nullptr, nullptr}, fwd_masks(ctx), true, s);
  }
  {
    ProfScope ps(ctx, kPProjectBackward, s);
    launch_project_backward(ctx->g, ctx->w_fwd, ctx->prm, ctx->F, g_means, g_scales, g_quats, g_opacity, g_colors,
                            accumulate != 0, s);
  }
  ctx->last_stream = s;
  return check_launch(ctx, "render_backward");
}

rtg_status rtg_l1_loss(rtg_ctx *ctx, int32_t F, int32_t C, int32_t H, int32_t W, const float *color,
                       const float *depth, const float *target_color, const float *target_depth,
                       const uint8_t *mask, float w_color, float w_depth, float *loss_out, float *dL_dcolor,
                       float *dL_ddepth, void *stream) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  if (F < 1 || C < 1 || H < 1 || W < 1) return fail(ctx, RTG_ERR_ARG, "l1_loss: bad sizes");
  if (!color || !depth || !target_color || !target_depth || !loss_out || !dL_dcolor || !dL_ddepth)
    return fail(ctx, RTG_ERR_ARG, "l1_loss: NULL pointer");
  cudaStream_t s = (cudaStream_t)stream;
  ProfScope ps(ctx, kPL1Loss, s);
  launch_l1_loss(ctx->w, F, C, H, W, color, depth, target_color, target_depth, mask, w_color, w_depth, loss_out,
                 dL_dcolor, dL_ddepth, s);
  ctx->last_stream = s;
  return check_launch(ctx, "l1_loss");
}

rtg_status rtg_select_top_error(rtg_ctx *ctx, int32_t F, int32_t C, int32_t H, int32_t W, const float *color,
                                const float *target_color, double frac, uint8_t *mask_out, void *stream) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  if (F < 1 || F > ctx->cap.max_frames || C < 1 || C > 64 || H < 1 || W < 1 || H > ctx->cap.max_height ||
      W > ctx->cap.max_width)
    return fail(ctx, RTG_ERR_ARG, "select_top_error: sizes outside the capacity");
  if (!(frac >= 0.0 && frac <= 1.0)) return fail(ctx, RTG_ERR_ARG, "select_top_error: frac outside [0, 1]");
  if (color == nullptr || target_color == nullptr || mask_out == nullptr)
    return fail(ctx, RTG_ERR_ARG, "select_top_error: NULL pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = (int64_t)H * W;
  const uint32_t k = (uint32_t)floor(frac * (double)n);
  ProfScope ps(ctx, kPSelect, s);
  if (k == 0u || (int64_t)k == n) {  // nothing or everything: no order needed
    if (cudaMemsetAsync(mask_out, k == 0u ? 0 : 1, (size_t)F * (size_t)n, s) != cudaSuccess)
      return check_launch(ctx, "select_top_error");
  } else {
    SelBufs b = ctx->sel;
    b.ticket = b.hist + (size_t)kSelPasses * F * kSelHistStride;
    launch_select_top_error(b, F, C, n, k, color, target_color, mask_out, s);
  }
  ctx->last_stream = s;
  return check_launch(ctx, "select_top_error");
}

rtg_status rtg_narrow_pixels(rtg_ctx *ctx, const uint8_t *mask, const float *target_color,
                             const float *target_depth, float w_color, float w_depth, float *loss_out, void *stream) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  if (!ctx->has_fwd) return fail(ctx, RTG_ERR_STATE, "narrow_pixels without a preceding forward");
  if (mask == nullptr) return fail(ctx, RTG_ERR_ARG, "narrow_pixels: mask is NULL");
  const bool fused = target_color != nullptr;
  if (fused != (target_depth != nullptr) || (fused && loss_out == nullptr))
    return fail(ctx, RTG_ERR_ARG, "narrow_pixels: give both targets and loss_out, or none");
  cudaStream_t s = (cudaStream_t)stream;
  const Tuning &tn = ctx->tune_fwd;
  const NarrowLoss nl{ctx->l1.color, ctx->l1.depth, target_color, target_depth, ctx->C};
  {
    ProfScope ps(ctx, kPNarrow, s);
    launch_narrow_pixels(ctx->w_fwd, ctx->F, ctx->T, tn.tws, tn.ths, mask, tn.schedule == 1 ? tn.gshift() : -1,
                         nl, s);
  }
  if (fused) {
    ProfScope ps(ctx, kPL1Loss, s);
    launch_loss_finalize(ctx->w_fwd, ctx->F * ctx->T, tn.gshift(), ctx->C, w_color, w_depth, loss_out, s);
  }
  // the backward_l1 of these pixels needs their loss; a fused loss of the forward covered others
  ctx->l1.tcolor = fused ? target_color : nullptr;
  ctx->l1.tdepth = fused ? target_depth : nullptr;
  ctx->narrowed = true;
  ctx->last_stream = s;
  return check_launch(ctx, "narrow_pixels");
}

rtg_status rtg_add_candidates(rtg_ctx *ctx, const rtg_camera *cams, int32_t F, int32_t C, const float *render_color,
                              const float *render_alpha, const float *render_depth, const int32_t *index_map,
                              const float *color, const float *depth, const uint8_t *unstable, int64_t n_gaussians,
                              const rtg_add_params *p, int64_t capacity, int64_t *count_out, int32_t *pixel_out,
                              uint8_t *kind_out, float *position_out, float *color_out, float *opacity_out,
                              void *stream) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  if (cams == nullptr || p == nullptr || count_out == nullptr)
    return fail(ctx, RTG_ERR_ARG, "add_candidates: NULL cameras, params or count_out");
  if (F < 1 || F > ctx->cap.max_frames || C < 1 || C > 64)
    return fail(ctx, RTG_ERR_ARG, "add_candidates: F or C out of range");
  const int W = cams[0].width, H = cams[0].height;
  for (int f = 0; f < F; ++f) {
    if (cams[f].width != W || cams[f].height != H)
      return fail(ctx, RTG_ERR_ARG, "add_candidates: all cameras must share width and height");
    if (!(cams[f].fx > 0.f) || !(cams[f].fy > 0.f))
      return fail(ctx, RTG_ERR_ARG, "add_candidates: focal lengths must be positive");
  }
  if (W < 1 || H < 1 || W > ctx->cap.max_width || H > ctx->cap.max_height)
    return fail(ctx, RTG_ERR_ARG, "add_candidates: image outside the capacity");
  if (!render_color || !render_alpha || !render_depth || !index_map || !color || !depth)
    return fail(ctx, RTG_ERR_ARG, "add_candidates: NULL image");
  if (n_gaussians < 0 || (n_gaussians > 0 && unstable == nullptr))
    return fail(ctx, RTG_ERR_ARG, "add_candidates: bad Gaussian count or NULL flags");
  if (capacity < 0 || (capacity > 0 && (!pixel_out || !kind_out || !position_out || !color_out || !opacity_out)))
    return fail(ctx, RTG_ERR_ARG, "add_candidates: bad capacity or NULL output");
  if (!(p->sample_rate >= 0.f && p->sample_rate <= 1.f))
    return fail(ctx, RTG_ERR_ARG, "add_candidates: sample_rate outside [0, 1]");
  AddArgs a;
  a.C = C; a.H = H; a.W = W; a.n = n_gaussians;
  a.rcolor = render_color; a.ralpha = render_alpha; a.rdepth = render_depth; a.index = index_map;
  a.color = color; a.depth = depth; a.unstable = unstable;
  a.dT = p->delta_T; a.dd = p->delta_d;
  a.thr_c = (float)C * p->delta_c;  // float32 product, as the mean test's threshold
  a.op_opaque = p->opacity_opaque; a.op_transparent = p->opacity_transparent;
  a.seed = p->seed;
  a.t24 = (uint32_t)floor((double)p->sample_rate * 16777216.0);
  a.capacity = capacity;
  a.count_out = (long long *)count_out;
  a.pix_out = pixel_out; a.kind_out = kind_out; a.pos_out = position_out; a.col_out = color_out;
  a.op_out = opacity_out;
  a.cnt = ctx->sel.tie;
  a.kinds = reinterpret_cast<uint8_t *>(ctx->sel.keys);  // F*H*W bytes of its F*H*W words
  AddFrames fr;
  memset(&fr, 0, sizeof(fr));
  for (int f = 0; f < F; ++f) {
    AddCam &c = fr.cam[f];
    c.fx = cams[f].fx; c.fy = cams[f].fy; c.cx = cams[f].cx; c.cy = cams[f].cy;
    for (int k = 0; k < 9; ++k) c.R[k] = cams[f].R[k];
    for (int k = 0; k < 3; ++k) c.t[k] = cams[f].t[k];
  }
  cudaStream_t s = (cudaStream_t)stream;
  {
    ProfScope ps(ctx, kPAdd, s);
    launch_add_candidates(a, fr, F, s);
  }
  ctx->last_stream = s;
  return check_launch(ctx, "add_candidates");
}

rtg_status rtg_transparent_reg(rtg_ctx *ctx, int64_t nu, const float *u_means, const float *u_scales,
                               const float *u_quats, const float *u_opacity, const float *means0,
                               const float *scales0, const float *quats0, float w_reg, float alpha_split,
                               float *g_means, float *g_scales, float *g_quats, float *loss_out, void *stream) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  if (nu < 0 || !(w_reg >= 0.f) || loss_out == nullptr) return fail(ctx, RTG_ERR_ARG, "transparent_reg: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  if (nu == 0) {
    if (cudaMemsetAsync(loss_out, 0, sizeof(float), s) != cudaSuccess) return check_launch(ctx, "transparent_reg");
    return RTG_OK;
  }
  if (!u_means || !u_scales || !u_quats || !u_opacity || !means0 || !scales0 || !quats0 || !g_means || !g_scales ||
      !g_quats)
    return fail(ctx, RTG_ERR_ARG, "transparent_reg: NULL array");
  RegArgs a{nu, u_means, u_scales, u_quats, u_opacity, means0, scales0, quats0, w_reg, alpha_split, g_means,
            g_scales, g_quats, ctx->w.loss_part, ctx->w.loss_done, ctx->w.loss_scal + 6};
  {
    ProfScope ps(ctx, kPL1Loss, s);
    launch_transparent_reg(a, loss_out, s);
  }
  ctx->last_stream = s;
  return check_launch(ctx, "transparent_reg");
}

rtg_status rtg_confidence_update(int64_t nu, int32_t C, const int32_t *ids, const float *g_colors, int32_t *eta,
                                 void *stream) {
  if (nu < 0 || C < 1 || C > 64) return RTG_ERR_ARG;
  if (nu == 0) return RTG_OK;
  if (ids == nullptr || g_colors == nullptr || eta == nullptr) return RTG_ERR_ARG;
  launch_confidence(nu, C, ids, g_colors, eta, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? RTG_OK : RTG_ERR_CUDA;
}

rtg_status rtg_fuse_window(int64_t nu, int32_t C, const int32_t *ids, const int32_t *eta_start,
                           const int32_t *eta_now, const float *u_means, const float *u_scales, const float *u_quats,
                           const float *u_opacity, const float *u_colors, float *means, float *scales, float *quats,
                           float *opacity, float *colors, void *stream) {
  if (nu < 0 || C < 1 || C > 64) return RTG_ERR_ARG;
  if (nu == 0) return RTG_OK;
  if (!ids || !eta_start || !eta_now || !u_means || !u_scales || !u_quats || !u_opacity || !u_colors || !means ||
      !scales || !quats || !opacity || !colors)
    return RTG_ERR_ARG;
  const FuseArrays a{means, scales, quats, opacity, colors, u_means, u_scales, u_quats, u_opacity, u_colors};
  launch_fuse(nu, C, ids, eta_start, eta_now, a, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? RTG_OK : RTG_ERR_CUDA;
}

rtg_status rtg_error_count(rtg_ctx *ctx, int32_t F, int32_t C, int32_t H, int32_t W, const float *render_color,
                           const float *render_depth, const int32_t *index_map, const float *color, const float *depth,
                           const uint8_t *unstable, int64_t n, const rtg_state_params *p, int32_t *err, void *stream) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  if (F < 1 || F > 32 || C < 1 || C > 64 || H < 1 || W < 1 || p == nullptr)
    return fail(ctx, RTG_ERR_ARG, "error_count: bad sizes or params");
  if (n < 0 || n > ctx->cap.max_gaussians) return fail(ctx, RTG_ERR_ARG, "error_count: n outside the capacity");
  if (!render_color || !render_depth || !index_map || !color || !depth || (n > 0 && (!unstable || !err)))
    return fail(ctx, RTG_ERR_ARG, "error_count: NULL pointer");
  if (n == 0) return RTG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  {
    ProfScope ps(ctx, kPErrorCount, s);
    launch_error_count(F, C, (int64_t)H * W, render_color, render_depth, index_map, color, depth, unstable, n,
                       (float)C * p->delta_c, p->delta_d, ctx->gauss_bits, err, s);
  }
  ctx->last_stream = s;
  return check_launch(ctx, "error_count");
}

rtg_status rtg_update_states(int64_t n, int32_t frame, const int32_t *t0, const rtg_state_params *p,
                             uint8_t *unstable, int32_t *eta, int32_t *err, uint8_t *remove, void *stream) {
  if (n < 0 || p == nullptr) return RTG_ERR_ARG;
  if (n == 0) return RTG_OK;
  if (!t0 || !unstable || !eta || !err || !remove) return RTG_ERR_ARG;
  launch_update_states(n, frame, t0, *p, unstable, eta, err, remove, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? RTG_OK : RTG_ERR_CUDA;
}

rtg_status rtg_compact_gaussians(rtg_ctx *ctx, int64_t n, int32_t C, const uint8_t *remove, const rtg_map_arrays *in,
                                 const rtg_map_arrays *out, int64_t *count_out, void *stream) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  if (n < 0 || n > ctx->cap.max_gaussians || C < 1 || C > 64 || !remove || !in || !out || !count_out)
    return fail(ctx, RTG_ERR_ARG, "compact_gaussians: bad arguments");
  const rtg_map_arrays *m[2] = {in, out};
  for (const rtg_map_arrays *a : m)
    if (!a->means || !a->scales || !a->quats || !a->opacity || !a->colors || !a->unstable || !a->eta || !a->err ||
        !a->t0)
      return fail(ctx, RTG_ERR_ARG, "compact_gaussians: NULL array");
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    if (cudaMemsetAsync(count_out, 0, sizeof(int64_t), s) != cudaSuccess) return check_launch(ctx, "compact");
    return RTG_OK;
  }
  {
    ProfScope ps(ctx, kPCompact, s);
    launch_compact(n, C, remove, ctx->w.block_cnt, *in, *out, (long long *)count_out, s);
  }
  ctx->last_stream = s;
  return check_launch(ctx, "compact_gaussians");
}

rtg_status rtg_decode_rgbd(int32_t F, int32_t H, int32_t W, const uint8_t *rgb, const uint16_t *depth,
                           float depth_scale, float *color, float *depth_out, void *stream) {
  if (F < 1 || H < 1 || W < 1 || !(depth_scale > 0.f) || !isfinite(depth_scale) || rgb == nullptr ||
      depth == nullptr || color == nullptr || depth_out == nullptr)
    return RTG_ERR_ARG;
  launch_decode_rgbd(F, H, W, rgb, depth, depth_scale, color, depth_out, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? RTG_OK : RTG_ERR_CUDA;
}

rtg_status rtg_adam_step(int64_t nu, int32_t C, float *means, float *scales, float *quats, float *opacity,
                         float *colors, const float *g_means, const float *g_scales, const float *g_quats,
                         const float *g_opacity, const float *g_colors, float *m, float *v, int32_t step,
                         const rtg_adam_params *hp, void *stream) {
  if (nu < 0 || C < 1 || C > 64 || step < 1 || hp == nullptr) return RTG_ERR_ARG;
  if (nu == 0) return RTG_OK;
  if (!means || !scales || !quats || !opacity || !colors || !g_means || !g_scales || !g_quats || !g_opacity ||
      !g_colors || !m || !v)
    return RTG_ERR_ARG;
  const double bc1 = 1.0 / (1.0 - pow((double)hp->beta1, step));
  const double bc2s = 1.0 / sqrt(1.0 - pow((double)hp->beta2, step));
  launch_adam(nu, C, means, scales, quats, opacity, colors, g_means, g_scales, g_quats, g_opacity, g_colors, m, v,
              *hp, (float)bc1, (float)bc2s, nullptr, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? RTG_OK : RTG_ERR_CUDA;
}

rtg_status rtg_adam_step_counted(int64_t nu, int32_t C, float *means, float *scales, float *quats, float *opacity,
                                 float *colors, const float *g_means, const float *g_scales, const float *g_quats,
                                 const float *g_opacity, const float *g_colors, float *m, float *v,
                                 int32_t *step_counter, const rtg_adam_params *hp, void *stream) {
  if (nu < 0 || C < 1 || C > 64 || hp == nullptr || step_counter == nullptr) return RTG_ERR_ARG;
  if (nu == 0) return RTG_OK;
  if (!means || !scales || !quats || !opacity || !colors || !g_means || !g_scales || !g_quats || !g_opacity ||
      !g_colors || !m || !v)
    return RTG_ERR_ARG;
  launch_adam(nu, C, means, scales, quats, opacity, colors, g_means, g_scales, g_quats, g_opacity, g_colors, m, v,
              *hp, 1.f, 1.f, step_counter, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? RTG_OK : RTG_ERR_CUDA;
}

rtg_status rtg_adam_step_counted_after_gradients(int64_t nu, int32_t C, float *means, float *scales, float *quats,
                                                float *opacity, float *colors, const float *g_means,
                                                const float *g_scales, const float *g_quats, const float *g_opacity,
                                                const float *g_colors, float *m, float *v, int32_t *step_counter,
                                                const rtg_adam_params *hp, void *stream) {
  if (nu < 0 || C < 1 || C > 64 || hp == nullptr || step_counter == nullptr) return RTG_ERR_ARG;
  if (nu == 0) return RTG_OK;
  if (!means || !scales || !quats || !opacity || !colors || !g_means || !g_scales || !g_quats || !g_opacity ||
      !g_colors || !m || !v)
    return RTG_ERR_ARG;
  launch_adam(nu, C, means, scales, quats, opacity, colors, g_means, g_scales, g_quats, g_opacity, g_colors, m, v,
              *hp, 1.f, 1.f, step_counter, (cudaStream_t)stream, true);
  return cudaGetLastError() == cudaSuccess ? RTG_OK : RTG_ERR_CUDA;
}

rtg_status rtg_unstable_index(rtg_ctx *ctx, int64_t n, const uint8_t *unstable, int32_t *ids, int64_t *nu_out,
                              void *stream) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  if (n < 0 || n > ctx->cap.max_gaussians) return fail(ctx, RTG_ERR_ARG, "n outside capacity");
  if (n > 0 && (unstable == nullptr || ids == nullptr)) return fail(ctx, RTG_ERR_ARG, "NULL pointer");
  if (nu_out == nullptr) return fail(ctx, RTG_ERR_ARG, "nu_out is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    cudaMemsetAsync(nu_out, 0, sizeof(int64_t), s);
    return check_launch(ctx, "unstable_index");
  }
  return rank_pass(ctx, unstable, n, nullptr, ids, nullptr, nu_out, s);
}

rtg_status rtg_unstable_rank(rtg_ctx *ctx, int64_t n, const uint8_t *unstable, int32_t *rank, int32_t *ids,
                             int64_t *nu_out, void *stream) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  if (n < 0 || n > ctx->cap.max_gaussians) return fail(ctx, RTG_ERR_ARG, "n outside capacity");
  if (n > 0 && (unstable == nullptr || ids == nullptr || rank == nullptr)) return fail(ctx, RTG_ERR_ARG, "NULL pointer");
  if (nu_out == nullptr) return fail(ctx, RTG_ERR_ARG, "nu_out is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    cudaMemsetAsync(nu_out, 0, sizeof(int64_t), s);
    return check_launch(ctx, "unstable_rank");
  }
  return rank_pass(ctx, unstable, n, rank, ids, nullptr, nu_out, s);
}

rtg_status rtg_gather_unstable(int64_t nu, int32_t C, const int32_t *ids, const float *means, const float *scales,
                               const float *quats, const float *opacity, const float *colors, float *u_means,
                               float *u_scales, float *u_quats, float *u_opacity, float *u_colors, void *stream) {
  if (nu < 0 || C < 1) return RTG_ERR_ARG;
  if (nu == 0) return RTG_OK;
  if (!ids || !means || !scales || !quats || !opacity || !colors || !u_means || !u_scales || !u_quats ||
      !u_opacity || !u_colors)
    return RTG_ERR_ARG;
  launch_gather(nu, C, ids, means, scales, quats, opacity, colors, u_means, u_scales, u_quats, u_opacity, u_colors,
                (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? RTG_OK : RTG_ERR_CUDA;
}

rtg_status rtg_scatter_unstable(int64_t nu, int32_t C, const int32_t *ids, const float *u_means,
                                const float *u_scales, const float *u_quats, const float *u_opacity,
                                const float *u_colors, float *means, float *scales, float *quats, float *opacity,
                                float *colors, void *stream) {
  if (nu < 0 || C < 1) return RTG_ERR_ARG;
  if (nu == 0) return RTG_OK;
  if (!ids || !means || !scales || !quats || !opacity || !colors || !u_means || !u_scales || !u_quats ||
      !u_opacity || !u_colors)
    return RTG_ERR_ARG;
  launch_scatter(nu, C, ids, u_means, u_scales, u_quats, u_opacity, u_colors, means, scales, quats, opacity, colors,
                 (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? RTG_OK : RTG_ERR_CUDA;
}

rtg_status rtg_unstable_mask(rtg_ctx *ctx, const rtg_camera *cams, int32_t F, const rtg_gaussians *g,
                             const rtg_render_params *prm, uint8_t *mask, void *stream) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  Prm P;
  rtg_status st = make_prm(ctx, prm, P);
  if (st != RTG_OK) return st;
  FrameSet fs;
  if ((st = make_frames(ctx, cams, F, prm, fs)) != RTG_OK) return st;
  GaussPtrs gp;
  if ((st = make_gauss(ctx, g, gp)) != RTG_OK) return st;
  if (mask == nullptr) return fail(ctx, RTG_ERR_ARG, "mask is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const int T = fs.cam[0].mtiles_x * fs.cam[0].mtiles_y;  // 16 x 16 tiles of the rule
  ctx->has_fwd = false;  // the mask pass reuses the forward's workspace
  ProfScope ps(ctx, kPUnstableMask, s);
  // every in-image tile is active: the unstable Gaussians are bucketed into all tiles
  Work w = ctx->w;
  if (gp.rank_map != nullptr) {
    w.rank = const_cast<int32_t *>(gp.rank_map);
    w.ids = const_cast<int32_t *>(gp.unstable_ids);
  }
  launch_tile_mask(fs, w, nullptr, T, fs.cam[0].mtiles_x, kTileShift, kTileShift, true, false,
                   gp.rank_map ? (long long)gp.n_unstable : -1ll, s);
  if (gp.u_means != nullptr && gp.rank_map == nullptr)
    if ((st = rank_pass(ctx, gp.unstable, gp.n, w.rank, w.ids, w.counters, nullptr, s)) != RTG_OK) return st;
  launch_project(gp, w, P, F, T, kProjMask, kCullUnstable, ctx->cap.max_pairs, s);
  launch_scan_tiles(w, F * T, ctx->cap.max_pairs, -1, nullptr, s, true);
  launch_mask_cover_tiles(w, P, gp.n, F, T, gp.C, mask, kCoverPlain, s);
  ctx->last_stream = s;
  return check_launch(ctx, "unstable_mask");
}

rtg_status rtg_get_stats(rtg_ctx *ctx, rtg_stats *out) {
  if (ctx == nullptr || out == nullptr) return RTG_ERR_ARG;
  if (cudaStreamSynchronize(ctx->last_stream) != cudaSuccess) {
    cudaError_t e = cudaGetLastError();
    return fail(ctx, RTG_ERR_CUDA, "get_stats: %s", cudaGetErrorString(e));
  }
  unsigned long long c[kNumCounters];
  if (cudaMemcpy(c, ctx->w.counters, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaError_t e = cudaGetLastError();
    return fail(ctx, RTG_ERR_CUDA, "get_stats: %s", cudaGetErrorString(e));
  }
  out->pairs = (int64_t)c[kPairs];
  out->fragments = (int64_t)c[kFragments];
  out->visible = (int64_t)c[kVisible];
  out->masked_pixels = (int64_t)c[kMaskedPix];
  out->n_unstable = (int64_t)c[kNumUnstable];
  out->warp_records = (int64_t)c[kWarpRecords];
  out->backward_steps = (int64_t)c[kBwdSteps];
  out->max_tile_pairs = (int32_t)c[kMaxTilePairs];
  out->status = (int32_t)*(volatile uint32_t *)ctx->status_host;
  out->tile_w = 1 << ctx->tune_fwd.tws;
  out->tile_h = 1 << ctx->tune_fwd.ths;
  out->window_stable = ctx->win.open ? (int64_t)c[kWinStable] : 0;
  out->window_pairs = 0;
  if (ctx->win.open && ctx->win.lists) {
    const int Wd = ctx->win.cams[0].width, Hd = ctx->win.cams[0].height;
    const int T = ((Wd + (1 << ctx->win.lists_tws) - 1) >> ctx->win.lists_tws) *
                  ((Hd + (1 << ctx->win.lists_ths) - 1) >> ctx->win.lists_ths);
    const size_t FT = (size_t)ctx->win.F * T;
    uint32_t last[2] = {0u, 0u};
    if (FT > 0 && cudaMemcpy(&last[0], ctx->win_soff + FT - 1, 4, cudaMemcpyDeviceToHost) == cudaSuccess &&
        cudaMemcpy(&last[1], ctx->win_scount + FT - 1, 4, cudaMemcpyDeviceToHost) == cudaSuccess)
      out->window_pairs = (int64_t)last[0] + last[1];
    else
      cudaGetLastError();
  }
  return RTG_OK;
}

rtg_status rtg_debug_binning(rtg_ctx *ctx, uint32_t *tile_offsets, uint32_t *sorted_ids, int32_t *rect,
                             uint32_t *zbits, void *stream) {
  if (ctx == nullptr) return RTG_ERR_ARG;
  if (!ctx->has_fwd) return fail(ctx, RTG_ERR_STATE, "debug_binning without a forward");
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaStreamSynchronize(ctx->last_stream) != cudaSuccess) return fail(ctx, RTG_ERR_CUDA, "sync failed");
  unsigned long long pairs = 0;
  cudaMemcpy(&pairs, ctx->w.counters + kPairs, sizeof(pairs), cudaMemcpyDeviceToHost);
  const size_t FT = (size_t)ctx->F * ctx->T;
  if (tile_offsets) cudaMemcpyAsync(tile_offsets, ctx->w.tile_offset, (FT + 1) * 4, cudaMemcpyDeviceToDevice, s);
  if (sorted_ids && pairs) cudaMemcpyAsync(sorted_ids, ctx->w.sorted, pairs * 4, cudaMemcpyDeviceToDevice, s);
  const int64_t NF = ctx->g.n * ctx->F;
  if ((rect || zbits) && NF > 0)
    launch(k_debug_extract, (unsigned)((NF + 255) / 256), 256, 0, s, ctx->w, ctx->g.n, ctx->F, rect, zbits);
  return check_launch(ctx, "debug_binning");
}

}  // extern "C"
