/*
 * rtg.h — C ABI of the masked, depth-split differentiable Gaussian rasterizer
 * (RTG-SLAM, "on-the-fly Gaussian optimization": Section 3.1 rendering, Section 3.2
 * optimization, Supplement B masked rendering) for NVIDIA B300 (sm_103a).
 *
 * Conventions (Section 3.1, the pixel ray r(u) = (R_g K^-1 u') theta + t_g):
 *   - A camera pose T_g = [R_g | t_g] maps CAMERA to WORLD; R is row-major, so
 *     p_world = R * p_cam + t.  Camera axes: x right, y down, z forward.
 *   - Pixel (x, y) has its centre at integer coordinates; K = [fx 0 cx; 0 fy cy; 0 0 1].
 *   - Quaternions are (w, x, y, z) and are normalised inside; scales are linear metres;
 *     Sigma = R(q) diag(s)^2 R(q)^T.  The disc normal is the axis of the smallest scale
 *     (lowest index on ties).
 *   - Images are planar: colour [F, C, H, W], depth / alpha / index [F, H, W], float32.
 *
 * Memory: every array argument is a caller-owned DEVICE pointer unless marked HOST.
 * The context owns only its workspace, allocated once by rtg_create; no entry point
 * allocates device memory afterwards, so the calls can be captured in a CUDA graph.
 *
 * Streams: every call is asynchronous on the given cudaStream_t (passed as void*;
 * NULL = the legacy default stream).  Argument errors are reported synchronously
 * by the return value; device-side conditions (pair-buffer overflow) are recorded
 * in a status word that rtg_get_status() returns once the stream has been
 * synchronised, and the affected kernels skip their work (outputs untouched).
 * No call aborts or throws.
 */
#ifndef RTG_H
#define RTG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RTG_OK = 0,
  RTG_ERR_ARG = -1,         /* invalid argument (NULL pointer, size out of range) */
  RTG_ERR_CUDA = -2,        /* a CUDA runtime call failed; see rtg_last_error */
  RTG_ERR_WORKSPACE = -3,   /* the (Gaussian, tile) pairs exceeded the capacity */
  RTG_ERR_TIMEOUT = -4,     /* reserved: a bounded device-side wait gave up */
  RTG_ERR_UNSUPPORTED = -5, /* a configuration the library does not implement */
  RTG_ERR_STATE = -6        /* call order violated (backward without a forward) */
} rtg_status;

#define RTG_MAX_FRAMES 32 /* cameras per call (keyframe batch) */
#define RTG_TILE 16       /* tile grid of the unstable-mask rule: 16 x 16 pixels (Supplement B) */

/* Pinhole camera and camera-to-world pose T_g (Section 3.1). HOST struct. */
typedef struct {
  float fx, fy, cx, cy;
  int32_t width, height;
  float R[9]; /* row-major camera-to-world rotation R_g */
  float t[3]; /* camera centre t_g in world coordinates */
} rtg_camera;

/* Rendering constants.  delta_alpha and cos_max_angle come from Section 3.1
 * (e^-0.5 and cos 60 deg); tile_discard_frac from Supplement B (0.5; 0 = off);
 * the others are the 3DGS conventions the paper builds on: alpha_min = 1/255,
 * f_max = 0.99, t_eps = 1e-4 (stop before a fragment that would take the
 * transmission below it), lowpass = 0.3 px^2 added to Sigma_2D, near_z = 0.2 m,
 * guard_band = 1.3 (cull centres outside 1.3x the half field of view). */
typedef struct {
  float near_z, alpha_min, f_max, t_eps, delta_alpha, cos_max_angle, lowpass, guard_band,
      tile_discard_frac;
} rtg_render_params;

/* Gaussian arrays (Section 3.1 keeps every parameter in flat arrays addressed by the
 * Gaussian's index).  Structure-of-arrays, float32, device pointers:
 * means [n,3], scales [n,3], quats [n,4], opacity [n], colors [n,channels],
 * unstable [n] (uint8, non-zero = unstable, Section 3.2 state).
 * Optional compact overrides u_*: when u_means is non-NULL, the parameters of the
 * k-th unstable Gaussian (ascending index) are read from u_means[k], u_scales[k], ...
 * instead of the full arrays, so an optimiser can own compact [n_unstable, .] leaves.
 * Either all five u_* pointers are set or none.
 * Optional precomputed unstable index (from rtg_unstable_rank, valid while the flags do
 * not change, e.g. for a whole optimisation window): rank_map [n] int32 (compact index of
 * Gaussian i, -1 if stable), unstable_ids [n_unstable] int32 ascending, and their count.
 * When rank_map is non-NULL the calls skip recomputing the index.
 * View-dependent colour (Section 3.1: c_i from the view direction r_i and the SH
 * coefficients SH_i): with sh_degree d in 1..3, channels must be 3 and colors (and
 * u_colors) hold (d+1)^2 x 3 SH coefficients per Gaussian, [n][(d+1)^2][3], index
 * k = l^2 + l + m of the real orthonormal spherical harmonics without the Condon-Shortley
 * phase.  The colour seen from a camera with centre t is sum_k SH[k] Y_k(r),
 * r = (p - t) / |p - t|, with no offset and no clamping.  sh_degree 0: colors holds the
 * channels directly.  The colour gradients of the backward then have the same layout as
 * colors (one row of (d+1)^2 x 3 per Gaussian), and the position gradient includes the
 * view-direction term. */
typedef struct {
  int64_t n;
  int32_t channels; /* 3 (RGB) or 8 (feature channels); 3 with SH */
  const float *means, *scales, *quats, *opacity, *colors;
  const uint8_t *unstable;
  const float *u_means, *u_scales, *u_quats, *u_opacity, *u_colors;
  const int32_t *rank_map, *unstable_ids;
  int64_t n_unstable;
  int32_t sh_degree; /* 0 (colours) or 1..3 (SH coefficients) */
} rtg_gaussians;

/* Workspace capacity; every later call must stay within it. */
typedef struct {
  int64_t max_gaussians;
  int32_t max_frames;   /* <= RTG_MAX_FRAMES */
  int32_t max_width, max_height;
  int32_t max_channels; /* 3 or 8 */
  int64_t max_pairs;    /* (Gaussian, tile) pairs over all frames of one call */
} rtg_capacity;

typedef struct rtg_ctx rtg_ctx;

/* Counters of the last completed forward (read after synchronising its stream). */
typedef struct {
  int64_t pairs;          /* (Gaussian, tile) pairs emitted over masked tiles */
  int64_t fragments;      /* composited (pixel, Gaussian) fragments, Eq. 1 terms */
  int64_t visible;        /* (frame, Gaussian) projections that touch a masked tile */
  int64_t masked_pixels;  /* pixels rendered */
  int64_t n_unstable;     /* unstable Gaussians (rows of the compact gradients) */
  int64_t warp_records;   /* records the forward's warps walked after culling (each warp
                             composites 32 pixels against a record at once) */
  int32_t status;         /* device status word (rtg_status) */
  int32_t max_tile_pairs; /* longest per-tile list */
  int32_t tile_w, tile_h; /* render tile of that forward (rtg_tuning) */
  int64_t window_stable;  /* (frame, stable Gaussian) projections of the open window, made once
                             by rtg_window_begin (0 without a window) */
  int64_t window_pairs;   /* stable (Gaussian, tile) pairs in the window's cached sorted lists
                             (0 without cached lists) */
  int64_t backward_steps; /* steps of the last backward's fragment replay: each step a warp
                             takes one fragment on every lane that still has one (so
                             fragments / backward_steps = active lanes of 32) */
} rtg_stats;

/* Launch configuration of the render path.  Section 3.1 rasterises by screen tiles but
 * fixes neither their size nor how the work is spread over the GPU, so these are free
 * choices for an autotuner.  None of them changes a rendered value: colour, depth, alpha,
 * index map and unstable mask are bit-identical under every valid setting; the loss and
 * the gradients agree to float32 rounding (their summation order changes).
 *   tile_w x tile_h   render tile: 8x8, 8x16, 16x8, 16x16 or 32x8 pixels.  The tile rule
 *                     of the unstable mask stays on its own 16x16 grid (RTG_TILE).
 *   batch             records a warp tests against its pixel box and stages per step:
 *                     32 or 64.
 *   schedule          0: one CTA per tile, one warp per 32 masked pixels of it;
 *                     1: persistent warps that take (tile, 32-pixel group) items from a
 *                     queue ordered by tile list length, longest first, spanning every
 *                     frame of the call.
 *   persist_ctas_per_sm  schedule 1: CTAs of 256 threads per SM, 1..8.
 *   sort_digit_bits   radix digit width of the per-tile depth sort: 4 or 8.
 *   sort_rank_max     buckets of at most this many keys are ordered by ranking (a key's
 *                     position is the number of smaller keys) instead of radix passes;
 *                     0..2048, 0 = never.
 *   overlap           1: each call's kernels are launched with programmatic dependent
 *                     launch, so a kernel's CTAs are scheduled while its predecessor in
 *                     the stream drains; each waits for the predecessor's completion
 *                     before it touches memory.  0: plain stream order.  Kernels launched
 *                     while tracing is on (rtg_profile_enable) use plain order; the calls
 *                     that take no context (Adam, gather / scatter, state updates) always
 *                     launch with overlap.
 * Defaults: 16x16, 32, schedule 0, 4, 8, 0, 1.  A setting takes effect at the next forward;
 * the backward always uses the setting of the forward it follows. */
typedef struct {
  int32_t tile_w, tile_h;
  int32_t batch;
  int32_t schedule;
  int32_t persist_ctas_per_sm;
  int32_t sort_digit_bits;
  int32_t sort_rank_max;
  int32_t overlap;
} rtg_tuning;

/* Bytes of device workspace rtg_create allocates for `cap`. */
rtg_status rtg_workspace_size(const rtg_capacity *cap, size_t *bytes);

/* Create a context on the current device; allocates the workspace once.
 * On failure *out is NULL and the return value says why. */
rtg_status rtg_create(rtg_ctx **out, const rtg_capacity *cap);

/* Free a context and its workspace (NULL is accepted). */
rtg_status rtg_destroy(rtg_ctx *ctx);

/* Replace / read the context's launch configuration (HOST structs).  An invalid setting
 * returns RTG_ERR_ARG and leaves the current one in place.  The workspace is sized for
 * every valid setting, but smaller tiles make more (Gaussian, tile) pairs, so a forward
 * can overflow max_pairs under one tiling and not another (RTG_ERR_WORKSPACE status). */
rtg_status rtg_set_tuning(rtg_ctx *ctx, const rtg_tuning *t);
rtg_status rtg_get_tuning(rtg_ctx *ctx, rtg_tuning *out);

/* Unstable-pixel mask (Supplement B, Eq. S2): mask[f,y,x] = 1 where some unstable
 * Gaussian covers the pixel (f >= alpha_min, i.e. T_unstable < 1), then every 16x16
 * tile with fewer than tile_discard_frac of its in-image pixels covered is cleared.
 * cams: HOST array of F cameras sharing width/height; mask: [F,H,W] uint8 output. */
rtg_status rtg_unstable_mask(rtg_ctx *ctx, const rtg_camera *cams, int32_t F, const rtg_gaussians *g,
                             const rtg_render_params *prm, uint8_t *mask, void *stream);

/* Forward render over all Gaussians on the masked pixels (Section 3.1):
 * colour by front-to-back alpha compositing (Eq. 1, 2, 3), depth from the first
 * processed fragment with f > delta_alpha through the ray/disc-plane intersection
 * (Eq. 4) with the three cases of Eq. 5, alpha = 1 - final transmission, and the
 * index map of the depth-hit Gaussian (-1 if none).
 * cams: HOST array of F cameras (same width/height).  mask: [F,H,W] uint8 or NULL
 * (all pixels).  Outputs are written on masked pixels only; other pixels keep their
 * contents.  index_map may be NULL.  The context keeps the sorted lists and
 * per-pixel state for rtg_render_backward, which must follow before the next forward
 * on the same context, with the Gaussian arrays unchanged; it may be called more than
 * once for one forward (each call starts from zero screen-space gradients). */
rtg_status rtg_render_forward(rtg_ctx *ctx, const rtg_camera *cams, int32_t F, const rtg_gaussians *g,
                              const uint8_t *mask, const rtg_render_params *prm, float *color, float *depth,
                              float *alpha, int32_t *index_map, void *stream);

/* L1 losses of Section 3.2 (Eq. 7, Eq. 8 with w_reg = 0) on the masked pixels:
 * L_color = mean |C - C_hat| over masked pixels and channels; L_depth = mean |D - D_hat|
 * over masked pixels with D_hat != -1 and D > 0 (no depth loss without intersection).
 * loss_out: device float[3] = (L, L_color, L_depth).  dL_dcolor [F,C,H,W] and
 * dL_ddepth [F,H,W] receive the gradient of L (sign(0) = 0; zero off the mask). */
rtg_status rtg_l1_loss(rtg_ctx *ctx, int32_t F, int32_t C, int32_t H, int32_t W, const float *color,
                       const float *depth, const float *target_color, const float *target_depth,
                       const uint8_t *mask, float w_color, float w_depth, float *loss_out, float *dL_dcolor,
                       float *dL_ddepth, void *stream);

/* Backward of the last forward on this context (Section 3.1: the depth is linear in
 * position and rotation, hence differentiable): replays the compositing back to front
 * and writes the gradients of the loss for the UNSTABLE Gaussians only, compact, in
 * ascending original index: g_means [nu,3], g_scales [nu,3] (linear scale),
 * g_quats [nu,4] (raw quaternion), g_opacity [nu], g_colors [nu,C].
 * dL_dcolor [F,C,H,W] and dL_ddepth [F,H,W] are read on masked pixels only.
 * accumulate = 0 overwrites the gradient arrays; non-zero adds to their contents (so the
 * gradients of several forward/backward calls, e.g. one keyframe each, can be summed
 * before one optimiser step). */
rtg_status rtg_render_backward(rtg_ctx *ctx, const float *dL_dcolor, const float *dL_ddepth, float *g_means,
                               float *g_scales, float *g_quats, float *g_opacity, float *g_colors,
                               int32_t accumulate, void *stream);

/* The forward fused with the L1 losses: renders as rtg_render_forward and, in the same
 * pass, accumulates the terms of Eq. 7 against target_color [F,C,H,W] and target_depth
 * [F,H,W] (device); loss_out (device float[3]) receives (L, L_color, L_depth) exactly as
 * rtg_l1_loss defines them.  rtg_render_backward_l1 is then the backward of that loss: it
 * forms dL/dC_hat and dL/dD_hat per pixel itself, so no gradient images are written or
 * read.  The targets and outputs must stay unchanged until that backward has run. */
rtg_status rtg_render_forward_l1(rtg_ctx *ctx, const rtg_camera *cams, int32_t F, const rtg_gaussians *g,
                                 const uint8_t *mask, const rtg_render_params *prm, const float *target_color,
                                 const float *target_depth, float w_color, float w_depth, float *color, float *depth,
                                 float *alpha, int32_t *index_map, float *loss_out, void *stream);
/* rtg_decode_rgbd and rtg_render_forward_l1 in one call: the RGB-D sensor frame (rgb
 * [F,H,W,3] 8-bit, depth16 [F,H,W] 16-bit, depth_scale units a metre; device) is decoded into
 * target_color [F,3,H,W] and target_depth [F,H,W] exactly as rtg_decode_rgbd decodes it, and
 * the fused-L1 forward of rtg_render_forward_l1 runs against them (H, W the cameras'). The
 * call's tile-mask pass reads only the mask, so it runs while the decode does.  Results
 * equal the two calls'.  Needs 3 colour channels without SH, the target planes and loss_out;
 * a NULL frame or a depth scale that is not positive and finite: RTG_ERR_ARG. */
rtg_status rtg_render_forward_l1_frame(rtg_ctx *ctx, const rtg_camera *cams, int32_t F, const rtg_gaussians *g,
                                       const uint8_t *mask, const rtg_render_params *prm, const uint8_t *rgb,
                                       const uint16_t *depth16, float depth_scale, float *target_color,
                                       float *target_depth, float w_color, float w_depth, float *color, float *depth,
                                       float *alpha, int32_t *index_map, float *loss_out, void *stream);
rtg_status rtg_render_backward_l1(rtg_ctx *ctx, float *g_means, float *g_scales, float *g_quats, float *g_opacity,
                                  float *g_colors, int32_t accumulate, void *stream);

/* One keyframe batch split by frame over several GPUs (each rank renders its own frames of
 * the batch on its own context).  The means of Eq. 7 run over the pixels of the whole batch,
 * so a rank's backward needs the batch's pixel counts, not its own:
 *   rtg_loss_counts writes, after an rtg_render_forward_l1 (or a fused masked forward with
 *   targets), counts_out (device double[4]) = (P, P_d, sum |C_hat - C|, sum |D_hat - D|)
 *   of that forward: its masked pixels, its pixels in the depth term, and its two L1 sums;
 *   the caller sums these over the ranks (one all-reduce);
 *   rtg_set_loss_scales then sets the next rtg_render_backward_l1's gradient scales from the
 *   summed counts totals (device double[4]): w_color / (P C) and w_depth / P_d, and, when
 *   loss_out (device float[3]) is not NULL, writes the batch's loss (L, L_color, L_depth).
 * Each rank's gradients are then its share of the batch gradient, and their sum (a second
 * all-reduce of the compact gradient arrays) is the gradient of the whole batch; every rank
 * applies the same Adam step.  Asynchronous on `stream`; RTG_ERR_STATE without a forward
 * with targets, RTG_ERR_ARG for NULL counts. */
rtg_status rtg_loss_counts(rtg_ctx *ctx, double *counts_out, void *stream);
rtg_status rtg_set_loss_scales(rtg_ctx *ctx, const double *totals, float w_color, float w_depth, float *loss_out,
                               void *stream);

/* The unstable-pixel mask and the forward in one pass (Supplement B with Section 3.1):
 * builds the mask exactly as rtg_unstable_mask does and writes it to mask_out [F,H,W]
 * (every in-image pixel), then renders exactly those pixels as rtg_render_forward does,
 * sharing one projection of the Gaussians between the two.  With both targets (and
 * loss_out) it also fuses the L1 losses as rtg_render_forward_l1 does, so either
 * rtg_render_backward_l1 (targets given) or rtg_render_backward may follow. */
rtg_status rtg_render_forward_masked(rtg_ctx *ctx, const rtg_camera *cams, int32_t F, const rtg_gaussians *g,
                                     const rtg_render_params *prm, uint8_t *mask_out, const float *target_color,
                                     const float *target_depth, float w_color, float w_depth, float *color,
                                     float *depth, float *alpha, int32_t *index_map, float *loss_out, void *stream);

/* Optimisation window (Section 3.2): within a window only the unstable Gaussians are
 * optimised; the stable ones keep their parameters.  rtg_window_begin projects every stable
 * Gaussian into the window's F cameras once and keeps those records in the workspace, and
 * also the stable Gaussians' sorted per-tile lists over whole frames for the current render
 * tile (it synchronises `stream` once; if those lists exceed max_pairs only the records are
 * kept).  A later forward (any of the three rtg_render_forward* calls) whose cameras, render
 * parameters, Gaussian arrays (the same pointers) and precomputed unstable index
 * (rank_map, unstable_ids, n_unstable; required here) are those of rtg_window_begin then
 * projects, bins and sorts only the unstable Gaussians and merges them with the cached
 * lists: its results are identical to a forward without the window (rtg_stats.visible
 * then counts the unstable projections only).  rtg_set_tuning with a new render tile
 * rebuilds the lists (synchronising that stream).  The caller promises that the stable
 * Gaussians' parameters and the unstable flags do not change while the window is open.
 * Any forward that does not match closes the window (it rewrites the records), as does
 * rtg_window_end; rtg_window_is_open reports the state (1 open, 0 closed). */
rtg_status rtg_window_begin(rtg_ctx *ctx, const rtg_camera *cams, int32_t F, const rtg_gaussians *g,
                            const rtg_render_params *prm, void *stream);
rtg_status rtg_window_end(rtg_ctx *ctx);
int32_t rtg_window_is_open(rtg_ctx *ctx);

/* Global keyframe optimisation (Section 3.2, "Keyframes and global optimization"): every
 * Gaussian is optimised over a few keyframes, but only on the pixels of each keyframe with
 * the largest colour errors (the top 40% in the paper).
 *
 * rtg_select_top_error writes mask_out [F,H,W] (uint8, device): per frame, 1 on the
 * k = floor(frac * H * W) pixels of largest colour error e = |c_0 - t_0| + ... + |c_{C-1} -
 * t_{C-1}| (summed in float32 in channel order) between color and target_color [F,C,H,W]
 * (float32, device), 0 elsewhere; among equal errors the lower pixel index (row-major) is
 * taken first.  The selection is exact: errors are ordered by their IEEE bit patterns (a NaN
 * error ranks above every number).  frac in [0, 1]; k is computed in double precision.
 * Needs no forward; uses only the context's workspace; the inputs are read, not kept.
 *
 * rtg_narrow_pixels restricts the pixel set of the last forward on this context to the
 * pixels set in mask [F,H,W] (uint8, device; pixels the forward did not render are ignored),
 * so that the next backward replays only those pixels.  The forward's per-pixel state and
 * per-tile lists are reused as they are: no projection, binning or compositing runs again,
 * and the gradients equal those of a forward rendered on the narrowed mask, up to float32
 * summation order.  rtg_stats.masked_pixels then counts the narrowed pixels.  Narrowing
 * again keeps the intersection.
 * With target_color [F,C,H,W] and target_depth [F,H,W] (device) and loss_out (device
 * float[3]) it also forms the L1 losses of Eq. 7/8 on the narrowed pixels against those
 * targets (weights w_color, w_depth), exactly as rtg_render_forward_l1 defines them, so that
 * rtg_render_backward_l1 may follow (the targets must stay unchanged until it has run).
 * Without targets (all three NULL) form the loss with rtg_l1_loss on the same mask and call
 * rtg_render_backward; rtg_render_backward_l1 then returns RTG_ERR_STATE. */
rtg_status rtg_select_top_error(rtg_ctx *ctx, int32_t F, int32_t C, int32_t H, int32_t W, const float *color,
                                const float *target_color, double frac, uint8_t *mask_out, void *stream);
rtg_status rtg_narrow_pixels(rtg_ctx *ctx, const uint8_t *mask, const float *target_color, const float *target_depth,
                             float w_color, float w_depth, float *loss_out, void *stream);

/* Gaussian adding (Section 3.2, "Gaussians adding", Eq. 6).  From a full-frame render of
 * the map (rtg_render_forward with mask NULL: render_color [F,C,H,W], render_alpha,
 * render_depth [F,H,W] float32, index_map [F,H,W] int32) and the input frame (color
 * [F,C,H,W], depth [F,H,W] float32, <= 0 = no measurement), the pixels that get a new
 * Gaussian:
 *   M_s: 1 - alpha > delta_T or |D_hat - D| > delta_d (D_hat = -1 without a hit): new
 *        geometry, an opaque Gaussian (opacity_opaque);
 *   M_c: not in M_s and the mean over channels of |C_hat - C| > delta_c, tested as the
 *        float32 sum (channel order) > C * delta_c: a transparent Gaussian
 *        (opacity_transparent), unless the Gaussian of the pixel's depth hit (index map)
 *        is unstable (unstable[i] != 0) or there is none, when nothing is added.
 * Pixels with depth <= 0 are in neither.  Every decision is taken in float32.  Of these, a
 * uniform sample_rate is drawn: pixel p of frame f is drawn iff the top 24 bits of output
 * number f*H*W + p of the SplitMix64 stream seeded with `seed` are below
 * floor(sample_rate * 2^24) (computed in double precision).
 * Outputs, in ascending (frame, pixel) order, for the first `capacity` new Gaussians:
 * pixel_out [capacity] int32 (f*H*W + y*W + x), kind_out [capacity] uint8 (1 opaque,
 * 2 transparent), position_out [capacity,3] float32 (R (D K^-1 (x, y, 1)) + t with the
 * frame's camera-to-world pose), color_out [capacity,C] (the input colour), opacity_out
 * [capacity].  count_out (device int64) receives the number of new Gaussians, which may
 * exceed capacity (then only the first capacity are written).  Scales and rotations of the
 * new Gaussians (Supplement A) are the caller's.  cams: HOST array of F cameras of one
 * size; unstable [n_gaussians] uint8 (device).  Uses the context's workspace only; needs no
 * forward on this context (the render may come from any). */
typedef struct {
  float delta_T, delta_d, delta_c; /* 0.5, 0.1 m, 0.1 */
  float sample_rate;               /* 0.05 */
  float opacity_opaque;            /* 0.99 */
  float opacity_transparent;       /* 0.1 */
  uint64_t seed;
} rtg_add_params;
rtg_status rtg_add_candidates(rtg_ctx *ctx, const rtg_camera *cams, int32_t F, int32_t C, const float *render_color,
                              const float *render_alpha, const float *render_depth, const int32_t *index_map,
                              const float *color, const float *depth, const uint8_t *unstable, int64_t n_gaussians,
                              const rtg_add_params *p, int64_t capacity, int64_t *count_out, int32_t *pixel_out,
                              uint8_t *kind_out, float *position_out, float *color_out, float *opacity_out,
                              void *stream);

/* Transparent-Gaussian regulariser (Section 3.2, the L_reg term of Eq. 8): over the nu
 * optimised Gaussians in compact form (u_* [nu,.], layouts as rtg_gaussians) those with
 * u_opacity < alpha_split (0.5: transparent Gaussians are added at 0.1, opaque ones at 0.99)
 * are held to their values when added (means0 [nu,3], scales0 [nu,3], quats0 [nu,4]):
 * L_reg = w_reg x the mean over their position, raw quaternion and scale components of the
 * squared difference (w_reg = 1000 in the paper).  *loss_out (device float) receives
 * w_reg L_reg; its gradient is ADDED to g_means, g_scales, g_quats [nu,.] (call it after the
 * backward, before Adam).  No transparent Gaussian: loss 0, gradients unchanged.  Uses
 * the context's loss scratch. */
rtg_status rtg_transparent_reg(rtg_ctx *ctx, int64_t nu, const float *u_means, const float *u_scales,
                               const float *u_quats, const float *u_opacity, const float *means0,
                               const float *scales0, const float *quats0, float w_reg, float alpha_split,
                               float *g_means, float *g_scales, float *g_quats, float *loss_out, void *stream);

/* Fusion and state management (Section 3.2: "Gaussian optimization" with Eq. 9, and "State
 * management").  Per-Gaussian state arrays are device arrays of the caller: eta [n] int32
 * (confidence count), err [n] int32 (error count), t0 [n] int32 (frame of creation), and
 * the unstable flags [n] uint8.
 *
 * rtg_confidence_update: after an optimisation iteration, eta[ids[k]] += 1 for each of the
 * nu optimised Gaussians ids[k] (distinct) whose colour gradient row g_colors[k] [nu,C] has a
 * non-zero entry (its colour was updated).
 *
 * rtg_fuse_window (Eq. 9): at the end of a window, for each optimised Gaussian i = ids[k]
 * with eta_now[i] > 0: w = (eta_now[i] - eta_start[i]) / eta_now[i] and every stored
 * parameter becomes (1 - w) * prev + w * optimised, in float32 rounded per operation; prev is
 * the full array's row (the value before the window), optimised the compact row k of u_*
 * [nu, .] (layouts as rtg_gaussians).  Gaussians with eta_now[i] == 0 keep their row.  This
 * replaces rtg_scatter_unstable at the end of a window.
 *
 * rtg_error_count: from a full-frame render of the optimised map (render_color [F,C,H,W],
 * render_depth [F,H,W], index_map [F,H,W]) and the input frames (color, depth; depth <= 0 =
 * no measurement): a pixel errs if the float32 channel sum of |C_hat - C| > C * delta_c or,
 * where the input has depth, |D_hat - D| > delta_d; every stable Gaussian (unstable[i] == 0)
 * that is the depth hit of an erring pixel of frame f gets err[i] += 1, once per frame.
 * Uses the context's workspace (n <= max_gaussians).
 *
 * rtg_update_states at frame `frame`: stable with err > delta_e -> unstable (eta = err = 0);
 * unstable with eta > delta_eta -> stable (err = 0); otherwise unstable with
 * frame - t0 > delta_t -> remove[i] = 1 (remove [n] uint8 output, 0 elsewhere).
 *
 * rtg_compact_gaussians: copies the rows of every array of `in` whose remove flag is 0, in
 * order, to the same arrays of `out` (distinct buffers with room for n rows; C colour
 * channels per Gaussian); *count_out (device int64) = rows kept.  Uses the context's
 * workspace (n <= max_gaussians). */
typedef struct {
  int32_t delta_eta; /* 100 (synthetic scenes), 200 or 400 in the paper */
  int32_t delta_e;   /* not given in the paper */
  int32_t delta_t;   /* frames; not given in the paper */
  float delta_c, delta_d; /* 0.1, 0.1 m */
} rtg_state_params;
typedef struct {
  float *means, *scales, *quats, *opacity, *colors;
  uint8_t *unstable;
  int32_t *eta, *err, *t0;
} rtg_map_arrays;
rtg_status rtg_confidence_update(int64_t nu, int32_t C, const int32_t *ids, const float *g_colors, int32_t *eta,
                                 void *stream);
rtg_status rtg_fuse_window(int64_t nu, int32_t C, const int32_t *ids, const int32_t *eta_start,
                           const int32_t *eta_now, const float *u_means, const float *u_scales, const float *u_quats,
                           const float *u_opacity, const float *u_colors, float *means, float *scales, float *quats,
                           float *opacity, float *colors, void *stream);
rtg_status rtg_error_count(rtg_ctx *ctx, int32_t F, int32_t C, int32_t H, int32_t W, const float *render_color,
                           const float *render_depth, const int32_t *index_map, const float *color, const float *depth,
                           const uint8_t *unstable, int64_t n, const rtg_state_params *p, int32_t *err, void *stream);
rtg_status rtg_update_states(int64_t n, int32_t frame, const int32_t *t0, const rtg_state_params *p,
                             uint8_t *unstable, int32_t *eta, int32_t *err, uint8_t *remove, void *stream);
rtg_status rtg_compact_gaussians(rtg_ctx *ctx, int64_t n, int32_t C, const uint8_t *remove, const rtg_map_arrays *in,
                                 const rtg_map_arrays *out, int64_t *count_out, void *stream);

/* Decode F RGB-D sensor frames (Section 3: each input frame is a colour image and a depth
 * map) into the float planes the loss reads.  DEVICE arrays:
 *   rgb   [F,H,W,3] uint8, interleaved;      color     [F,3,H,W] float32 = value / 255
 *   depth [F,H,W] uint16, depth_scale units; depth_out [F,H,W] float32 = value / depth_scale
 * (metres; a 0, no measurement, stays 0).  Both quotients are IEEE float32 divisions, equal
 * bit for bit to the same conversion on the host.  F, H, W >= 1, depth_scale > 0 and finite,
 * no NULL pointer, else RTG_ERR_ARG.  Asynchronous on `stream`; needs no context. */
rtg_status rtg_decode_rgbd(int32_t F, int32_t H, int32_t W, const uint8_t *rgb, const uint16_t *depth,
                           float depth_scale, float *color, float *depth_out, void *stream);

/* Adam (Kingma & Ba, Algorithm 1) on compact unstable parameters, in place, with the
 * per-group learning rates of Supplement C.  The scale is optimised in log space
 * (s <- s * exp(-step), gradient s * dL/ds).  m and v hold nu * (11 + C) float32 each,
 * laid out group by group like the parameters: means [nu,3], then scales [nu,3], quats
 * [nu,4], opacity [nu], colours [nu,C]; start them at zero.  `step` counts from 1.
 * C is the number of colour values per Gaussian ((d+1)^2 x 3 with SH colour).  With
 * colors_dc > 0, the first colors_dc values of each colour row (the degree-0 SH
 * coefficients: 3) use lr_colors and the others lr_colors_rest (Supplement C: 0.05 x
 * lr_SH0); colors_dc = 0 gives every colour value lr_colors. */
typedef struct {
  float lr_means, lr_scales, lr_quats, lr_opacity, lr_colors, beta1, beta2, eps;
  float lr_colors_rest;
  int32_t colors_dc;
} rtg_adam_params;
rtg_status rtg_adam_step(int64_t nu, int32_t C, float *means, float *scales, float *quats, float *opacity,
                         float *colors, const float *g_means, const float *g_scales, const float *g_quats,
                         const float *g_opacity, const float *g_colors, float *m, float *v, int32_t step,
                         const rtg_adam_params *hp, void *stream);

/* The same Adam step with its count kept on the device: step_counter is a device int32[2]
 * (start both at 0).  [0] counts completed steps: the call uses t = [0] + 1 for the bias
 * corrections and stores t when it finishes; [1] is scratch that returns to 0 after every
 * call.  The call needs no host-side step number and can be replayed from a captured CUDA
 * graph.  Two calls on one counter must not overlap on the GPU.  nu = 0 does nothing. */
rtg_status rtg_adam_step_counted(int64_t nu, int32_t C, float *means, float *scales, float *quats, float *opacity,
                                 float *colors, const float *g_means, const float *g_scales, const float *g_quats,
                                 const float *g_opacity, const float *g_colors, float *m, float *v,
                                 int32_t *step_counter, const rtg_adam_params *hp, void *stream);

/* rtg_adam_step_counted for a stream on which the kernel just in front of this call writes
 * neither the parameters nor m, v nor the step counter (it may write the gradients: a
 * backward, a regulariser's gradient).  Under that contract the step starts loading the
 * parameters and moments while that kernel finishes; the results are those of
 * rtg_adam_step_counted.  If the kernel in front does write any of them, the results are
 * undefined: use rtg_adam_step_counted.  Arguments and errors as rtg_adam_step_counted. */
rtg_status rtg_adam_step_counted_after_gradients(int64_t nu, int32_t C, float *means, float *scales, float *quats,
                                                float *opacity, float *colors, const float *g_means,
                                                const float *g_scales, const float *g_quats, const float *g_opacity,
                                                const float *g_colors, float *m, float *v, int32_t *step_counter,
                                                const rtg_adam_params *hp, void *stream);

/* Unstable-subset helpers: ids[k] = index of the k-th unstable Gaussian (ascending),
 * *nu_out (device int64) = their count.  gather copies full rows into compact arrays;
 * scatter writes compact rows back into the full arrays. */
rtg_status rtg_unstable_index(rtg_ctx *ctx, int64_t n, const uint8_t *unstable, int32_t *ids, int64_t *nu_out,
                              void *stream);
/* As rtg_unstable_index, and also rank[n] (device int32): the compact index of Gaussian i
 * among the unstable ones, -1 if it is stable.  Feeds rtg_gaussians.rank_map. */
rtg_status rtg_unstable_rank(rtg_ctx *ctx, int64_t n, const uint8_t *unstable, int32_t *rank, int32_t *ids,
                             int64_t *nu_out, void *stream);
rtg_status rtg_gather_unstable(int64_t nu, int32_t C, const int32_t *ids, const float *means, const float *scales,
                               const float *quats, const float *opacity, const float *colors, float *u_means,
                               float *u_scales, float *u_quats, float *u_opacity, float *u_colors, void *stream);
rtg_status rtg_scatter_unstable(int64_t nu, int32_t C, const int32_t *ids, const float *u_means,
                                const float *u_scales, const float *u_quats, const float *u_opacity,
                                const float *u_colors, float *means, float *scales, float *quats, float *opacity,
                                float *colors, void *stream);

/* Allocation-free form of rtg_unstable_index, for callers that cannot allocate device
 * memory (the paper has no counterpart; this is a property of the library, not of the
 * method).  A thread that runs beside a real-time mapping loop should not call cudaMalloc,
 * which can synchronise the device and stall the other threads' kernels, and a program
 * that has given its whole memory budget to its own pool may have none left for a
 * context workspace.  This call needs no context and allocates nothing: its scratch is a
 * fixed array of per-block counts inside the library, enough for n <= 16,777,216
 * Gaussians (64 KB, kept on every device that loads the library until the process
 * exits).  Larger n returns RTG_ERR_WORKSPACE without launching anything.  Outputs are as
 * for rtg_unstable_index: ids [nu] (device int32, ascending) and *nu_out (device int64).
 * The first call on each device looks up the scratch array's device address, so make it
 * before any stream capture.  The address is kept per device ordinal for the life of the
 * process: after cudaDeviceReset, or under a second driver context on the same device, it
 * would be stale, so neither is supported.  Calls share that one array, so two calls that overlap on
 * the GPU (different streams, no ordering between them) race; order them on one stream.
 * Every scratch entry a call reads is written earlier in the same call, so nothing needs
 * clearing between calls. */
rtg_status rtg_unstable_index_static(int64_t n, const uint8_t *unstable, int32_t *ids, int64_t *nu_out,
                                     void *stream);

/* Counters of the last forward (synchronises the context's last stream). HOST out. */
rtg_status rtg_get_stats(rtg_ctx *ctx, rtg_stats *out);

/* Device status word (RTG_OK or the first device-side error since the last reset);
 * call after synchronising the stream.  rtg_reset_status clears it. */
rtg_status rtg_get_status(rtg_ctx *ctx);
rtg_status rtg_reset_status(rtg_ctx *ctx);

/* Human-readable message of the last error on this context (never NULL). */
const char *rtg_last_error(rtg_ctx *ctx);

/* Tracing (per-kernel device time).  While enabled (off by default), every kernel
 * launcher of this context's entry points is bracketed by CUDA events on the stream it
 * runs on; do not enable it while capturing a CUDA graph.  rtg_profile_read waits for
 * the recorded events, then fills launches[k] and total_ms[k] for each kernel kind k
 * (names from rtg_profile_kind_name, count from rtg_profile_kinds) since the previous
 * read, and clears the record list.  Arrays are HOST, n_kinds >= rtg_profile_kinds(). */
rtg_status rtg_profile_enable(rtg_ctx *ctx, int32_t on);
int32_t rtg_profile_kinds(void);
const char *rtg_profile_kind_name(int32_t kind);
rtg_status rtg_profile_read(rtg_ctx *ctx, int64_t *launches, double *total_ms, int32_t n_kinds);

/* Arithmetic-pipe throughput probe (no counterpart in the paper: it measures the device, so
 * that the compositing kernels, which are bound by instruction issue rather than by HBM,
 * can be set against a measured roof).  Launches one kernel that fills every SM of the
 * current device (2,048 threads an SM, 8 independent dependency chains a thread) with
 * `iters` x 32 instructions a thread of one kind: kind 0 FP32 fused multiply-add
 * (counted as 2 flops), kind 1 the SFU base-2 exponential (ex2.approx, 1 op).  `out` is a
 * device float array of at least 2,048 x (number of SMs) entries; the kernel never writes
 * it in practice, but it must be valid.  *ops_out (HOST) receives the operations the
 * launch performs; the caller times the launch with CUDA events on `stream`.  Errors:
 * RTG_ERR_ARG for a bad kind, iters <= 0 or NULL pointers; RTG_ERR_CUDA if the launch
 * fails. */
rtg_status rtg_alu_probe(int32_t kind, int32_t iters, float *out, int64_t *ops_out, void *stream);

/* Binning introspection of the last forward (for exactness tests): tile_offsets
 * [F*T+1] (uint32, T = ceil(W/tile_w)*ceil(H/tile_h) render tiles per frame under the
 * forward's tuning, frame-major, row-major tiles), sorted_ids [pairs] (uint32 Gaussian
 * index per list entry, each tile's list in front-to-back order), and per (frame,
 * Gaussian): rect [F*n*4] int32 (first and last render-tile column and row touched, or -1
 * if culled) and zbits [F*n] uint32 (IEEE bits of the float32 camera depth used as the
 * sort key).  Any output may be NULL. */
rtg_status rtg_debug_binning(rtg_ctx *ctx, uint32_t *tile_offsets, uint32_t *sorted_ids, int32_t *rect,
                             uint32_t *zbits, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RTG_H */
