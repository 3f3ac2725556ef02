// Kernel declarations and small block-level helpers shared by the translation units.
#pragma once

#include "rtg_internal.cuh"

namespace rtg {

constexpr int kScanBlock = 1024;   // threads per block of the unstable-index scan
constexpr int kSortThreads = 256;  // threads per tile-sort CTA
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortCap = 2048;     // keys a tile-sort CTA sorts entirely in shared memory
constexpr int kSortCapSmall = 512; // ... in the variant for tiles of at most 64 pixels
constexpr int kLossBlocks = 296;   // 2 x 148 SMs
constexpr int kScanSingleMax = 8192;   // tiles up to which one CTA scans them all
constexpr int kScanBlockTiles = 4096;  // tiles per CTA of the multi-block scan (4 per thread)
constexpr int kQueueClasses = 4 * 32 + 4;  // cost classes of the persistent schedule's queue

// Blocks of `block` threads that one resident wave of `kernel` holds on the current
// device (SMs x blocks per SM at this kernel's register and shared-memory use).  Grid-
// stride kernels launched with this grid never queue a second wave of blocks that only
// find the work already taken.  Cached per kernel.
int resident_grid(const void *kernel, int block, size_t smem = 0);

// Programmatic dependent launch (sm_90 and later).  While the calling thread's overlap flag
// is set, launch() marks each kernel as a programmatic dependent of the previous kernel in
// its stream: its CTAs may be scheduled as soon as every CTA of the predecessor has begun,
// and they wait in grid_dep_wait() until the predecessor has completed and its writes are
// visible.  Every kernel opens with grid_dep_wait() (it returns at once after a plain
// launch), so no kernel reads or writes memory its predecessor still uses; the wait is
// transitive, since a kernel completes only after its own wait returned.  The wait then
// lets the kernel's own successor be scheduled.
__device__ __forceinline__ void grid_dep_wait() {
  asm volatile("griddepcontrol.wait;\n\tgriddepcontrol.launch_dependents;" ::: "memory");
}

bool launch_overlap();
void set_launch_overlap(bool on);

template <typename... P, typename... A>
void launch(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A... args) {
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = launch_overlap() ? &attr : nullptr;
  cfg.numAttrs = launch_overlap() ? 1 : 0;
  (void)cudaLaunchKernelEx(&cfg, kernel, args...);  // errors surface in the caller's check
}

// Launch configuration of the render path (the C ABI's rtg_tuning, validated, with the
// tile sides as shifts).
struct Tuning {
  int tws, ths;       // render tile 2^tws x 2^ths pixels
  int batch;          // records per warp batch: 32 or 64
  int schedule;       // 0: CTA per tile; 1: persistent warps over the item queue
  int ctas_per_sm;    // schedule 1
  int sort_bits;      // 4 or 8
  int sort_rank_max;  // 0..kSortCap
  int overlap;        // programmatic dependent launch between the kernels of a call
  int num_sms;        // of the context's device
  int gshift() const { return tws + ths - 5; }  // log2(32-pixel groups per tile)
};

// Cameras of one call, passed by value to the first kernel of a forward.
struct FrameSet {
  int F;
  DevCam cam[kMaxFrames];
};

__device__ __forceinline__ int block_sum_int(int v, int *s_warp) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) s_warp[wid] = v;
  __syncthreads();
  int t = 0;
  for (int k = 0; k < nw; ++k) t += s_warp[k];
  __syncthreads();
  return t;
}

// Reserves `cnt` consecutive slots of a global counter for every thread of the block with a
// single atomic per block (same-address atomics serialise in one L2 slice, so one per warp
// over a million threads is slow).  Returns this thread's first slot.  With `counter2`, the
// block's sum of `cnt2` is added to it in the same barrier round (a count: no slot is
// returned).  All threads of the block must call it; s_w must hold 2 * blockDim.x / 32
// entries.
__device__ __forceinline__ unsigned long long block_reserve(unsigned long long *counter, uint32_t cnt, uint32_t *s_w,
                                                            unsigned long long *s_base,
                                                            unsigned long long *counter2 = nullptr,
                                                            uint32_t cnt2 = 0u) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t incl = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_w[wid] = incl;
  if (counter2 != nullptr) {
    const uint32_t c2 = __reduce_add_sync(0xffffffffu, cnt2);
    if (lane == 0) s_w[nw + wid] = c2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0, run2 = 0;
    for (int k = 0; k < nw; ++k) {
      const uint32_t c = s_w[k];
      s_w[k] = run;
      run += c;
      if (counter2 != nullptr) run2 += s_w[nw + k];
    }
    if (counter2 != nullptr && run2) atomicAdd(counter2, (unsigned long long)run2);
    *s_base = run ? atomicAdd(counter, (unsigned long long)run) : 0ull;
  }
  __syncthreads();
  const unsigned long long r = *s_base + s_w[wid] + incl - cnt;
  __syncthreads();
  return r;
}

// First item of warp `wid` of a persistent 8-warp CTA.  The queue holds the longest lists
// first and a tile's groups next to each other.  With `spread` (grids of at most two CTAs
// an SM, where a CTA's warps are a quarter of the SM's or more) the first items go out a
// tile at a time (P = a full tile's groups, up to 8), round robin over the CTAs, so that
// the longest lists do not share the issue slots of a few SMs while the groups of a tile,
// which read the same records, share a CTA: warp k of CTA b takes item
// (k / P) * P * grid + P * b + k % P.  Otherwise (four or more CTAs an SM) CTA b takes
// items 8b .. 8b + 7, neighbouring tiles of the queue, whose records overlap in L1.
__device__ __forceinline__ uint32_t first_item(const Work &w, int wid, int spread) {
  if (!spread) return blockIdx.x * 8u + (uint32_t)wid;
  const int gs = w.cams[0].tws + w.cams[0].ths - 5;
  const uint32_t P = 1u << (gs < 0 ? 0 : (gs > 3 ? 3 : gs));
  const uint32_t k = (uint32_t)wid;
  return (k / P) * P * gridDim.x + P * blockIdx.x + k % P;
}

// 32 x 32 bit-matrix transpose across a warp: lane i passes row i (bit j = element (i, j))
// and gets column i back (bit j = element (j, i)).  Five butterfly stages: stage s swaps the
// off-diagonal s x s blocks of every 2s x 2s block between lanes i and i ^ s, so after the
// stages for s = 16, 8, 4, 2, 1 every block has been transposed in place.
__device__ __forceinline__ uint32_t bit_transpose32(uint32_t x, int lane) {
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    // low s bits of every 2s-bit group: 0x0000ffff, 0x00ff00ff, 0x0f0f0f0f, 0x33333333, 0x55555555
    const uint32_t m = s == 16 ? 0x0000ffffu : s == 8 ? 0x00ff00ffu : s == 4 ? 0x0f0f0f0fu : s == 2 ? 0x33333333u
                                                                                                   : 0x55555555u;
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, s);
    x = (lane & s) ? ((x & ~m) | ((y & ~m) >> s)) : ((x & m) | ((y & m) << s));
  }
  return x;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Pixel order inside a render tile of 2^tws x 2^ths pixels (returns the raster index
// y << tws | x of position t): Z order, the low bits of x and y interleaved (x first), the
// remaining bits of the longer side on top.  Every aligned run of 32 positions is then an
// 8 x 4 block, so the 32 pixels a warp composites form a compact box (a 16-pixel-wide tile
// in raster order would give a warp two rows).  The tile passes list masked pixels in this
// order.
__device__ __forceinline__ int tile_order_pixel(int t, int tws, int ths) {
  const int m = tws < ths ? tws : ths;
  int x = 0, y = 0;
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    if (b < m) {
      x |= ((t >> (2 * b)) & 1) << b;
      y |= ((t >> (2 * b + 1)) & 1) << b;
    }
  }
  const int hi = t >> (2 * m);
  if (tws > ths) x |= hi << m;
  else y |= hi << m;
  return (y << tws) | x;
}

// ---- host launchers (each defined in the translation unit of its kernels)
// bin.cu
// Per-tile masked-pixel counts over a grid of 2^tws x 2^ths tiles (tiles_x per row), and,
// with `lists`, the compacted pixel lists.  `setup`: also publish the cameras and clear
// the per-call counters (the first kernel of every call).
void launch_tile_mask(const FrameSet &fs, const Work &w, const uint8_t *mask, int T, int tiles_x, int tws, int ths,
                      bool setup, bool lists, long long nu_preset, cudaStream_t s, bool early = false);
void launch_rank(const uint8_t *unstable, int64_t n, int32_t *block_cnt, int32_t *rank, int32_t *ids,
                 unsigned long long *nu_counter, int64_t *nu_out, cudaStream_t s);
enum ProjMode { kProjForward = 0, kProjMask = 1, kProjFused = 2, kProjWindow = 3 };
// Which (frame, Gaussian) pairs the coarse cull considers (kCullUnstable walks the
// precomputed unstable list when there is one).
enum CullSet { kCullAll = 0, kCullUnstable = 1, kCullStable = 2 };
void launch_project(const GaussPtrs &g, const Work &w, const Prm &prm, int F, int T, int mode, int cull_set,
                    int64_t max_pairs, cudaStream_t s);
// Bins projected entries into the masked render tiles: with `cands`, the cull's candidates
// that the fused projection marked projected; with `stable`, the open window's list.
void launch_bin(const Work &w, int64_t N, int T, int64_t max_pairs, bool cands, bool stable, cudaStream_t s);
void launch_window_reset(const Work &w, cudaStream_t s);
// gshift >= 0: also build the persistent schedule's item queue (2^gshift groups per tile).
// extra != nullptr: tiles with masked pixels also hold extra[t] cached stable pairs.
// emit: also scatter the staged pairs into their buckets (fused into the scan when one CTA
// scans all the tiles, else a k_emit launch after it).
void launch_scan_tiles(const Work &w, int FT, int64_t max_pairs, int gshift, const uint32_t *extra, cudaStream_t s,
                       bool emit = false);
void launch_emit(const Work &w, cudaStream_t s);
// Rebuilds the persistent schedule's queue from the current pixel counts, with each tile's
// list length taken from the forward's offsets (which it leaves unchanged).
void launch_requeue(const Work &w, int FT, int gshift, cudaStream_t s);
// sort.cu
// Cached sorted stable lists of an open window (keys == nullptr: none): per tile its
// count and offset into keys.
struct StableLists {
  const unsigned long long *keys;
  const uint32_t *off;
  const uint32_t *count;
};
// keys_out != nullptr: write each tile's sorted keys there instead of the index lists.
// small: the tiles have at most 64 pixels (short lists; a variant with smaller buffers).
// order (or nullptr): CTA b sorts tile order[b] for b < counters[kSortTiles] (the tiles
// with keys, listed by the single-CTA scan with a persistent queue); the others return
void launch_sort_tiles(const Work &w, int FT, int bits, int rank_max, const StableLists &sl,
                       unsigned long long *keys_out, bool small, const uint32_t *order, cudaStream_t s);
void init_sort_attributes();
// frame.cu
void launch_decode_rgbd(int F, int H, int W, const uint8_t *rgb, const uint16_t *depth, float depth_scale,
                        float *color, float *depth_out, cudaStream_t s);
// forward.cu
// loss_out != nullptr (persistent schedule with fused targets): the forward also finalizes
// the L1 loss (loss_out[0..2] and the gradient scales), as launch_loss_finalize would.
// fmask != nullptr: also write, per (tile list entry, 32-pixel group), the lanes that
// composited the entry (8 x max_pairs words; the bucket keys and staging of the call are
// free by then), for launch_backward.
void launch_forward(int C, const Work &w, const Prm &prm, int64_t N, int F, int T, const Tuning &tn, float *color,
                    float *depth, float *alpha, int32_t *index_map, const float *tcolor, const float *tdepth,
                    float *loss_out, float w_c, float w_d, uint32_t *fmask, cudaStream_t s);
// backward.cu
// fmask: the last forward's composited-lane masks (nullptr after the forward was narrowed to
// a pixel subset: the groups changed, so the backward walks the lists with the culling).
void launch_backward(int C, const Work &w, const Prm &prm, int64_t N, int F, int T, const Tuning &tn,
                     const float *dL_dcolor, const float *dL_ddepth, const L1Fused &l1, const uint32_t *fmask,
                     bool segments, cudaStream_t s);
void init_backward_attributes();
void launch_loss_finalize(const Work &w, int FT, int gshift, int C, float w_c, float w_d, float *loss_out,
                          cudaStream_t s);
void launch_project_backward(const GaussPtrs &g, const Work &w, const Prm &prm, int F, float *g_means,
                             float *g_scales, float *g_quats, float *g_opacity, float *g_colors, bool accumulate,
                             cudaStream_t s);
// loss_adam_mask.cu
void launch_loss_counts(const Work &w, int C, double *out, cudaStream_t s);
void launch_set_loss_scales(const Work &w, int C, const double *tot, float w_c, float w_d, float *loss_out,
                            cudaStream_t s);
void launch_l1_loss(const Work &w, int F, int C, int H, int W, const float *color, const float *depth,
                    const float *tcolor, const float *tdepth, const uint8_t *mask, float w_c, float w_d,
                    float *loss_out, float *dL_dcolor, float *dL_ddepth, cudaStream_t s);
// Transparent-Gaussian regulariser over the compact optimised set (nu rows).
struct RegArgs {
  int64_t nu;
  const float *means, *scales, *quats, *opacity;  // current compact parameters
  const float *means0, *scales0, *quats0;         // values when the Gaussians were added
  float w_reg, alpha_split;
  float *g_means, *g_scales, *g_quats;            // gradients, added to
  float *part;                                    // [kLossBlocks * 2] scratch
  uint32_t *done;                                 // ticket, zero between calls
  float *scale;                                   // device scalar: 2 w_reg / (10 n_t)
};
void launch_transparent_reg(const RegArgs &a, float *loss_out, cudaStream_t s);
void launch_adam(int64_t nu, int C, float *means, float *scales, float *quats, float *opacity, float *colors,
                 const float *g_means, const float *g_scales, const float *g_quats, const float *g_opacity,
                 const float *g_colors, float *m, float *v, const rtg_adam_params &hp, float bc1, float bc2_sqrt,
                 int32_t *step_dev, cudaStream_t s, bool early = false);
void launch_gather(int64_t nu, int C, const int32_t *ids, const float *means, const float *scales,
                   const float *quats, const float *opacity, const float *colors, float *um, float *us, float *uq,
                   float *uo, float *uc, cudaStream_t s);
void launch_scatter(int64_t nu, int C, const int32_t *ids, const float *um, const float *us, const float *uq,
                    const float *uo, const float *uc, float *means, float *scales, float *quats, float *opacity,
                    float *colors, cudaStream_t s);
// mode 0: rtg_unstable_mask; 1: fused, and the render grid is the 16 x 16 mask grid, so the
// kernel also writes the render tiles' pixel counts and lists; 2: fused, other render grid.
enum CoverMode { kCoverPlain = 0, kCoverFusedSame = 1, kCoverFusedOther = 2 };
void launch_mask_cover_tiles(const Work &w, const Prm &prm, int64_t N, int F, int T, int C, uint8_t *mask,
                             int mode, cudaStream_t s);
// select.cu
constexpr int kSelThreads = 256;    // threads per block of the top-error selection
constexpr int kSelPerBlock = 1024;  // pixels per block (4 per thread)
constexpr int kSelPasses = 3;       // radix passes of 11, 10 and 10 bits
constexpr int kSelHistStride = 2048;
// Scratch of the top-error selection: keys [F][n] (error bits), hist [3][F][2048] followed by
// ticket [4][F] (cleared at the start of every call), state [F][2] (threshold key, equal
// keys still to take), tie [F][blocks per frame].
struct SelBufs {
  uint32_t *keys, *hist, *ticket, *state, *tie;
};
inline size_t sel_scratch_words(int F) { return (size_t)kSelPasses * F * kSelHistStride + (size_t)(kSelPasses + 1) * F; }
void launch_select_top_error(const SelBufs &b, int F, int C, int64_t n, uint32_t k, const float *color,
                             const float *target, uint8_t *mask, cudaStream_t s);
// Inputs of the L1 partials formed while narrowing (tcolor == nullptr: none): the last
// forward's colour and depth, the targets and the channel count.
struct NarrowLoss {
  const float *color, *depth, *tcolor, *tdepth;
  int C;
};
// Keeps only the pixels set in mask [F,H,W] in the last forward's per-tile pixel lists and
// sets the masked-pixel counter to their number; gshift >= 0 also rebuilds the persistent
// schedule's queue.  With nl.tcolor, also writes the fused L1 partials of the new groups.
void launch_narrow_pixels(const Work &w, int F, int T, int tws, int ths, const uint8_t *mask, int gshift,
                          const NarrowLoss &nl, cudaStream_t s);
// adding.cu
// Arguments of the Gaussian-adding pass: the render (colour [F,C,H,W], alpha, depth, index
// map [F,H,W]), the input frame (colour, depth), the stability flags, the thresholds (the
// colour one as C * delta_c), the draw (seed, floor(rate * 2^24)) and the outputs.
struct AddArgs {
  int C, H, W;
  int64_t n;
  const float *rcolor, *ralpha, *rdepth;
  const int32_t *index;
  const float *color, *depth;
  const uint8_t *unstable;
  float dT, dd, thr_c, op_opaque, op_transparent;
  uint64_t seed;
  uint32_t t24;
  int64_t capacity;
  long long *count_out;
  int32_t *pix_out;
  uint8_t *kind_out;
  float *pos_out, *col_out, *op_out;
  uint32_t *cnt;    // [F][blocks per frame] counts, then bases (the selection's tie scratch)
  uint8_t *kinds;   // [F][H][W] kind of each pixel (the selection's key scratch)
};
struct AddCam {
  float fx, fy, cx, cy;
  float R[9], t[3];
};
struct AddFrames {
  AddCam cam[kMaxFrames];
};
void launch_add_candidates(const AddArgs &a, const AddFrames &fr, int F, cudaStream_t s);
// state.cu
struct FuseArrays {
  float *means, *scales, *quats, *opacity, *colors;
  const float *u_means, *u_scales, *u_quats, *u_opacity, *u_colors;
};
void launch_confidence(int64_t nu, int C, const int32_t *ids, const float *g_colors, int32_t *eta, cudaStream_t s);
void launch_fuse(int64_t nu, int C, const int32_t *ids, const int32_t *eta_start, const int32_t *eta_now,
                 const FuseArrays &a, cudaStream_t s);
// bits: [n] uint32 scratch, zero on entry and left zero
void launch_error_count(int F, int C, int64_t HW, const float *rcolor, const float *rdepth, const int32_t *index_map,
                        const float *color, const float *depth, const uint8_t *unstable, int64_t n, float thr_c,
                        float dd, uint32_t *bits, int32_t *err, cudaStream_t s);
void launch_update_states(int64_t n, int32_t frame, const int32_t *t0, const rtg_state_params &p, uint8_t *unstable,
                          int32_t *eta, int32_t *err, uint8_t *remove, cudaStream_t s);
void launch_compact(int64_t n, int C, const uint8_t *remove, int32_t *block_cnt, const rtg_map_arrays &in,
                    const rtg_map_arrays &out, long long *count_out, cudaStream_t s);

}  // namespace rtg
