// Per-tile depth ordering: the second level of a most-significant-digit radix sort on
// the packed key (tile, IEEE bits of z_c, Gaussian index).  The tile digit was
// resolved by bucketing (k_emit); here one CTA per tile sorts its bucket by the
// remaining 64 bits with a stable least-significant-digit radix sort (digits of
// kBits = 4 or 8 bits), skipping digit positions on which all keys of the bucket agree.
// Buckets of up to kSortCap keys stay in shared memory for every pass; longer buckets
// stream through global memory in chunks, keeping running digit offsets so every pass
// stays stable.  A Gaussian enters a tile at most once, so the keys of a bucket are
// distinct, and buckets up to a tuned length are ordered by ranking instead: each key's
// position is the number of smaller keys.  The output is the list of Gaussian indices per
// tile in front-to-back order (Supplement B sorts by a key made of the tile and the
// view-space depth).
#include "kernels.cuh"

namespace rtg {

namespace {

template <int kCap>
struct SortSmem {
  unsigned long long a[kCap];
  unsigned long long b[kCap];
  uint16_t lrank[kCap];
  uint32_t cnt[kSortWarps * 256];  // [warp][digit], 2^kBits digits used
  uint32_t tot[256];
  uint32_t base[256];
  uint32_t run[256];
  unsigned long long red[2 * kSortWarps];
};

__device__ __forceinline__ unsigned long long shfl_xor_u64(unsigned long long v, int o) {
  return __shfl_xor_sync(0xffffffffu, v, o);
}

// OR and AND over the keys src[0..n) (global or shared), block-wide.
template <class S>
__device__ void varying_bits(const unsigned long long *src, uint32_t n, S &s, unsigned long long &vary) {
  unsigned long long o = 0ull, a = ~0ull;
  for (uint32_t j = threadIdx.x; j < n; j += kSortThreads) {
    const unsigned long long k = src[j];
    o |= k;
    a &= k;
  }
  for (int d = 16; d > 0; d >>= 1) {
    o |= shfl_xor_u64(o, d);
    a &= shfl_xor_u64(a, d);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s.red[wid] = o;
    s.red[kSortWarps + wid] = a;
  }
  __syncthreads();
  o = 0ull;
  a = ~0ull;
  for (int k = 0; k < kSortWarps; ++k) {
    o |= s.red[k];
    a &= s.red[kSortWarps + k];
  }
  vary = o & ~a;
  __syncthreads();
}

// Stable ranking of m <= kCap shared-memory keys by the kBits-bit digit at `shift`:
// warp w owns a contiguous chunk; within it, lanes with equal digits are grouped with
// match.any and ranked by lane order, chunk by chunk.  Afterwards
//   lrank[j]     rank of key j among equal digits of its warp chunk,
//   cnt[w][d]    number of digit-d keys in the chunks of warps before w,
//   tot[d]       number of digit-d keys.
template <int kBits, class S>
__device__ void rank_digits(const unsigned long long *src, int m, int shift, S &s) {
  constexpr int kRadix = 1 << kBits;
  constexpr unsigned long long kMask = (unsigned long long)(kRadix - 1);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < kSortWarps * kRadix; k += kSortThreads) s.cnt[k] = 0u;
  __syncthreads();
  const int per = (((m + kSortWarps - 1) / kSortWarps) + 31) & ~31;
  const int beg = wid * per, end = min(m, beg + per);
  uint32_t *mycnt = s.cnt + wid * kRadix;
  for (int b = beg; b < end; b += 32) {
    const int j = b + lane;
    const bool valid = j < end;
    const unsigned digit = valid ? (unsigned)((src[j] >> shift) & kMask) : 256u + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, digit);
    const int leader = __ffs(peers) - 1;
    uint32_t before = 0;
    if (valid && lane == leader) {
      before = mycnt[digit];
      mycnt[digit] = before + __popc(peers);
    }
    before = __shfl_sync(0xffffffffu, before, leader);
    if (valid) s.lrank[j] = (uint16_t)(before + __popc(peers & lanemask_lt()));
  }
  __syncthreads();
  if (threadIdx.x < kRadix) {
    const int d = threadIdx.x;
    uint32_t run = 0;
    for (int k = 0; k < kSortWarps; ++k) {
      const uint32_t c = s.cnt[k * kRadix + d];
      s.cnt[k * kRadix + d] = run;
      run += c;
    }
    s.tot[d] = run;
  }
  __syncthreads();
}

// Exclusive scan of kRadix <= 256 values by 256 threads (value of thread d is in[d]).
template <int kRadix, class S>
__device__ void scan_digits(const uint32_t *in, uint32_t *out, S &s) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t v = (int)threadIdx.x < kRadix ? in[threadIdx.x] : 0u;
  uint32_t inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  __shared__ uint32_t s_w[kSortWarps];
  if (lane == 31) s_w[wid] = inc;
  __syncthreads();
  uint32_t pre = 0;
  for (int k = 0; k < wid; ++k) pre += s_w[k];
  if ((int)threadIdx.x < kRadix) out[threadIdx.x] = pre + inc - v;
  __syncthreads();
}

template <int kBits, class S>
__device__ __forceinline__ void scatter_chunk(const unsigned long long *src, int m, int shift, const uint32_t *base,
                                              unsigned long long *dst, S &s) {
  constexpr int kRadix = 1 << kBits;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (((m + kSortWarps - 1) / kSortWarps) + 31) & ~31;
  const int beg = wid * per, end = min(m, beg + per);
  for (int j = beg + lane; j < end; j += 32) {
    const unsigned long long k = src[j];
    const unsigned d = (unsigned)((k >> shift) & (unsigned long long)(kRadix - 1));
    dst[base[d] + s.cnt[wid * kRadix + d] + s.lrank[j]] = k;
  }
}

}  // namespace


// Number of keys of the ascending array a[0..n) that are smaller than k.
__device__ __forceinline__ uint32_t count_below(const unsigned long long *a, uint32_t n, unsigned long long k) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a[mid] < k) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Writes list entry `pos` of the tile: the Gaussian index, or the whole key (keys_out).
__device__ __forceinline__ void put(const Work &w, unsigned long long *keys_out, uint32_t off, uint32_t pos,
                                    unsigned long long k) {
  if (keys_out != nullptr) keys_out[off + pos] = k;
  else w.sorted[off + pos] = (uint32_t)k;
}

// One CTA per tile.  The tile's bucket keys[off, off + n_b) is sorted (radix passes, or
// ranking for short buckets).  With cached stable lists (an open optimisation window),
// the bucket holds the unstable pairs only and the tile's list is the merge of the sorted
// bucket with the cached, sorted stable keys of the tile: a key's position is its index in
// its own list plus the number of smaller keys in the other (all keys are distinct).
template <int kBits, int kCap>
__global__ void __launch_bounds__(kSortThreads) k_sort_tiles(Work w, int rank_max, StableLists sl,
                                                             unsigned long long *keys_out,
                                                             const uint32_t *__restrict__ order) {
  grid_dep_wait();
  constexpr int kRadix = 1 << kBits;
  constexpr unsigned long long kMask = (unsigned long long)(kRadix - 1);
  if (w.counters[kSkip] != 0ull) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SortSmem<kCap> &s = *reinterpret_cast<SortSmem<kCap> *>(smem_raw);
  int tile = blockIdx.x;
  if (order != nullptr) {  // the tiles with keys, longest first: the heavy sorts start in the first wave
    const uint32_t listed = (uint32_t)w.counters[kSortTiles], t = order[blockIdx.x];
    if (blockIdx.x >= listed) return;
    tile = (int)t;
  }
  const uint32_t off = w.tile_offset[tile];
  const uint32_t n = w.tile_offset[tile + 1] - off;
  if (n == 0) return;
  const uint32_t nb = sl.keys != nullptr ? w.tile_count[tile] : n;  // bucket (unstable) keys
  const uint32_t ns = n - nb;                                        // cached stable keys
  const unsigned long long *sorted_b = nullptr;                      // the sorted bucket
  if (nb == 0) {
    // nothing to sort
  } else if (nb <= (uint32_t)(rank_max < kCap ? rank_max : kCap)) {  // distinct keys: position = number of smaller keys
    for (uint32_t j = threadIdx.x; j < nb; j += kSortThreads) s.a[j] = w.keys[off + j];
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < nb; j += kSortThreads) {
      const unsigned long long k = s.a[j];
      uint32_t pos = 0;
      for (uint32_t i = 0; i < nb; ++i) pos += s.a[i] < k ? 1u : 0u;
      s.b[pos] = k;
    }
    __syncthreads();
    sorted_b = s.b;
  } else if (nb <= (uint32_t)kCap) {
    for (uint32_t j = threadIdx.x; j < nb; j += kSortThreads) s.a[j] = w.keys[off + j];
    __syncthreads();
    unsigned long long vary;
    varying_bits(s.a, nb, s, vary);
    unsigned long long *cur = s.a, *oth = s.b;
    for (int shift = 0; shift < 64; shift += kBits) {
      if (((vary >> shift) & kMask) == 0ull) continue;
      rank_digits<kBits>(cur, (int)nb, shift, s);
      scan_digits<kRadix>(s.tot, s.base, s);
      scatter_chunk<kBits>(cur, (int)nb, shift, s.base, oth, s);
      __syncthreads();
      unsigned long long *t = cur;
      cur = oth;
      oth = t;
    }
    sorted_b = cur;
  } else {
    // long bucket: chunked passes through global memory
    unsigned long long *src = w.keys + off, *dst = w.keys_alt + off;
    unsigned long long vary;
    varying_bits(src, nb, s, vary);
    for (int shift = 0; shift < 64; shift += kBits) {
      if (((vary >> shift) & kMask) == 0ull) continue;
      if ((int)threadIdx.x < kRadix) s.tot[threadIdx.x] = 0u;
      __syncthreads();
      for (uint32_t j = threadIdx.x; j < nb; j += kSortThreads)
        atomicAdd(&s.tot[(unsigned)((src[j] >> shift) & kMask)], 1u);
      __syncthreads();
      scan_digits<kRadix>(s.tot, s.run, s);
      for (uint32_t c0 = 0; c0 < nb; c0 += kCap) {
        const int m = (int)min((uint32_t)kCap, nb - c0);
        for (int j = threadIdx.x; j < m; j += kSortThreads) s.a[j] = src[c0 + j];
        __syncthreads();
        rank_digits<kBits>(s.a, m, shift, s);
        scatter_chunk<kBits>(s.a, m, shift, s.run, dst, s);
        __syncthreads();
        if ((int)threadIdx.x < kRadix) s.run[threadIdx.x] += s.tot[threadIdx.x];
        __syncthreads();
      }
      unsigned long long *t = src;
      src = dst;
      dst = t;
      __syncthreads();
    }
    sorted_b = src;
  }
  if (ns == 0) {
    for (uint32_t j = threadIdx.x; j < nb; j += kSortThreads) put(w, keys_out, off, j, sorted_b[j]);
    return;
  }
  // merge with the tile's cached stable keys (staged in the free shared buffer if they fit)
  const unsigned long long *sk = sl.keys + sl.off[tile];
  unsigned long long *freebuf = sorted_b == s.a ? s.b : s.a;
  if (ns <= (uint32_t)kCap) {
    for (uint32_t j = threadIdx.x; j < ns; j += kSortThreads) freebuf[j] = sk[j];
    __syncthreads();
    sk = freebuf;
  }
  for (uint32_t j = threadIdx.x; j < nb; j += kSortThreads) {
    const unsigned long long k = sorted_b[j];
    put(w, keys_out, off, j + count_below(sk, ns, k), k);
  }
  for (uint32_t j = threadIdx.x; j < ns; j += kSortThreads) {
    const unsigned long long k = sk[j];
    put(w, keys_out, off, j + count_below(sorted_b, nb, k), k);
  }
}

void init_sort_attributes() {
  cudaFuncSetAttribute(k_sort_tiles<8, kSortCap>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(SortSmem<kSortCap>));
  cudaFuncSetAttribute(k_sort_tiles<4, kSortCap>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(SortSmem<kSortCap>));
}

void launch_sort_tiles(const Work &w, int FT, int bits, int rank_max, const StableLists &sl,
                       unsigned long long *keys_out, bool small, const uint32_t *order, cudaStream_t s) {
  // Tiles of at most 64 pixels have short lists: the variant whose buffers hold kSortCapSmall
  // keys fits twice as many CTAs on an SM (longer buckets take the chunked global-memory
  // path, longer stable lists are searched in place).
  if (small) {
    if (bits == 4)
      launch(k_sort_tiles<4, kSortCapSmall>, FT, kSortThreads, sizeof(SortSmem<kSortCapSmall>), s, w, rank_max, sl,
             keys_out, order);
    else
      launch(k_sort_tiles<8, kSortCapSmall>, FT, kSortThreads, sizeof(SortSmem<kSortCapSmall>), s, w, rank_max, sl,
             keys_out, order);
  } else if (bits == 4) {
    launch(k_sort_tiles<4, kSortCap>, FT, kSortThreads, sizeof(SortSmem<kSortCap>), s, w, rank_max, sl, keys_out,
           order);
  } else {
    launch(k_sort_tiles<8, kSortCap>, FT, kSortThreads, sizeof(SortSmem<kSortCap>), s, w, rank_max, sl, keys_out,
           order);
  }
}

}  // namespace rtg
