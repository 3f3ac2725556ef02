// Allocation-free variant of the unstable-index scan (rtg_unstable_index without a context).
//
// Some callers cannot allocate device memory: a state-management thread running beside a
// real-time mapping loop must not call cudaMalloc (it can synchronise the whole device and
// stall the other threads' kernels), and an application that has handed its memory budget
// to its own pool may have nothing left to give a context workspace.  This entry point
// therefore needs no rtg_ctx: its only scratch, the per-block counts of the two-kernel
// scan, lives in a fixed array in this file.  The caller still owns inputs and outputs.
#include <mutex>

#include "kernels.cuh"

namespace {

constexpr int64_t kStaticMaxGaussians = (int64_t)1 << 24;  // 16,777,216 Gaussians
constexpr int kStaticBlocks = (int)((kStaticMaxGaussians + rtg::kScanBlock - 1) / rtg::kScanBlock);
constexpr int kMaxDevices = 64;

// Per-block unstable counts (64 KB).  Every device that loads the library holds one copy
// until the process exits.  k_rank_count writes every entry it uses before k_rank_write
// reads it, so nothing here has to start at zero.
static __device__ __align__(256) int32_t g_block_counts[kStaticBlocks];

std::mutex g_mutex;
int32_t *g_counts_addr[kMaxDevices] = {};

// Device address of g_block_counts on the current device, looked up once per device.
// (In host code the symbol itself is only a host-side stand-in, not a device address.)
rtg_status scratch_for_current_device(int32_t **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return RTG_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return RTG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_counts_addr[dev] == nullptr) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_block_counts) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return RTG_ERR_CUDA;
    }
    g_counts_addr[dev] = (int32_t *)p;
  }
  *out = g_counts_addr[dev];
  return RTG_OK;
}

}  // namespace

extern "C" rtg_status rtg_unstable_index_static(int64_t n, const uint8_t *unstable, int32_t *ids, int64_t *nu_out,
                                                void *stream) {
  if (n < 0 || nu_out == nullptr || (n > 0 && (unstable == nullptr || ids == nullptr))) return RTG_ERR_ARG;
  if (n > kStaticMaxGaussians) return RTG_ERR_WORKSPACE;  // beyond the fixed scratch
  int32_t *counts = nullptr;
  rtg_status st = scratch_for_current_device(&counts);
  if (st != RTG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    if (cudaMemsetAsync(nu_out, 0, sizeof(int64_t), s) != cudaSuccess) {
      cudaGetLastError();
      return RTG_ERR_CUDA;
    }
    return RTG_OK;
  }
  rtg::launch_rank(unstable, n, counts, nullptr, ids, nullptr, nu_out, s);
  if (cudaGetLastError() != cudaSuccess) return RTG_ERR_CUDA;
  return RTG_OK;
}
