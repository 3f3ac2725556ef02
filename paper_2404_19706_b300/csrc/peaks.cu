// Throughput probes of the two arithmetic pipes the compositing kernels run on: FP32
// fused multiply-add and the special-function unit's base-2 exponential (the footprint's
// 2^-q).  The forward and backward compositing are not HBM-bound (their records sit in
// L2), so their binding roof is instruction issue on these pipes; these probes give the
// measured denominators of that roofline on the device at hand.  The paper has no
// counterpart: they measure the hardware, not the method.
//
// Every thread runs kChains independent dependency chains, so each SM sub-partition always
// has an independent instruction to issue; the launch fills every SM with 2,048 threads.
#include "kernels.cuh"

namespace rtg {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;  // 2,048 threads an SM

// kind 0: x = x * a + b on FP32 (2 flops an instruction); kind 1: x = 2^-x (one SFU op).
template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_alu_probe(float *out, int iters, float a, float b) {
  grid_dep_wait();
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = b + 0.001f * (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        if (KIND == 0) x[c] = fmaf(x[c], a, b);
        else x[c] = ex2_approx(-x[c]);
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // a store the compiler cannot drop, taken by no thread for these inputs (the chains stay finite)
  if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace rtg

extern "C" rtg_status rtg_alu_probe(int32_t kind, int32_t iters, float *out, int64_t *ops_out, void *stream) {
  if ((kind != 0 && kind != 1) || iters <= 0 || out == nullptr || ops_out == nullptr) return RTG_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess) {
    cudaGetLastError();
    return RTG_ERR_CUDA;
  }
  const int blocks = sms * rtg::kProbeBlocksPerSm;
  cudaStream_t s = (cudaStream_t)stream;
  if (kind == 0)
    rtg::launch(rtg::k_alu_probe<0>, blocks, rtg::kProbeThreads, 0, s, out, (int)iters, 0.9999999f, 1e-7f);
  else
    rtg::launch(rtg::k_alu_probe<1>, blocks, rtg::kProbeThreads, 0, s, out, (int)iters, 0.f, 0.5f);
  if (cudaGetLastError() != cudaSuccess) return RTG_ERR_CUDA;
  const int64_t instr = (int64_t)blocks * rtg::kProbeThreads * iters * 4 * rtg::kChains;
  *ops_out = kind == 0 ? 2 * instr : instr;  // FLOPs (an FMA is two) or SFU operations
  return RTG_OK;
}
