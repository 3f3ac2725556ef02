// Sensor-frame decode: the RGB-D frames the method consumes (Section 3: every input frame is
// a colour image and a depth map) arrive as 8-bit interleaved colour and 16-bit depth in
// fixed units.  One thread per pixel writes the planar float colour (value / 255) and the
// depth in metres (value / depth_scale; 0, no measurement, stays 0), both with IEEE
// division, so the result equals the host conversion bit for bit.  Moving the frame in
// this form costs 5 bytes a pixel instead of 16.  Frames whose pixel count is a multiple of
// 4 (with aligned arrays) take four pixels a thread with vector loads and stores.
#include "kernels.cuh"

namespace rtg {

__global__ void __launch_bounds__(256) k_decode_rgbd(int64_t P, int64_t HW, const uint8_t *__restrict__ rgb,
                                                     const uint16_t *__restrict__ depth, float depth_scale,
                                                     float *__restrict__ color, float *__restrict__ depth_out) {
  grid_dep_wait();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = p / HW, q = p - f * HW;
    const uint8_t r = rgb[3 * p], g = rgb[3 * p + 1], b = rgb[3 * p + 2];
    float *c = color + f * 3 * HW + q;
    c[0] = (float)r / 255.f;
    c[HW] = (float)g / 255.f;
    c[2 * HW] = (float)b / 255.f;
    depth_out[p] = (float)depth[p] / depth_scale;
  }
}

// Four pixels a thread (HW a multiple of 4, every array 16-byte aligned): three 4-byte loads
// of colour, one 8-byte load of depth, a float4 store per plane.
__global__ void __launch_bounds__(256) k_decode_rgbd4(int64_t P4, int64_t HW4, const uint32_t *__restrict__ rgb,
                                                      const uint2 *__restrict__ depth, float depth_scale,
                                                      float4 *__restrict__ color, float4 *__restrict__ depth_out) {
  grid_dep_wait();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < P4; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = k / HW4, q = k - f * HW4;
    const uint32_t w0 = rgb[3 * k], w1 = rgb[3 * k + 1], w2 = rgb[3 * k + 2];
    const uint2 dd = depth[k];
    // bytes r0 g0 b0 r1 | g1 b1 r2 g2 | b2 r3 g3 b3 (little endian)
    auto byte = [](uint32_t w, int i) { return (float)((w >> (8 * i)) & 0xffu); };
    float4 *c = color + f * 3 * HW4 + q;
    c[0] = make_float4(byte(w0, 0) / 255.f, byte(w0, 3) / 255.f, byte(w1, 2) / 255.f, byte(w2, 1) / 255.f);
    c[HW4] = make_float4(byte(w0, 1) / 255.f, byte(w1, 0) / 255.f, byte(w1, 3) / 255.f, byte(w2, 2) / 255.f);
    c[2 * HW4] = make_float4(byte(w0, 2) / 255.f, byte(w1, 1) / 255.f, byte(w2, 0) / 255.f, byte(w2, 3) / 255.f);
    depth_out[k] = make_float4((float)(dd.x & 0xffffu) / depth_scale, (float)(dd.x >> 16) / depth_scale,
                               (float)(dd.y & 0xffffu) / depth_scale, (float)(dd.y >> 16) / depth_scale);
  }
}

void launch_decode_rgbd(int F, int H, int W, const uint8_t *rgb, const uint16_t *depth, float depth_scale,
                        float *color, float *depth_out, cudaStream_t s) {
  const int64_t HW = (int64_t)H * W, P = (int64_t)F * HW;
  if (P <= 0) return;
  const uintptr_t a = (uintptr_t)rgb | (uintptr_t)depth | (uintptr_t)color | (uintptr_t)depth_out;
  if (HW % 4 == 0 && (a & 15u) == 0u) {
    const int64_t P4 = P / 4, blocks = (P4 + 255) / 256;
    const int res = resident_grid((const void *)k_decode_rgbd4, 256);
    launch(k_decode_rgbd4, (unsigned)(blocks < res ? blocks : res), 256, 0, s, P4, HW / 4,
           reinterpret_cast<const uint32_t *>(rgb), reinterpret_cast<const uint2 *>(depth), depth_scale,
           reinterpret_cast<float4 *>(color), reinterpret_cast<float4 *>(depth_out));
    return;
  }
  const int64_t blocks = (P + 255) / 256;
  const int res = resident_grid((const void *)k_decode_rgbd, 256);
  launch(k_decode_rgbd, (unsigned)(blocks < res ? blocks : res), 256, 0, s, P, HW, rgb, depth, depth_scale, color,
         depth_out);
}

}  // namespace rtg
