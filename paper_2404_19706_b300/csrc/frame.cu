// Sensor-frame decode: the RGB-D frames the method consumes (Section 3: every input frame is
// a colour image and a depth map) arrive as 8-bit interleaved colour and 16-bit depth in
// fixed units.  One thread per pixel writes the planar float colour (value / 255) and the
// depth in metres (value / depth_scale; 0, no measurement, stays 0), both with IEEE
// division, so the result equals the host conversion bit for bit.  Moving the frame in
// this form costs 5 bytes a pixel instead of 16.
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

void launch_decode_rgbd(int F, int H, int W, const uint8_t *rgb, const uint16_t *depth, float depth_scale,
                        float *color, float *depth_out, cudaStream_t s) {
  const int64_t HW = (int64_t)H * W, P = (int64_t)F * HW;
  if (P <= 0) return;
  const int64_t blocks = (P + 255) / 256;
  const int res = resident_grid((const void *)k_decode_rgbd, 256);
  launch(k_decode_rgbd, (unsigned)(blocks < res ? blocks : res), 256, 0, s, P, HW, rgb, depth, depth_scale, color,
         depth_out);
}

}  // namespace rtg
