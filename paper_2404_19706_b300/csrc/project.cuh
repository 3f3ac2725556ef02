// EWA projection of one Gaussian into one camera (Section 3.1, Eq. 2 footprint and the
// disc-plane record used by Eq. 4/5).  Shared by the forward projection kernel and the
// unstable-mask kernel so that both evaluate exactly the same footprint.
#pragma once

#include "rtg_internal.cuh"

namespace rtg {

// ----------------------------------------------------------------------------- SH colour
// View-dependent colour (Section 3.1: c_i from the view direction r_i and the SH
// coefficients): the real, orthonormal spherical harmonics up to degree 3 (no
// Condon-Shortley phase), index k = l^2 + l + m, as polynomials of the unit direction
// (x, y, z).  c = sum_k SH[k] Y_k(r) with r = (p - t) / |p - t| from the camera centre t;
// no offset, no clamping.
constexpr int kShMax = 16;  // (3 + 1)^2
constexpr float kSh0 = 0.28209479177387814f;   // 1 / (2 sqrt(pi))
constexpr float kSh1 = 0.48860251190291992f;   // sqrt(3 / (4 pi))
constexpr float kSh2a = 1.0925484305920792f;   // sqrt(15 / pi) / 2
constexpr float kSh2b = 0.31539156525252005f;  // sqrt(5 / pi) / 4
constexpr float kSh2c = 0.54627421529603959f;  // sqrt(15 / pi) / 4
constexpr float kSh3a = 0.59004358992664352f;  // sqrt(35 / (2 pi)) / 4
constexpr float kSh3b = 2.8906114426405538f;   // sqrt(105 / pi) / 2
constexpr float kSh3c = 0.45704579946446572f;  // sqrt(21 / (2 pi)) / 4
constexpr float kSh3d = 0.37317633259011540f;  // sqrt(7 / pi) / 4
constexpr float kSh3e = 1.4453057213202769f;   // sqrt(105 / pi) / 4

__device__ __forceinline__ void sh_basis(int degree, float x, float y, float z, float (&Y)[kShMax]) {
  Y[0] = kSh0;
  if (degree < 1) return;
  Y[1] = kSh1 * y;
  Y[2] = kSh1 * z;
  Y[3] = kSh1 * x;
  if (degree < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kSh2a * x * y;
  Y[5] = kSh2a * y * z;
  Y[6] = kSh2b * (3.f * zz - 1.f);
  Y[7] = kSh2a * x * z;
  Y[8] = kSh2c * (xx - yy);
  if (degree < 3) return;
  Y[9] = kSh3a * y * (3.f * xx - yy);
  Y[10] = kSh3b * x * y * z;
  Y[11] = kSh3c * y * (5.f * zz - 1.f);
  Y[12] = kSh3d * z * (5.f * zz - 3.f);
  Y[13] = kSh3c * x * (5.f * zz - 1.f);
  Y[14] = kSh3e * z * (xx - yy);
  Y[15] = kSh3a * x * (xx - 3.f * yy);
}

// sum_k s_k grad Y_k at (x, y, z) (the polynomials' partial derivatives)
__device__ __forceinline__ void sh_dir_grad(int degree, float x, float y, float z, const float (&s)[kShMax],
                                            float &gx, float &gy, float &gz) {
  gx = 0.f; gy = 0.f; gz = 0.f;
  if (degree < 1) return;
  gy += kSh1 * s[1];
  gz += kSh1 * s[2];
  gx += kSh1 * s[3];
  if (degree < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  gx += kSh2a * y * s[4];  gy += kSh2a * x * s[4];
  gy += kSh2a * z * s[5];  gz += kSh2a * y * s[5];
  gz += 6.f * kSh2b * z * s[6];
  gx += kSh2a * z * s[7];  gz += kSh2a * x * s[7];
  gx += 2.f * kSh2c * x * s[8];  gy -= 2.f * kSh2c * y * s[8];
  if (degree < 3) return;
  gx += 6.f * kSh3a * x * y * s[9];  gy += 3.f * kSh3a * (xx - yy) * s[9];
  gx += kSh3b * y * z * s[10];  gy += kSh3b * x * z * s[10];  gz += kSh3b * x * y * s[10];
  gy += kSh3c * (5.f * zz - 1.f) * s[11];  gz += 10.f * kSh3c * y * z * s[11];
  gz += kSh3d * (15.f * zz - 3.f) * s[12];
  gx += kSh3c * (5.f * zz - 1.f) * s[13];  gz += 10.f * kSh3c * x * z * s[13];
  gx += 2.f * kSh3e * x * z * s[14];  gy -= 2.f * kSh3e * y * z * s[14];  gz += kSh3e * (xx - yy) * s[14];
  gx += 3.f * kSh3a * (xx - yy) * s[15];  gy -= 6.f * kSh3a * x * y * s[15];
}

// Colour of a Gaussian at p with coefficients coef [K][3] seen from the camera centre t.
__device__ __forceinline__ void sh_color(int degree, const float *__restrict__ coef, const float p[3],
                                         const float t[3], float (&col)[3]) {
  const float dx = p[0] - t[0], dy = p[1] - t[1], dz = p[2] - t[2];
  const float il = 1.f / sqrtf(dx * dx + dy * dy + dz * dz);
  float Y[kShMax];
  sh_basis(degree, dx * il, dy * il, dz * il, Y);
  const int K = (degree + 1) * (degree + 1);
  col[0] = col[1] = col[2] = 0.f;
  for (int k = 0; k < K; ++k) {
    col[0] = fmaf(coef[3 * k], Y[k], col[0]);
    col[1] = fmaf(coef[3 * k + 1], Y[k], col[1]);
    col[2] = fmaf(coef[3 * k + 2], Y[k], col[2]);
  }
}

struct Projected {
  df mux, muy;          // pixel-space centre (double-float)
  float u11, u12, u22;  // U with U^T U = Sigma_2D^-1 * kQScale^2 (upper triangular)
  float a, c;           // Sigma_2D diagonal (support bounds)
  float X, Y, Z;        // camera-frame centre
  float n[3];           // camera-frame disc normal (axis of the smallest scale)
  float d0;             // p_c . n_c
  int x0, y0, x1, y1;   // pixel bounding box of the alpha_min support (inclusive)
  float rx, ry;         // half-extents of that support around mu, with a safety margin
};

// Returns false when the Gaussian is culled (behind the near plane, outside the guard
// band, or with an empty support inside the image).  R is R(q) of the unit quaternion.
__device__ __forceinline__ bool project_gaussian(const DevCam &cam, const Prm &prm, const GParams &P,
                                                 const float R[9], int kmin, Projected &o) {
  // world -> camera, p_c = R_g^T (p - t_g), carried in double-float
  df d0 = two_sum(P.p[0], -cam.t[0]);
  df d1 = two_sum(P.p[1], -cam.t[1]);
  df d2 = two_sum(P.p[2], -cam.t[2]);
  df X = df_add(df_add(df_mul_f(d0, cam.R[0]), df_mul_f(d1, cam.R[3])), df_mul_f(d2, cam.R[6]));
  df Y = df_add(df_add(df_mul_f(d0, cam.R[1]), df_mul_f(d1, cam.R[4])), df_mul_f(d2, cam.R[7]));
  df Z = df_add(df_add(df_mul_f(d0, cam.R[2]), df_mul_f(d1, cam.R[5])), df_mul_f(d2, cam.R[8]));
  if (!(Z.hi > prm.near_z)) return false;
  const float rz = __fdividef(1.f, Z.hi);
  df tx = df_div_rcp(X, Z, rz), ty = df_div_rcp(Y, Z, rz);
  if (!(fabsf(tx.hi) <= cam.lim_x) || !(fabsf(ty.hi) <= cam.lim_y)) return false;
  o.mux = df_add(df_mul_f(tx, cam.fx), df{cam.cx, 0.f});
  o.muy = df_add(df_mul_f(ty, cam.fy), df{cam.cy, 0.f});
  const float Xf = X.hi, Yf = Y.hi, Zf = Z.hi;
  o.X = Xf; o.Y = Yf; o.Z = Zf;
  // A = W R with W = R_g^T: the Gaussian's axes in camera coordinates
  float A[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int cc = 0; cc < 3; ++cc)
      A[3 * r + cc] = cam.R[r] * R[cc] + cam.R[3 + r] * R[3 + cc] + cam.R[6 + r] * R[6 + cc];
  // M = J A S with J the perspective Jacobian at the centre; Sigma_2D = M M^T + lowpass I
  const float iz = rz;
  const float j00 = cam.fx * iz, j02 = -cam.fx * Xf * iz * iz;
  const float j11 = cam.fy * iz, j12 = -cam.fy * Yf * iz * iz;
  float a0 = 0.f, b0 = 0.f, c0 = 0.f;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    float m0 = (j00 * A[j] + j02 * A[6 + j]) * P.s[j];
    float m1 = (j11 * A[3 + j] + j12 * A[6 + j]) * P.s[j];
    a0 = fmaf(m0, m0, a0);
    b0 = fmaf(m0, m1, b0);
    c0 = fmaf(m1, m1, c0);
  }
  // det(M M^T) by Cauchy-Binet: the 2x2 minors of J A equal (fx fy / Z^3) times the
  // components of v = R^T (p - t) (A is a rotation), so the determinant is a sum of
  // squares and keeps full relative accuracy for thin, tilted footprints.
  float v[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) v[j] = R[j] * d0.hi + R[3 + j] * d1.hi + R[6 + j] * d2.hi;
  const float kk = cam.fx * cam.fy * iz * iz * iz;
  const float w0 = kk * v[0] * P.s[1] * P.s[2];
  const float w1 = kk * v[1] * P.s[0] * P.s[2];
  const float w2 = kk * v[2] * P.s[0] * P.s[1];
  const float lam = prm.lowpass;
  const float a = a0 + lam, c = c0 + lam;
  const float det = fmaf(w0, w0, fmaf(w1, w1, w2 * w2)) + lam * (a0 + c0) + lam * lam;
  float b = b0;
  if (2.f * b0 * b0 > a * c) b = copysignf(sqrtf(fmaxf(fmaf(a, c, -det), 0.f)), b0);
  if (!(det > 0.f)) return false;
  // Cholesky factor of the conic: Sigma_2D^-1 = U^T U, U = [[sqrt(c/det), -b/sqrt(c det)], [0, 1/sqrt(c)]]
  const float isc = rsqrtf(c), isd = rsqrtf(det);
  o.u11 = kQScale * (c * isc * isd);
  o.u12 = -kQScale * (b * isc * isd);
  o.u22 = kQScale * isc;
  o.a = a;
  o.c = c;
  // support f >= alpha_min  <=>  d^T Sigma_2D^-1 d <= 2 ln(alpha / alpha_min); its x extent is
  // sqrt(that * a), its y extent sqrt(that * c).  A small margin keeps the box a superset.
  if (!(P.alpha >= prm.alpha_min)) return false;
  const float pthr = 2.f * __logf(P.alpha / prm.alpha_min);
  const float rx = sqrtf(pthr * a) * 1.0001f + 1e-3f;
  const float ry = sqrtf(pthr * c) * 1.0001f + 1e-3f;
  o.rx = rx;
  o.ry = ry;
  const float mx = o.mux.hi, my = o.muy.hi;
  float fx0 = ceilf(mx - rx), fx1 = floorf(mx + rx), fy0 = ceilf(my - ry), fy1 = floorf(my + ry);
  fx0 = fmaxf(fx0, 0.f);
  fy0 = fmaxf(fy0, 0.f);
  fx1 = fminf(fx1, (float)(cam.W - 1));
  fy1 = fminf(fy1, (float)(cam.H - 1));
  if (!(fx0 <= fx1) || !(fy0 <= fy1)) return false;
  o.x0 = (int)fx0; o.x1 = (int)fx1; o.y0 = (int)fy0; o.y1 = (int)fy1;
  // column kmin of A, chosen by selects (a run-time index would put A in local memory)
#pragma unroll
  for (int r = 0; r < 3; ++r) o.n[r] = kmin == 0 ? A[3 * r] : (kmin == 1 ? A[3 * r + 1] : A[3 * r + 2]);
  o.d0 = Xf * o.n[0] + Yf * o.n[1] + Zf * o.n[2];
  return true;
}

// Footprint value f = min(f_max, alpha 2^-q) at pixel (px, py); q = |U d|^2, d = u - mu.
// The forward, the backward and the mask all use this expression, so their decisions agree.
__device__ __forceinline__ float footprint(float px, float py, float mxh, float myh, float mxl, float myl, float u11,
                                           float u12, float u22, float alpha, float f_max, float &dx, float &dy,
                                           float &t1, float &t2, float &g) {
  dx = (px - mxh) - mxl;
  dy = (py - myh) - myl;
  t1 = fmaf(u11, dx, u12 * dy);
  t2 = u22 * dy;
  const float q = fmaf(t1, t1, t2 * t2);
  g = ex2_approx(-q);
  return fminf(f_max, alpha * g);
}

// Conservative test that a footprint reaches alpha_min at some point of the pixel box
// [x0, x1] x [y0, y1] (pixel centres).  The support is q <= log2(alpha / alpha_min) with
// q = |U d|^2 convex in d, so its minimum over the box is 0 when the centre is inside, and
// otherwise lies on an edge, where it is a one-dimensional quadratic minimised at a clamped
// stationary point.  Margins cover FP32 rounding, so a record this test rejects has no pixel
// of the box with f >= alpha_min (per-pixel results do not change); it rejects the records
// whose bounding box, but not their ellipse, meets the box.
__device__ __forceinline__ bool reaches_box(const float4 &r0, const float4 &r1, float x0, float x1, float y0, float y1,
                                            float alpha_min) {
  const float dx0 = (x0 - r0.x) - r0.z, dx1 = (x1 - r0.x) - r0.z;
  const float dy0 = (y0 - r0.y) - r0.w, dy1 = (y1 - r0.y) - r0.w;
  if (dx0 <= 0.f && dx1 >= 0.f && dy0 <= 0.f && dy1 >= 0.f) return true;
  const float u11 = r1.x, u12 = r1.y, u22 = r1.z;
  const float a = u11 * u11, b = u11 * u12, c = fmaf(u12, u12, u22 * u22);
  // approximate reciprocals: they only move the edge minimiser, and q changes quadratically
  // there, far inside the margin below
  const float ia = __fdividef(1.f, a), ic = __fdividef(1.f, c);
  // q at (dx, dy) in the footprint's own form
  auto qat = [&](float dx, float dy) {
    const float t1 = fmaf(u11, dx, u12 * dy), t2 = u22 * dy;
    return fmaf(t1, t1, t2 * t2);
  };
  const float ya = fminf(fmaxf(-b * dx0 * ic, dy0), dy1), yb = fminf(fmaxf(-b * dx1 * ic, dy0), dy1);
  const float xa = fminf(fmaxf(-b * dy0 * ia, dx0), dx1), xb = fminf(fmaxf(-b * dy1 * ia, dx0), dx1);
  const float qmin = fminf(fminf(qat(dx0, ya), qat(dx1, yb)), fminf(qat(xa, dy0), qat(xb, dy1)));
  const float thr = __log2f(r1.w) - __log2f(alpha_min);
  return qmin <= fmaf(fabsf(thr), 1e-4f, thr) + 1e-3f;
}

}  // namespace rtg
