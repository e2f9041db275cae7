// fr_device.cuh -- device helpers shared by the insertion kernels:
// the exact Hermitian-fold predicate, error-free sums, blob evaluation.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fr_internal.h"

namespace fr {

// ---------------------------------------------------------------- exact fold
//
// The fold decision (R00 kx + R01 ky < 0) must be taken on the exact real
// value, not an FP32-rounded one: a pixel on the wrong side lands at q instead
// of -q, an error of O(|p|) in two voxels.

// f = m * 2^e with integer m (|m| < 2^24): IEEE-754 binary32 decoding.
__device__ __forceinline__ long long decode_f32(float f, int *e) {
  unsigned int b = __float_as_uint(f);
  int ex = (b >> 23) & 0xFF;
  long long m = b & 0x7FFFFF;
  if (ex == 0) {
    *e = -149;  // subnormal (or zero)
  } else {
    m |= 0x800000;
    *e = ex - 150;
  }
  return (b >> 31) ? -m : m;
}

__device__ __forceinline__ int sgn64(long long v) { return (v > 0) - (v < 0); }

// Exact sign of a*ka + b*kb for binary32 a, b and integers |ka|, |kb| <= 4096.
static __device__ __noinline__ int exact_sign_fk2(float a, int ka, float b, int kb) {
  int ea, eb;
  long long A = decode_f32(a, &ea) * (long long)ka;  // |A| < 2^37
  long long B = decode_f32(b, &eb) * (long long)kb;
  if (A == 0) return sgn64(B);
  if (B == 0) return sgn64(A);
  long long big, small;
  int sh;
  if (ea >= eb) { big = A; small = B; sh = ea - eb; }
  else          { big = B; small = A; sh = eb - ea; }
  // sign(big * 2^sh + small)
  if (sh <= 25) return sgn64((big << sh) + small);  // |.| < 2^62
  if (sh > 50) return sgn64(big);                    // |big 2^sh| >= 2^51 > |small|
  // small = hi * 2^25 + lo, 0 <= lo < 2^25 ; sum = (big 2^(sh-25) + hi) 2^25 + lo
  long long hi = small >> 25;            // arithmetic shift = floor division
  long long lo = small - (hi << 25);
  long long C = (big << (sh - 25)) + hi;  // |.| < 2^62
  if (C != 0) return sgn64(C);
  return lo > 0 ? 1 : 0;
}

// fold iff R00*kx + R01*ky < 0 (exact).  Fast path: the FP32 value decides
// whenever it is far from zero relative to its rounding error bound.
__device__ __forceinline__ bool fold_pred(float r00, float r01, int kx, int ky) {
  float fx = (float)kx, fy = (float)ky;
  float x = fmaf(r00, fx, r01 * fy);
  float mag = fabsf(r00 * fx) + fabsf(r01 * fy);
  if (fabsf(x) > mag * 4.76837158e-7f) return x < 0.0f;  // 2^-21 * mag
  return exact_sign_fk2(r00, kx, r01, ky) < 0;
}

// ---------------------------------------------------------------- error-free sums

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  float bp = s - a;
  float ap = s - bp;
  e = (a - ap) + (b - bp);
}

// (hi, lo) += x, keeping hi + lo a non-overlapping double-float.
__device__ __forceinline__ void dd_add(float &hi, float &lo, float x) {
  float s, e;
  two_sum(hi, x, s, e);
  e += lo;
  hi = s + e;
  lo = e - (hi - s);
}

// (hi, lo) += (xh, xl)
__device__ __forceinline__ void dd_add2(float &hi, float &lo, float xh, float xl) {
  float s, e;
  two_sum(hi, xh, s, e);
  e += lo + xl;
  hi = s + e;
  lo = e - (hi - s);
}

// Exact decision of |v - (kx e1 + ky e2)|^2 <= a^2 for integer v, k and
// binary32 e1, e2, a, in double-float arithmetic (error-free products and
// sums): the result differs from the real-number decision only if the two
// sides agree to ~2^-44 relative.  Used to re-decide candidates whose FP32 r^2
// lies within rounding of a^2 -- with a non-orthonormal FP32 rotation and an
// integer a^2, |R k| may sit a few ulps either side of a lattice distance.
static __device__ __noinline__ bool exact_r2_le_a2(int vx, int vy, int vz, float e1x, float e1y,
                                            float e1z, float e2x, float e2y, float e2z, int kx,
                                            int ky, float a) {
  const float e1[3] = {e1x, e1y, e1z}, e2[3] = {e2x, e2y, e2z};
  const int v[3] = {vx, vy, vz};
  float rh = 0.f, rl = 0.f;  // running r^2 as hi + lo
  for (int c = 0; c < 3; ++c) {
    // d = v_c - e1_c kx - e2_c ky
    const float p1 = e1[c] * (float)kx, x1 = fmaf(e1[c], (float)kx, -p1);
    const float p2 = e2[c] * (float)ky, x2 = fmaf(e2[c], (float)ky, -p2);
    float s, t, s2, t2;
    two_sum((float)v[c], -p1, s, t);
    two_sum(s, -p2, s2, t2);
    const float dl = ((t + t2) - x1) - x2;
    // d^2 = s2^2 + 2 s2 dl (+ dl^2, negligible)
    const float q = s2 * s2, qe = fmaf(s2, s2, -q);
    float h, e;
    two_sum(rh, q, h, e);
    rh = h;
    rl += e + qe + 2.0f * s2 * dl;
  }
  const float ah = a * a, al = fmaf(a, a, -ah);
  float dh, de;
  two_sum(rh, -ah, dh, de);
  return dh + (de + (rl - al)) <= 0.0f;
}

// ---------------------------------------------------------------- blob weights

// Tabulated blob: nodes at r^2 = i a^2 / (lut_n - 1), linear interpolation in
// r^2.  entry i = (b_i, b_{i+1} - b_i).  Requires 0 <= r2 * scale < lut_n.
// floor() by adding 2^23 with round-toward-zero: the low significand bits of
// the sum are the integer part, and x - floor(x) is exact.
__device__ __forceinline__ float blob_lut(const float2 *lut, float r2, float scale) {
  float x = r2 * scale;
  float t = __fadd_rz(x, 8388608.0f);
  int i = __float_as_int(t) - 0x4B000000;
  float f = x - (t - 8388608.0f);
  float2 e = lut[i];
  return fmaf(f, e.y, e.x);
}

// On-the-fly blob: b = I0(x)/I0(alpha), x = alpha sqrt(s), s = 1 - r^2/a^2,
// with the polynomial approximations of Abramowitz & Stegun (Handbook of
// Mathematical Functions, 1964), formula 9.8.1 for x <= 3.75 (|rel err| <
// 1.6e-7) and 9.8.2 for x > 3.75 (|rel err| < 1.9e-7).  For x > 3.75 the
// ratio is taken as exp(x - alpha) sqrt(alpha / x) P(3.75/x) / P(3.75/alpha)
// so nothing overflows.  The host supplies inv_i0a = 1/I0(alpha) and
// inv_pa = 1/P(3.75/alpha); no division is left on the device.
__device__ __forceinline__ float as_981(float t2) {  // t = x / 3.75
  return fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, 0.0045813f, 0.0360768f),
                                                    0.2659732f), 1.2067492f), 3.0899424f),
                       3.5156229f), 1.0f);
}
__device__ __forceinline__ float as_982(float u) {  // u = 3.75 / x
  return fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, 0.00392377f,
         -0.01647633f), 0.02635537f), -0.02057706f), 0.00916281f), -0.00157565f),
         0.00225319f), 0.01328592f), 0.39894228f);
}
__device__ __forceinline__ float blob_otf(float r2, float inv_a2, float alpha, float inv_i0a,
                                          float inv_pa) {
  const float t = r2 * inv_a2;                   // (r/a)^2
  const float s = fmaxf(1.0f - t, 1e-30f);
  const float rs = rsqrtf(s);                    // 1 / sqrt(s)
  const float sq = s * rs;                       // sqrt(s)
  const float x = alpha * sq;                    // alpha sqrt(s)
  if (x <= 3.75f) {
    const float u = x * (1.0f / 3.75f);
    return as_981(u * u) * inv_i0a;
  }
  // x - alpha = -alpha t / (1 + sqrt(s)) has no cancellation, so exp() sees an
  // argument accurate to a few ulp even when x is close to alpha
  const float xm = -alpha * t / (1.0f + sq);
  // sqrt(alpha / x) = s^(-1/4) = sqrt(rs)
  return expf(xm) * sqrtf(rs) * (as_982((3.75f / alpha) * rs) * inv_pa);
}

// Polynomial blob: b(r) = sum_k c_k x^k, x = 2 r^2 / a^2 - 1, the
// Chebyshev interpolant of degree 11 converted to the power basis on the host,
// evaluated as E(x^2) + x O(x^2) with E, O the even and odd parts (Horner in
// x^2 for each; absolute error below 1e-6 for the blobs it is enabled for).
// The branch-free gather box runs the same operations with packed FMAs.
__device__ __forceinline__ float blob_poly(float r2, float two_inv_a2, const float *c) {
  const float x = fmaf(r2, two_inv_a2, -1.0f);
  const float y = x * x;
  float e = c[POLY_N - 2], o = c[POLY_N - 1];
#pragma unroll
  for (int k = POLY_N / 2 - 2; k >= 0; --k) {
    e = fmaf(e, y, c[2 * k]);
    o = fmaf(o, y, c[2 * k + 1]);
  }
  return fmaf(o, x, e);
}

template <int WMODE>
__device__ __forceinline__ float blob_w(const float2 *lut, float r2, const InsertArgs &a,
                                        float inv_a2) {
  if (WMODE == W_LUT) return blob_lut(lut, r2, a.lut_scale);
  if (WMODE == W_POLY) return blob_poly(r2, 2.0f * inv_a2, a.poly);
  return blob_otf(r2, inv_a2, a.g.alpha, a.inv_i0a, a.inv_pa);
}

// ---------------------------------------------------------------- pixels

__device__ __forceinline__ float2 load_pixel(const void *images, int f16, size_t idx) {
  if (f16) {
    __half2 h = __ldg(reinterpret_cast<const __half2 *>(images) + idx);
    return __half22float2(h);
  }
  return __ldg(reinterpret_cast<const float2 *>(images) + idx);
}

__device__ __forceinline__ void set_err(int *err, int bit) {
  if (err) atomicOr(err, bit);
}

}  // namespace fr
