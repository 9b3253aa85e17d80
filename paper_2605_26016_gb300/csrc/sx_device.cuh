// Device helpers shared by the stencil and FFT backends.
#pragma once
#include <stdint.h>

namespace sx {

// FP64 -> FP32 by integer bit operations (round half up on the first dropped
// bit; magnitudes below 2^-126 become zero).  Avoids the FP64 conversion pipe,
// which runs at ~1/70 of the FP32 rate on GB300.
__device__ __forceinline__ float f64_to_f32(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned a = hi & 0x7FFFFFFFu;
  if (a < 0x38100000u) return 0.0f;
  unsigned m = __funnelshift_l(lo, a - 0x38000000u, 3);
  m += (lo >> 28) & 1u;
  return __uint_as_float(m | (hi & 0x80000000u));
}

// FP32 -> FP64 by integer bit operations (exact for normal numbers; FP32
// subnormals become zero).
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned a = b & 0x7FFFFFFFu;
  if (a < 0x00800000u) return 0.0;
  const unsigned hi = (b & 0x80000000u) | ((a >> 3) + 0x38000000u);
  return __hiloint2double((int)hi, (int)(b << 29));
}

// Conversion between FP64 and the arithmetic type R of a kernel through the
// integer-bit helpers above (identity when the types agree).
template <typename To, typename From>
__device__ __forceinline__ To cvt(From v) {
  if constexpr (sizeof(To) == sizeof(From))
    return v;
  else if constexpr (sizeof(To) == 4)
    return f64_to_f32(v);
  else
    return f32_to_f64(v);
}

__device__ __forceinline__ int wrap_axis(int c, int n, int periodic, bool &ok) {
  if (c >= 0 && c < n) return c;
  if (!periodic) {
    ok = false;
    return 0;
  }
  c %= n;
  return c < 0 ? c + n : c;
}

// LLG right-hand side f = g [S x B + alpha S x (S x B)], g = -gamma/(1+alpha^2)
template <typename R>
__device__ __forceinline__ void llg_rhs_t(const R s[3], const R B[3], R g, R alpha, R f[3]) {
  const R t0 = s[1] * B[2] - s[2] * B[1];
  const R t1 = s[2] * B[0] - s[0] * B[2];
  const R t2 = s[0] * B[1] - s[1] * B[0];
  const R u0 = s[1] * t2 - s[2] * t1;
  const R u1 = s[2] * t0 - s[0] * t2;
  const R u2 = s[0] * t1 - s[1] * t0;
  f[0] = g * (t0 + alpha * u0);
  f[1] = g * (t1 + alpha * u1);
  f[2] = g * (t2 + alpha * u2);
}

__device__ __forceinline__ void rhs32(const float s[3], const float B[3], float g, float alpha, float f[3]) {
  llg_rhs_t<float>(s, B, g, alpha, f);
}

// S' = N[S + d] in FP64 with d given in FP32.  x = S + d, eps = |x|^2 - 1,
// c - 1 = t = eps (-1/2 + eps g(eps)) with g = 3/8 - 5/16 eps + 35/128 eps^2
// (binomial series of (1+eps)^(-1/2)), S' = x + x t.  11 FP64 operations.
__device__ __forceinline__ void renormalise64(const double S[3], const float d[3], double out[3]) {
  const double x0 = S[0] + f32_to_f64(d[0]);
  const double x1 = S[1] + f32_to_f64(d[1]);
  const double x2 = S[2] + f32_to_f64(d[2]);
  const double eps = fma(x0, x0, fma(x1, x1, fma(x2, x2, -1.0)));
  const float e = f64_to_f32(eps);
  const float gq = fmaf(e, fmaf(e, 0.2734375f, -0.3125f), 0.375f);
  const double t = eps * fma(eps, f32_to_f64(gq), -0.5);
  out[0] = fma(x0, t, x0);
  out[1] = fma(x1, t, x1);
  out[2] = fma(x2, t, x2);
}

}  // namespace sx
