// Device helpers shared by the stencil and FFT backends.
#pragma once
#include <stdint.h>

#include "sx_fixed.h"
#include "sx_internal.h"

namespace sx {

// FP64 -> FP32 by integer bit operations (round half up on the first dropped
// bit; magnitudes below 2^-126 become zero; NaN, infinity and magnitudes beyond
// the FP32 range give unspecified finite values: the FP64 state update, not the
// FP32 field, detects them).  Avoids the FP64 conversion pipe,
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
// subnormals become zero; NaN and infinity give finite values, so callers that
// can meet them test for them separately).
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

// Larger of two values that propagates NaN from either operand (fmax drops a
// NaN operand, which would let a non-finite spin read as zero torque).
__device__ __forceinline__ double max_nan(double a, double b) { return (a > b || a != a) ? a : b; }

// |S_i x b_i| at site i of two component-plane fields of n sites.
__device__ __forceinline__ double torque_at(const double *__restrict__ S, const double *__restrict__ b, int64_t n,
                                            int64_t i) {
  const double s0 = S[i], s1 = S[n + i], s2 = S[2 * n + i];
  const double b0 = b[i], b1 = b[n + i], b2 = b[2 * n + i];
  const double t0 = s1 * b2 - s2 * b1, t1 = s2 * b0 - s0 * b2, t2 = s0 * b1 - s1 * b0;
  return sqrt(t0 * t0 + t1 * t1 + t2 * t2);
}

// NaN-propagating maximum over the NT threads of a block (sm: NT doubles);
// every thread returns the block's maximum.
template <int NT>
__device__ __forceinline__ double block_max_nan(double v, double *sm) {
  sm[threadIdx.x] = v;
  __syncthreads();
#pragma unroll
  for (int s = NT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] = max_nan(sm[threadIdx.x], sm[threadIdx.x + s]);
    __syncthreads();
  }
  const double r = sm[0];
  __syncthreads();
  return r;
}

// Torque maximum of a grid-stride share of the sites, reduced over the block
// (first pass of max_i |S_i x b_i|; the second pass is block_max_nan over the
// per-block partials).
template <int NT>
__device__ __forceinline__ double block_torque_max(const double *__restrict__ S, const double *__restrict__ b,
                                                   int64_t n, double *sm) {
  double best = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT)
    best = max_nan(best, torque_at(S, b, n, i));
  return block_max_nan<NT>(best, sm);
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

// The exact normalisation of renormalise64's rare cases (a large step, or a
// non-finite value), out of line so that its temporaries do not add to the
// register pressure of the kernels that inline the fast path.  d is widened
// with the IEEE conversion, which keeps NaN and infinity.
static __device__ __noinline__ bool renormalise64_exact(double s0, double s1, double s2, float d0, float d1, float d2,
                                                 double *out) {
  const double x0 = s0 + (double)d0, x1 = s1 + (double)d1, x2 = s2 + (double)d2;
  const double n2 = fma(x0, x0, fma(x1, x1, x2 * x2));
  if (!(n2 > 0.0 && n2 <= 1.79769313486231570e308)) {
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    return true;
  }
  const double r = 1.0 / sqrt(n2);
  out[0] = x0 * r;
  out[1] = x1 * r;
  out[2] = x2 * r;
  return false;
}

// S' = N[S + d] with FP64 state S and an FP32 step d.  x = S + d in FP64 (3
// additions, the rounding of the FP64 sum); t = |x|^(-1) - 1 in 64-bit fixed
// point (sx_fixed.h, error < 2^-57) whenever every |x_c| < 2 and
// | |x|^2 - 1 | < 2^-10; S' = x + x t (3 FP64 fused multiply-adds).  Larger steps
// and non-finite values take the exact x / |x| (renormalise64_exact).  Returns
// true, with out = x, when |x|^2 is zero or not finite: the caller reports that
// as a numeric error.  6 FP64 operations per site on the common path.
__device__ __forceinline__ bool renormalise64(const double S[3], const float d[3], double out[3]) {
  const double x0 = S[0] + f32_to_f64(d[0]);
  const double x1 = S[1] + f32_to_f64(d[1]);
  const double x2 = S[2] + f32_to_f64(d[2]);
  double t;
  // a NaN or infinite step widens to a magnitude of at least 2^128 and so fails the |x_c| < 2 test
  if (fx::t_of_x(fx::dbits(x0), fx::dbits(x1), fx::dbits(x2), t)) {
    out[0] = fma(x0, t, x0);
    out[1] = fma(x1, t, x1);
    out[2] = fma(x2, t, x2);
    return false;
  }
  return renormalise64_exact(S[0], S[1], S[2], d[0], d[1], d[2], out);
}

// x <- x / |x| in FP64 (the state update of FP64 plans).  Returns true, with x
// unchanged, when |x|^2 is zero or not finite.
__device__ __forceinline__ bool unit64_checked(double x[3]) {
  const double n2 = fma(x[0], x[0], fma(x[1], x[1], x[2] * x[2]));
  if (!(n2 > 0.0 && n2 <= 1.79769313486231570e308)) return true;
  const double r = rsqrt(n2);
  x[0] *= r;
  x[1] *= r;
  x[2] *= r;
  return false;
}

// Status word of a context (device memory, set by kernels, read and cleared by
// the host, see kStatusNumeric).
__device__ __forceinline__ void report_numeric(int *status, bool bad) {
  if (bad && status) atomicOr(status, kStatusNumeric);
}

}  // namespace sx
