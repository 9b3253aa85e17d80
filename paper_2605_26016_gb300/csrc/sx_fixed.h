// 64-bit fixed-point helpers of the FP64 state renormalisation S' = x / |x|.
//
// GB300 executes FP64 arithmetic at about 1/70 of its FP32 rate, so the part of
// the normalisation that needs more than FP32 precision but no FP64 dynamic
// range -- eps = |x|^2 - 1 and t = (1 + eps)^(-1/2) - 1 for a spin x within
// 2^-10 of the unit sphere -- is computed here in integer arithmetic at
// 2^-60 resolution, finer than FP64 rounding of unit-size values (2^-53).
// The state sum x = S + d and the final S' = x + x t stay FP64 operations.
//
// The functions compile for the host as well (plain C++ with unsigned
// __int128), so that the arithmetic can be checked on a CPU against extended
// precision.
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define SX_FX_HD __host__ __device__ __forceinline__
#else
#define SX_FX_HD static inline
#endif

namespace sx {
namespace fx {

SX_FX_HD uint64_t dbits(double v) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t b;
  memcpy(&b, &v, 8);
  return b;
#endif
}

SX_FX_HD double from_bits(uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double v;
  memcpy(&v, &b, 8);
  return v;
#endif
}

SX_FX_HD uint64_t umulhi(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

SX_FX_HD int64_t mulhi(int64_t a, int64_t b) {
#if defined(__CUDA_ARCH__)
  return __mul64hi(a, b);
#else
  return (int64_t)(((__int128)a * b) >> 64);
#endif
}

SX_FX_HD int clz64(uint64_t a) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)a);
#else
  return a ? __builtin_clzll(a) : 64;
#endif
}

// |v| 2^62 rounded toward zero, for the bit pattern b of a double with |v| < 2
// (exponent field at most 1023).
SX_FX_HD uint64_t mag62(uint64_t b) {
  const int e = (int)((b >> 52) & 0x7FF);
  const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int s = e - 1013;  // v = m 2^(e - 1075), so v 2^62 = m 2^(e - 1013)
  const uint64_t r = s >= 0 ? (m << s) : (s > -64 ? (m >> -s) : 0ull);
  return e == 0 ? 0ull : r;
}

// The double T 2^-60 (exact) for |T| < 2^53.
SX_FX_HD double fixed60_to_double(int64_t T) {
  if (T == 0) return 0.0;
  const uint64_t sgn = T < 0 ? (1ull << 63) : 0ull;
  const uint64_t a = T < 0 ? (uint64_t)(-T) : (uint64_t)T;
  const int lz = clz64(a);                      // >= 11
  const uint64_t m = a << (lz - 11);            // leading bit at position 52
  const uint64_t e = (uint64_t)(1026 - lz);     // T 2^-60 = (m 2^-52) 2^(3 - lz)
  return from_bits(sgn | (((e - 1) << 52) + m));  // m's leading bit adds the last 1 to the exponent
}

// t = (1 + eps)^(-1/2) - 1 with eps = |x|^2 - 1 for the bit patterns b0..b2 of
// the components of x.  Returns false (t untouched) unless every |x_c| < 2 and
// |eps| < 2^-10; NaN and infinity fail the first test.
//   eps: sum of floor(U_c^2 / 2^64) with U_c = |x_c| 2^62, minus 2^60 (eps 2^60);
//   t = -eps/2 + 3/8 eps^2 - 5/16 eps^3 + 35/128 eps^4 - 63/256 eps^5 (binomial
//       series; the remainder 231/1024 eps^6 < 2^-62), the first three terms in
//       fixed point (eps^2 at 2^82, eps^3 at 2^91), the last two (< 2.6e-13) in
//       FP32 and rounded to the 2^-60 grid.
// Error: each truncation is below one unit of 2^-60, so |t - t_exact| < 2^-57.
SX_FX_HD bool t_of_x(uint64_t b0, uint64_t b1, uint64_t b2, double &t) {
  const uint64_t e0 = (b0 >> 52) & 0x7FF, e1 = (b1 >> 52) & 0x7FF, e2 = (b2 >> 52) & 0x7FF;
  if ((e0 > 1023) | (e1 > 1023) | (e2 > 1023)) return false;
  const uint64_t u0 = mag62(b0), u1 = mag62(b1), u2 = mag62(b2);
  const uint64_t Q = umulhi(u0, u0) + umulhi(u1, u1) + umulhi(u2, u2);  // |x|^2 2^60 (< 3 2^62)
  const uint64_t one = 1ull << 60, lim = 1ull << 50;
  if (Q <= one - lim || Q >= one + lim) return false;
  const int64_t E = (int64_t)Q - (int64_t)one;    // eps 2^60, |E| < 2^50
  const int64_t Es = E * 8192;                     // eps 2^73
  const int64_t P2 = mulhi(Es, Es);                // eps^2 2^82 (< 2^62)
  const int64_t P3 = mulhi(P2, Es);                // eps^3 2^91 (|.| < 2^61)
  const float ef = (float)(int32_t)(E >> 20) * 0x1p-40f;
  const float e2f = ef * ef;
  const float r45 = e2f * e2f * (0.2734375f - 0.24609375f * ef);  // 35/128 eps^4 - 63/256 eps^5
#if defined(__CUDA_ARCH__)
  const int64_t R45 = (int64_t)__float2int_rn(r45 * 0x1p60f);
#else
  const int64_t R45 = (int64_t)lrintf(r45 * 0x1p60f);
#endif
  const int64_t T = -(E >> 1) + (((P2 >> 3) * 3) >> 22) - (((P3 >> 3) * 5) >> 32) + R45;
  t = fixed60_to_double(T);
  return true;
}

}  // namespace fx
}  // namespace sx
