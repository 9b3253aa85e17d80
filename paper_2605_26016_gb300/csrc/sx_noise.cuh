// Counter-based thermal noise for the stochastic LLG field ("Stochastic
// Landau-Lifshitz-Gilbert simulations": B_th = sigma eta, eta ~ N(0,1) per
// Cartesian component).
//
// Generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11): ten rounds, each two 32x32->64-bit
// products with multipliers 0xD2511F53 and 0xCD9E8D57, the key bumped by the
// Weyl increments 0x9E3779B9 and 0xBB67AE85 before every round but the first.
// Counter (site_lo, site_hi, step_lo, replica << 8), key (seed_lo, seed_hi).
//
// Normals: u = (2*(x>>9)+1) * 2^-24 in (0,1); Box-Muller eta0, eta1 =
// sqrt(-2 ln u0) (cos, sin)(2 pi u1), eta2 = sqrt(-2 ln u2) cos(2 pi u3).
// ln and sincos are short polynomial evaluations in which every operation is
// a single correctly rounded FP32 operation (explicit _rn intrinsics, so the
// compiler cannot fuse or split them; each Horner step is one fused
// multiply-add, rounded once as IEEE 754 specifies), which makes the normals
// reproducible bit for bit on any IEEE machine that performs the same
// operation sequence:
//   ln u:  u = m 2^e with m in [sqrt(1/2), sqrt(2)], s = (m-1)/(m+1),
//          ln u = e ln2 + 2 s (1 + s^2/3 + s^4/5 + s^6/7 + s^8/9);
//   2 pi u: q = floor(4u), x = (4u - q) pi/2, Taylor sin to x^15 and cos to
//          x^14 in Horner form, then the quadrant rotation by q.
#pragma once
#include <stdint.h>

namespace sx {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t a = c[0], b = c[2];
    const uint32_t h0 = __umulhi(0xD2511F53u, a), l0 = 0xD2511F53u * a;
    const uint32_t h1 = __umulhi(0xCD9E8D57u, b), l1 = 0xCD9E8D57u * b;
    c[0] = h1 ^ c[1] ^ k0;
    c[1] = l1;
    c[2] = h0 ^ c[3] ^ k1;
    c[3] = l0;
  }
}

// Philox4x32-10 with the round keys precomputed (k0[r] = seed_lo + r 0x9E3779B9,
// k1[r] = seed_hi + r 0xBB67AE85): the same ten rounds as philox4x32_10, with
// the key schedule taken from kernel parameters instead of recomputed per site.
struct PhiloxKeys {
  uint32_t k0[10], k1[10];
};

inline PhiloxKeys philox_keys(uint64_t seed) {
  PhiloxKeys k;
  uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    k.k0[r] = a;
    k.k1[r] = b;
    a += 0x9E3779B9u;
    b += 0xBB67AE85u;
  }
  return k;
}

__device__ __forceinline__ void philox4x32_10_rk(uint32_t c[4], const PhiloxKeys &K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t a = c[0], b = c[2];
    const uint32_t h0 = __umulhi(0xD2511F53u, a), l0 = 0xD2511F53u * a;
    const uint32_t h1 = __umulhi(0xCD9E8D57u, b), l1 = 0xCD9E8D57u * b;
    c[0] = h1 ^ c[1] ^ K.k0[r];
    c[1] = l1;
    c[2] = h0 ^ c[3] ^ K.k1[r];
    c[3] = l0;
  }
}

// u = (2 (x >> 9) + 1) 2^-24: the float 1 + (x >> 9) 2^-23 built from its bits,
// minus 1 - 2^-24.  Both operands and the difference are exact FP32 values, so
// the subtraction is exact and u equals the value of the formula.
__device__ __forceinline__ float unit_open(uint32_t x) {
  return __fsub_rn(__uint_as_float(0x3F800000u | (x >> 9)), 0.99999994039535522f);
}

__device__ __forceinline__ float ln_open(float u) {
  const uint32_t bits = __float_as_uint(u);
  int e = (int)(bits >> 23) - 127;
  float m = __uint_as_float((bits & 0x007FFFFFu) | 0x3F800000u);
  if (m > 1.41421356f) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  const float s2 = __fmul_rn(s, s);
  float p = 0.111111111f;
  p = __fmaf_rn(p, s2, 0.142857143f);
  p = __fmaf_rn(p, s2, 0.2f);
  p = __fmaf_rn(p, s2, 0.333333333f);
  p = __fmaf_rn(p, s2, 1.0f);
  return __fmaf_rn(__int2float_rn(e), 0.693147181f, __fmul_rn(__fmul_rn(2.0f, s), p));
}

__device__ __forceinline__ void cos_sin_2pi(float u, float &cs, float &sn) {
  const float t = __fmul_rn(4.0f, u);
  const int q = (int)t;
  const float x = __fmul_rn(__fsub_rn(t, __int2float_rn(q)), 1.57079633f);
  const float x2 = __fmul_rn(x, x);
  float ps = -7.64716373e-13f;
  ps = __fmaf_rn(ps, x2, 1.60590438e-10f);
  ps = __fmaf_rn(ps, x2, -2.50521084e-8f);
  ps = __fmaf_rn(ps, x2, 2.75573192e-6f);
  ps = __fmaf_rn(ps, x2, -1.98412698e-4f);
  ps = __fmaf_rn(ps, x2, 8.33333333e-3f);
  ps = __fmaf_rn(ps, x2, -1.66666667e-1f);
  ps = __fmaf_rn(ps, x2, 1.0f);
  const float sx = __fmul_rn(ps, x);
  float pc = -1.14707456e-11f;
  pc = __fmaf_rn(pc, x2, 2.08767570e-9f);
  pc = __fmaf_rn(pc, x2, -2.75573192e-7f);
  pc = __fmaf_rn(pc, x2, 2.48015873e-5f);
  pc = __fmaf_rn(pc, x2, -1.38888889e-3f);
  pc = __fmaf_rn(pc, x2, 4.16666667e-2f);
  pc = __fmaf_rn(pc, x2, -0.5f);
  pc = __fmaf_rn(pc, x2, 1.0f);
  const float cx = pc;
  // quadrant rotation by q = 0..3: (cos, sin) = (c, s), (-s, c), (-c, -s), (s, -c); negation flips the sign
  // bit, which is exact, so the selects equal the case analysis
  const bool odd = (q & 1) != 0;
  const float a = odd ? sx : cx, b = odd ? cx : sx;
  cs = __uint_as_float(__float_as_uint(a) ^ ((unsigned)((q + 1) & 2) << 30));
  sn = __uint_as_float(__float_as_uint(b) ^ ((unsigned)(q & 2) << 30));
}

// Box-Muller on the four Philox words c: eta0, eta1 from (c0, c1), eta2 from (c2, c3).
__device__ __forceinline__ void box_muller3(const uint32_t c[4], float &e0, float &e1, float &e2) {
  const float r0 = __fsqrt_rn(__fmul_rn(-2.0f, ln_open(unit_open(c[0]))));
  float cs, sn, cs2, sn2;
  cos_sin_2pi(unit_open(c[1]), cs, sn);
  const float r1 = __fsqrt_rn(__fmul_rn(-2.0f, ln_open(unit_open(c[2]))));
  cos_sin_2pi(unit_open(c[3]), cs2, sn2);
  e0 = __fmul_rn(r0, cs);
  e1 = __fmul_rn(r0, sn);
  e2 = __fmul_rn(r1, cs2);
}

// Three standard normals for (seed, replica, site, step).
__device__ __forceinline__ void normals3(uint64_t seed, uint32_t replica, uint64_t site, uint64_t step, float &e0,
                                         float &e1, float &e2) {
  uint32_t c[4] = {(uint32_t)site, (uint32_t)(site >> 32), (uint32_t)step, replica << 8};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  box_muller3(c, e0, e1, e2);
}

// The same normals with the round keys of the seed precomputed (philox_keys).
__device__ __forceinline__ void normals3(const PhiloxKeys &K, uint32_t replica, uint64_t site, uint64_t step,
                                         float &e0, float &e1, float &e2) {
  uint32_t c[4] = {(uint32_t)site, (uint32_t)(site >> 32), (uint32_t)step, replica << 8};
  philox4x32_10_rk(c, K);
  box_muller3(c, e0, e1, e2);
}

}  // namespace sx
