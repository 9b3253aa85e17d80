// Stencil backend: the sparse-convolution realisation of the bilinear field
//   b_a^alpha(R) = sum_b sum_delta sum_beta K_ab^{alpha beta}(delta) S_b^beta(R + delta)
// ("Backend representations"), fused with the normalised Heun step of the
// stochastic LLG equation ("Atomistic spin dynamics", "Stochastic LLG").
//
// GB300 design:
//  * Lattice families fix the tap geometry at compile time (which (b, delta)
//    taps exist and whether a tap is a scalar or a full 3x3 tensor); the J
//    values are kernel parameters, so any Hamiltonian whose taps fit a family
//    runs on it.  Families: simple cubic nearest neighbours, simple cubic
//    3x3x3 cube (three distance shells), bcc as two sublattices with four
//    distance shells.
//  * A CTA owns a 32 x BY column tile and marches along z.  Each S^n plane is
//    loaded once (FP64 from HBM, turned into FP32 with integer bit operations,
//    staged in shared memory as float4) and every (source sublattice, dx, dy)
//    group is read from shared memory once and pushed into per-thread register
//    accumulators for every dz, so a site costs one LDS.128 per group instead
//    of one per tap.
//  * Heun fusion: the predictor runs on the tile plus an r-wide halo and keeps
//    S~ in shared memory; the corrector runs on the interior.  HBM traffic per
//    spin-step is one FP64 read and one FP64 write (48 B).  Thermal noise is
//    drawn once per site and step and reused by the corrector.
//  * Mixed precision: field, torque and predictor in FP32; the corrector's
//    state sum S^n + dt/2 (f0 + f1) and its renormalisation in FP64 (GB300's
//    FP64 pipe is ~1/70 of FP32, so conversions use integer bit operations and
//    the FP64 pipe only runs the normalisation).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <utility>
#include <vector>

#include "sx_device.cuh"
#include "sx_internal.h"
#include "sx_noise.cuh"
#include "sx_schedule.h"

namespace sx {

// ------------------------------------------------------------------ families

struct TapSpec {
  int a, b, dx, dy, dz, tensor, coef;
};

template <int N>
struct TapArr {
  TapSpec t[N];
  int n, niso, nten;
};

// Taps are ordered by (b, dy, dx, a, dz) so that one (b, dx, dy) group is one
// shared-memory read that serves every target sublattice and every dz.
template <int N, class Pred>
constexpr TapArr<N> make_taps(int nsub, int R, Pred keep) {
  TapArr<N> r{};
  int n = 0, ni = 0, nt = 0;
  for (int b = 0; b < nsub; ++b)
    for (int dy = -R; dy <= R; ++dy)
      for (int dx = -R; dx <= R; ++dx)
        for (int a = 0; a < nsub; ++a)
          for (int dz = -R; dz <= R; ++dz) {
            const int k = keep(a, b, dx, dy, dz);  // 0: absent, 1: scalar, 2: tensor
            if (!k) continue;
            r.t[n] = TapSpec{a, b, dx, dy, dz, k == 2, k == 2 ? nt : ni};
            if (k == 2)
              ++nt;
            else
              ++ni;
            ++n;
          }
  r.n = n;
  r.niso = ni;
  r.nten = nt;
  return r;
}

struct KeepSC6 {
  int mode;
  constexpr int operator()(int, int, int dx, int dy, int dz) const {
    return dx * dx + dy * dy + dz * dz == 1 ? mode : 0;
  }
};
struct KeepSC26 {
  int mode;
  constexpr int operator()(int, int, int dx, int dy, int dz) const {
    const int d2 = dx * dx + dy * dy + dz * dz;
    return d2 == 0 ? 0 : (d2 == 1 ? mode : 1);
  }
};
// simple cubic, four distance shells (100), (110), (111), (200): the frustrated
// exchange of the hopfion calculation
struct KeepSC32 {
  constexpr int operator()(int, int, int dx, int dy, int dz) const {
    const int d2 = dx * dx + dy * dy + dz * dz;
    return (d2 >= 1 && d2 <= 4) ? 1 : 0;
  }
};
// bcc conventional cell as sublattices at (0,0,0) and (1/2,1/2,1/2): squared bond
// lengths in units of (a/2)^2 are 3, 4, 8, 11 for the first four shells
struct KeepBCC4 {
  constexpr int operator()(int a, int b, int dx, int dy, int dz) const {
    const int o = b - a;
    const int hx = 2 * dx + o, hy = 2 * dy + o, hz = 2 * dz + o;
    const int d2 = hx * hx + hy * hy + hz * hz;
    return (d2 == 3 || d2 == 4 || d2 == 8 || d2 == 11) ? 1 : 0;
  }
};

enum FamilyId {
  FAM_SC6_ISO = 0,
  FAM_SC6_TEN,
  FAM_SC26_ISO,
  FAM_SC26_TEN,
  FAM_SC32_ISO,
  FAM_BCC4,
  FAM_SC26_SHELL,
  FAM_COUNT
};

template <int ID>
struct Family;
template <>
struct Family<FAM_SC6_ISO> {
  static constexpr int NSUB = 1, R = 1, BY = 16, NTAP = 6, MINB = 2, RYF = 2, TYF = 8, MINBF = 2, SHELL = 0, TYP = 16;
  static constexpr TapArr<NTAP> L = make_taps<NTAP>(1, 1, KeepSC6{1});
};
template <>
struct Family<FAM_SC6_TEN> {
  static constexpr int NSUB = 1, R = 1, BY = 16, NTAP = 6, MINB = 2, RYF = 2, TYF = 8, MINBF = 2, SHELL = 0, TYP = 16;
  static constexpr TapArr<NTAP> L = make_taps<NTAP>(1, 1, KeepSC6{2});
};
template <>
struct Family<FAM_SC26_ISO> {
  static constexpr int NSUB = 1, R = 1, BY = 16, NTAP = 26, MINB = 2, RYF = 2, TYF = 8, MINBF = 2, SHELL = 0, TYP = 16;
  static constexpr TapArr<NTAP> L = make_taps<NTAP>(1, 1, KeepSC26{1});
};
template <>
struct Family<FAM_SC26_TEN> {
  static constexpr int NSUB = 1, R = 1, BY = 16, NTAP = 26, MINB = 2, RYF = 2, TYF = 8, MINBF = 2, SHELL = 0, TYP = 16;
  static constexpr TapArr<NTAP> L = make_taps<NTAP>(1, 1, KeepSC26{2});
};
// simple cubic 3x3x3 cube with one exchange constant per distance shell (100), (110), (111) and, on
// the in-plane nearest-neighbour bonds, the off-diagonal entries of interfacial DMI (xz, zx on x bonds,
// yz, zy on y bonds).  The field of a plane is summed by shells (push_shell26): in-plane edge and
// corner sums E and K of the plane, then J1 C + J2 E + J3 K for the outputs one plane away and
// J1 E + J2 K (+ DMI) for the outputs in the plane -- about half the arithmetic of 26 separate taps.
template <>
struct Family<FAM_SC26_SHELL> {
  static constexpr int NSUB = 1, R = 1, BY = 16, NTAP = 26, MINB = 2, RYF = 2, TYF = 8, MINBF = 2, SHELL = 1, TYP = 16;
  static constexpr TapArr<NTAP> L = make_taps<NTAP>(1, 1, KeepSC26{1});
};
template <>
struct Family<FAM_SC32_ISO> {
  static constexpr int NSUB = 1, R = 2, BY = 16, NTAP = 32, MINB = 1, RYF = 1, TYF = 16, MINBF = 1, SHELL = 0, TYP = 16;
  static constexpr TapArr<NTAP> L = make_taps<NTAP>(1, 2, KeepSC32{});
};
template <>
struct Family<FAM_BCC4> {
  static constexpr int NSUB = 2, R = 2, BY = 16, NTAP = 100, MINB = 1, RYF = 1, TYF = 16, MINBF = 1, SHELL = 0, TYP = 16;
  static constexpr TapArr<NTAP> L = make_taps<NTAP>(2, 2, KeepBCC4{});
};

constexpr int family_r(int fam) {
  return fam == FAM_BCC4 ? Family<FAM_BCC4>::R : fam == FAM_SC32_ISO ? Family<FAM_SC32_ISO>::R : Family<FAM_SC6_ISO>::R;
}
constexpr int family_by(int fam) {
  return fam == FAM_BCC4 ? Family<FAM_BCC4>::BY : fam == FAM_SC32_ISO ? Family<FAM_SC32_ISO>::BY
                                                                      : Family<FAM_SC6_ISO>::BY;
}

constexpr int kMaxIso = 104;
constexpr int kMaxTen = 8;

// Per-launch arguments (passed by value, read from the kernel-parameter bank).
struct StencilArgs {
  int nx, ny, nz, px, py, pz;
  int tz;  // output planes per CTA
  int thermal;
  int regen;  // two-pass thermal steps: 1 = the corrector regenerates the normals, the predictor does not store them
  long long nsite;
  float Jiso[kMaxIso];
  float Jt[kMaxTen][9];
  float zee[2][3], twoK[2], axis[2][3], inv_mm[2], sigma[2];
  float g, alpha, dt, hdt;
  unsigned long long seed, step;
  unsigned replica;
  int *status;      // the context's status word (numeric errors of the state update)
  PhiloxKeys keys;  // round keys of seed
};

struct GridBar;

struct StencilPlan {
  int family;
  int tz;           // z chunk of the fused Heun step (and of single-image field launches)
  int tz2;          // z chunk of the two-pass Heun passes
  int nsm;          // SMs of the device
  int occ_field;    // resident CTAs per SM of the field kernel
  int scheme;       // SX_STENCIL_FUSED or SX_STENCIL_TWO_PASS
  float *d_St;      // two-pass workspace: S~ (3 nsite floats)
  float *d_f0;      // two-pass workspace: f0 (3 nsite floats)
  float *d_eta;     // two-pass workspace: thermal normals (3 nsite floats)
  int2 *d_sched;    // balanced schedule of the two-pass kernels (nsched CTAs)
  int nsched;
  GridBar *d_bar;   // grid barrier and error word of the persistent multi-step kernel
  int persistent;   // 1: nsched CTAs of the persistent kernel fit on the device at once
  int occ_persist;  // resident CTAs per SM of the persistent kernel (0: not available)
  int sched_factor; // balanced schedule over sched_factor x the resident CTA slots (0: grid-tiled passes)
  int tma_ok;       // the lattice allows tensor-copied planes (x rows of a multiple of 16 bytes in FP32)
  int tma;          // interior tiles stage their planes with tensor copies: bit 0 predictor and field
                    // passes, bit 1 corrector
  // overlapped two-pass launch (sched_factor == kSchedOverlap): unit queue, one done flag per predictor
  // unit, queue counter; ovl_grid CTAs (0: not set up)
  int *d_order;
  int *d_done;
  int *d_queue;
  int n_order;
  int n_done;
  int ovl_grid;
  StencilArgs base;
};

constexpr int kSchedOverlap = 5;  // two-pass launch shape: one launch of overlapped predictor/corrector units

// ------------------------------------------------------------------ helpers

template <class F, int I>
struct TapAt {
  static constexpr TapSpec s = F::L.t[I];
  static constexpr TapSpec prev = F::L.t[I > 0 ? I - 1 : 0];
  static constexpr int a = s.a, b = s.b, dx = s.dx, dy = s.dy, dz = s.dz, tensor = s.tensor, coef = s.coef;
  static constexpr bool fresh = I == 0 || prev.b != b || prev.dx != dx || prev.dy != dy;
};

// ------------------------------------------------------------------ async copies

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// 8-byte global -> shared copy that zero-fills when !ok (no global read then)
__device__ __forceinline__ void cp_async8(unsigned dst, const void *src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(ok ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ------------------------------------------------------------------ geometry

// Fused-kernel geometry: a CTA of 32 x TYF threads owns a 32 x BY predictor
// region (BY = RYF * TYF rows; each thread RYF adjacent rows of one column),
// whose interior TX x TY columns are its outputs.
template <class F>
struct G {
  static constexpr int NS = F::NSUB, R = F::R, RY = F::RYF, TYT = F::TYF, BY = RY * TYT;
  static constexpr int BX = 32, NT = BX * TYT, TX = BX - 2 * R, TY = BY - 2 * R;
  static constexpr int LX = BX + 2 * R, LY = BY + 2 * R;
  static constexpr int Q = R + 1;                   // ring depth (planes)
  static constexpr int SN = NS * LY * LX;           // sites per staged S^n plane (load region)
  static constexpr int ST = NS * BY * BX;           // sites per S~ plane (predictor region)
  static constexpr int NI = TX * TY;                // interior (output) columns
  static constexpr int NLOAD = (SN + NT - 1) / NT;  // load-region sites per thread
  // shared memory: S^n ring (float4), S~ ring (float4), f0/eta ring, FP64 staging of the next plane, FP64
  // state of this iteration's corrector sites
  static constexpr size_t OFF_ST = (size_t)Q * SN * 16;
  static constexpr size_t OFF_FQ = OFF_ST + (size_t)Q * ST * 16;
  static constexpr size_t OFF_STAGE = OFF_FQ + (size_t)Q * NS * 6 * NI * 4;
  static constexpr size_t OFF_S64 = OFF_STAGE + (size_t)3 * SN * 8;
  static constexpr size_t SMEM = OFF_S64 + (size_t)NS * 3 * NI * 8;
};

// Per-thread accumulator of one output site and one dz: (x, y) packed for the
// f32x2 FMA pipe path, z alone.  Each lane of __ffma2_rn is one fused
// multiply-add, so the sums equal scalar fmaf sums taken in the same order.
struct Acc3 {
  float2 xy;
  float z;
};

// accumulate one staged plane into acc[a][R - dz] for every tap
template <class F, int I>
__device__ __forceinline__ void tap_push(const StencilArgs &p, const float4 *__restrict__ base, int pitch_sub,
                                         int pitch_row, float4 &v, Acc3 (&acc)[F::NSUB][2 * F::R + 1]) {
  using t = TapAt<F, I>;
  if constexpr (t::fresh) v = base[t::b * pitch_sub + t::dy * pitch_row + t::dx];
  Acc3 &o = acc[t::a][F::R - t::dz];
  if constexpr (t::tensor) {
    const float *J = p.Jt[t::coef];
    o.xy = __ffma2_rn(make_float2(J[2], J[5]), make_float2(v.z, v.z), o.xy);
    o.xy = __ffma2_rn(make_float2(J[1], J[4]), make_float2(v.y, v.y), o.xy);
    o.xy = __ffma2_rn(make_float2(J[0], J[3]), make_float2(v.x, v.x), o.xy);
    o.z = fmaf(J[6], v.x, fmaf(J[7], v.y, fmaf(J[8], v.z, o.z)));
  } else {
    const float J = p.Jiso[t::coef];
    o.xy = __ffma2_rn(make_float2(J, J), make_float2(v.x, v.y), o.xy);
    o.z = fmaf(J, v.z, o.z);
  }
}

template <class F, int... I>
__device__ __forceinline__ void push_all(std::integer_sequence<int, I...>, const StencilArgs &p,
                                         const float4 *__restrict__ base, int pitch_sub, int pitch_row,
                                         Acc3 (&acc)[F::NSUB][2 * F::R + 1]) {
  float4 v;
  (tap_push<F, I>(p, base, pitch_sub, pitch_row, v, acc), ...);
}

// Field of one staged plane by distance shells (FAM_SC26_SHELL): p.Jiso[0..2] = J1..J3, p.Jt[0..3] the
// in-plane nearest-neighbour bonds (dx, dy) = (-1, 0), (1, 0), (0, -1), (0, 1) (only their DMI entries
// [2], [6] (x bonds) and [5], [7] (y bonds) are read).  acc[0][0] collects the outputs one plane below
// the staged plane, acc[0][1] those in it, acc[0][2] those one plane above.
__device__ __forceinline__ void push_shell26(const StencilArgs &p, const float4 *__restrict__ base, int pitch_row,
                                             Acc3 (&acc)[1][3]) {
  const float4 c = base[0];
  const float4 w = base[-1], e = base[1];
  const float4 n = base[-pitch_row], s = base[pitch_row];
  const float4 nw = base[-pitch_row - 1], ne = base[-pitch_row + 1];
  const float4 sw = base[pitch_row - 1], se = base[pitch_row + 1];
  const float2 Exy = __fadd2_rn(__fadd2_rn(make_float2(w.x, w.y), make_float2(e.x, e.y)),
                                __fadd2_rn(make_float2(n.x, n.y), make_float2(s.x, s.y)));
  const float Ez = (w.z + e.z) + (n.z + s.z);
  const float2 Kxy = __fadd2_rn(__fadd2_rn(make_float2(nw.x, nw.y), make_float2(ne.x, ne.y)),
                                __fadd2_rn(make_float2(sw.x, sw.y), make_float2(se.x, se.y)));
  const float Kz = (nw.z + ne.z) + (sw.z + se.z);
  const float J1 = p.Jiso[0], J2 = p.Jiso[1], J3 = p.Jiso[2];
  // outputs one plane away: J1 C + J2 E + J3 K
  const float2 Txy = __ffma2_rn(make_float2(J3, J3), Kxy,
                                __ffma2_rn(make_float2(J2, J2), Exy, __fmul2_rn(make_float2(J1, J1), make_float2(c.x, c.y))));
  const float Tz = fmaf(J3, Kz, fmaf(J2, Ez, J1 * c.z));
  acc[0][0].xy = __fadd2_rn(acc[0][0].xy, Txy);
  acc[0][0].z += Tz;
  acc[0][2].xy = __fadd2_rn(acc[0][2].xy, Txy);
  acc[0][2].z += Tz;
  // outputs in the plane: J1 E + J2 K and the DMI entries of the four in-plane bonds
  float2 Mxy = __ffma2_rn(make_float2(J2, J2), Kxy, __fmul2_rn(make_float2(J1, J1), Exy));
  float Mz = fmaf(J2, Kz, J1 * Ez);
  Mxy.x = fmaf(p.Jt[1][2], e.z, fmaf(p.Jt[0][2], w.z, Mxy.x));
  Mxy.y = fmaf(p.Jt[3][5], s.z, fmaf(p.Jt[2][5], n.z, Mxy.y));
  Mz = fmaf(p.Jt[3][7], s.y, fmaf(p.Jt[2][7], n.y, fmaf(p.Jt[1][6], e.x, fmaf(p.Jt[0][6], w.x, Mz))));
  acc[0][1].xy = __fadd2_rn(acc[0][1].xy, Mxy);
  acc[0][1].z += Mz;
}

// Field of one staged plane into the accumulators: shell sums for FAM_SC26_SHELL, the tap list otherwise.
template <class F>
__device__ __forceinline__ void push_plane(const StencilArgs &p, const float4 *__restrict__ base, int pitch_sub,
                                           int pitch_row, Acc3 (&acc)[F::NSUB][2 * F::R + 1]) {
  if constexpr (F::SHELL)
    push_shell26(p, base, pitch_row, acc);
  else
    push_all<F>(std::make_integer_sequence<int, F::NTAP>{}, p, base, pitch_sub, pitch_row, acc);
}

template <class F>
__device__ __forceinline__ void zero_acc(Acc3 (&acc)[F::NSUB][2 * F::R + 1]) {
#pragma unroll
  for (int a = 0; a < F::NSUB; ++a)
#pragma unroll
    for (int j = 0; j < 2 * F::R + 1; ++j) {
      acc[a][j].xy = make_float2(0.0f, 0.0f);
      acc[a][j].z = 0.0f;
    }
}

template <class F>
__device__ __forceinline__ void shift_acc(Acc3 (&acc)[F::NSUB][2 * F::R + 1]) {
#pragma unroll
  for (int a = 0; a < F::NSUB; ++a) {
#pragma unroll
    for (int j = 0; j < 2 * F::R; ++j) acc[a][j] = acc[a][j + 1];
    acc[a][2 * F::R].xy = make_float2(0.0f, 0.0f);
    acc[a][2 * F::R].z = 0.0f;
  }
}

// Site index (within one component array; the stencil backend requires nsite < 2^32) of the
// load-region sites this thread stages, without the plane term, which is added per z step; x and
// y are wrapped once here.  A site outside an open face gets index 0 (a valid address that the
// zero-filling copy does not read).
template <int NLOAD, int NT, int SN, int LX, int LY, class GEO>
__device__ __forceinline__ void load_offsets(const GEO &p, int xs, int ys, int tid, uint32_t (&off)[NLOAD],
                                             unsigned &okmask) {
  okmask = 0u;
  const uint32_t subvol = (uint32_t)p.nz * (uint32_t)p.ny * (uint32_t)p.nx;
#pragma unroll
  for (int j = 0; j < NLOAD; ++j) {
    const int e = tid + j * NT;
    off[j] = 0;
    if (e < SN) {
      const int s = e / (LX * LY);
      const int r = e - s * (LX * LY);
      const int row = r / LX, col = r - row * LX;
      bool ok = true;
      const int gx = wrap_axis(xs + col, p.nx, p.px, ok);
      const int gy = wrap_axis(ys + row, p.ny, p.py, ok);
      off[j] = (uint32_t)s * subvol + (uint32_t)gy * (uint32_t)p.nx + (uint32_t)gx;
      if (ok) okmask |= 1u << j;
    }
  }
}

// Issue the zero-filling async copies of plane q into the FP64 staging area.
template <int NLOAD, int NT, int SN, class GEO>
__device__ __forceinline__ void issue_plane(const GEO &p, const double *__restrict__ S, int q, int tid,
                                            const uint32_t (&off)[NLOAD], unsigned okmask, double *stage) {
  bool zok = true;
  const int gz = wrap_axis(q, p.nz, p.pz, zok);
  const uint32_t zoff = (uint32_t)gz * (uint32_t)p.ny * (uint32_t)p.nx;
  const double *S1 = S + p.nsite, *S2 = S + 2 * p.nsite;
#pragma unroll
  for (int j = 0; j < NLOAD; ++j) {
    const int e = tid + j * NT;
    if (e < SN) {
      const bool ok = zok && ((okmask >> j) & 1u);
      const uint32_t i = off[j] + zoff;
      cp_async8(smem_addr(stage + e), S + i, ok);
      cp_async8(smem_addr(stage + SN + e), S1 + i, ok);
      cp_async8(smem_addr(stage + 2 * SN + e), S2 + i, ok);
    }
  }
}

// Turn this thread's staged FP64 sites into FP32 float4 (integer conversion).
template <int NLOAD, int NT, int SN>
__device__ __forceinline__ void convert_plane(const double *stage, float4 *dst, int tid) {
#pragma unroll
  for (int j = 0; j < NLOAD; ++j) {
    const int e = tid + j * NT;
    if (e < SN)
      dst[e] = make_float4(f64_to_f32(stage[e]), f64_to_f32(stage[SN + e]), f64_to_f32(stage[2 * SN + e]), 0.0f);
  }
}

__device__ __forceinline__ void onsite32(const StencilArgs &p, int a, const float s[3], float b[3]) {
  const float q = p.twoK[a] * (s[0] * p.axis[a][0] + s[1] * p.axis[a][1] + s[2] * p.axis[a][2]);
  b[0] += p.zee[a][0] + q * p.axis[a][0];
  b[1] += p.zee[a][1] + q * p.axis[a][1];
  b[2] += p.zee[a][2] + q * p.axis[a][2];
}

// ------------------------------------------------------------------ fused Heun

// One normalised Heun step from Sin to Sout.  Per z iteration k (plane q = z0 - 2R + k):
//   1. this thread's staged copy of plane q lands -> FP32 ring slot; the copies of plane q+1 and
//      of the FP64 state of the corrector sites are issued (asynchronous, no registers held);
//   2. plane q is pushed into the predictor accumulators of the thread's RY rows; the predictor of
//      plane q - R runs on the whole 32 x BY region (tile + halo) and writes S~ and, for interior
//      columns, f0 and eta;
//   3. interior rows push S~ of plane q - R into the corrector accumulators and finish the
//      corrector of plane q - 2R in FP64.
// Rows of one thread share the column's bookkeeping and, where their neighbourhoods overlap, the
// shared-memory reads of the field push; each row's tap order is that of the pass kernels.
template <int FID>
__global__ void __launch_bounds__(G<Family<FID>>::NT, Family<FID>::MINBF)
    k_heun_fused(const StencilArgs p, const double *__restrict__ Sin, double *__restrict__ Sout) {
  using F = Family<FID>;
  using g = G<F>;
  constexpr int NS = F::NSUB, R = F::R, Q = g::Q, RY = g::RY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4 *sn = reinterpret_cast<float4 *>(smem_raw);                 // [Q][SN]
  float4 *st = reinterpret_cast<float4 *>(smem_raw + g::OFF_ST);     // [Q][ST]
  float *fq = reinterpret_cast<float *>(smem_raw + g::OFF_FQ);       // [Q][NS][6][NI]
  double *stage = reinterpret_cast<double *>(smem_raw + g::OFF_STAGE);  // [3][SN]
  double *s64 = reinterpret_cast<double *>(smem_raw + g::OFF_S64);   // [NS][3][NI]

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int x0 = blockIdx.x * g::TX, y0 = blockIdx.y * g::TY, z0 = blockIdx.z * p.tz;
  const int tzc = min(p.tz, p.nz - z0);
  const int ry0 = ty * RY;                       // first region row of this thread
  const int cx = x0 - R + tx;                    // this thread's predictor column
  bool xok = true;
  const int wx = wrap_axis(cx, p.nx, p.px, xok);
  const bool xin = tx >= R && tx < 32 - R && cx < p.nx;
  const uint32_t plane = (uint32_t)p.ny * (uint32_t)p.nx, subvol = (uint32_t)p.nz * plane;
  const double *Sin1 = Sin + p.nsite, *Sin2 = Sin + 2 * p.nsite;
  double *Sout1 = Sout + p.nsite, *Sout2 = Sout + 2 * p.nsite;
  bool col_ok[RY], rin[RY], inner[RY];
  int wy[RY], cy[RY], ii[RY];
#pragma unroll
  for (int j = 0; j < RY; ++j) {
    cy[j] = y0 - R + ry0 + j;
    col_ok[j] = xok;
    wy[j] = wrap_axis(cy[j], p.ny, p.py, col_ok[j]);
    rin[j] = ry0 + j >= R && ry0 + j < g::BY - R;  // interior row (the same for the whole warp)
    inner[j] = rin[j] && xin && cy[j] < p.ny;
    ii[j] = (ry0 + j - R) * g::TX + (tx - R);      // interior index (valid when inner)
  }

  uint32_t off[g::NLOAD];
  unsigned okmask;
  load_offsets<g::NLOAD, g::NT, g::SN, g::LX, g::LY>(p, x0 - 2 * R, y0 - 2 * R, tid, off, okmask);

  Acc3 accp[RY][NS][2 * R + 1];
  Acc3 accc[RY][NS][2 * R + 1];
#pragma unroll
  for (int j = 0; j < RY; ++j) {
    zero_acc<F>(accp[j]);
    zero_acc<F>(accc[j]);
  }

  const int niter = tzc + 4 * R;
  issue_plane<g::NLOAD, g::NT, g::SN>(p, Sin, z0 - 2 * R, tid, off, okmask, stage);
  cp_commit();

  for (int k = 0; k < niter; ++k) {
    const int q = z0 - 2 * R + k;
    cp_wait<0>();
    convert_plane<g::NLOAD, g::NT, g::SN>(stage, sn + (k % Q) * g::SN, tid);
    const int kp = k - 2 * R, kc = k - 4 * R;
    const int c = z0 + kc;
    if (kc >= 0) {  // FP64 state of this iteration's corrector sites (staged 2R planes ago: L2-resident)
#pragma unroll
      for (int j = 0; j < RY; ++j) {
        if (inner[j]) {
#pragma unroll
          for (int a = 0; a < NS; ++a) {
            const uint32_t i = a * subvol + (uint32_t)c * plane + (uint32_t)cy[j] * (uint32_t)p.nx + (uint32_t)cx;
            cp_async8(smem_addr(s64 + (a * 3 + 0) * g::NI + ii[j]), Sin + i, true);
            cp_async8(smem_addr(s64 + (a * 3 + 1) * g::NI + ii[j]), Sin1 + i, true);
            cp_async8(smem_addr(s64 + (a * 3 + 2) * g::NI + ii[j]), Sin2 + i, true);
          }
        }
      }
    }
    cp_commit();
    if (k + 1 < niter) issue_plane<g::NLOAD, g::NT, g::SN>(p, Sin, q + 1, tid, off, okmask, stage);
    cp_commit();
    __syncthreads();

    // predictor field: push the staged plane q into the accumulators of every row
    {
      const float4 *base = sn + (k % Q) * g::SN + (ry0 + R) * g::LX + (tx + R);
#pragma unroll
      for (int j = 0; j < RY; ++j)
        push_plane<F>(p, base + j * g::LX, g::LX * g::LY, g::LX, accp[j]);
    }
    if (kp >= 0) {
      // predictor at plane pz = q - R for every column of the 32 x BY region
      const int pz = q - R;
      bool zok = true;
      const int wz = wrap_axis(pz, p.nz, p.pz, zok);
      const float4 *cen = sn + ((k - R) % Q) * g::SN + (ry0 + R) * g::LX + (tx + R);
      float4 *out = st + (kp % Q) * g::ST + ry0 * 32 + tx;
      float *fo = fq + (kp % Q) * (NS * 6 * g::NI);
#pragma unroll
      for (int j = 0; j < RY; ++j) {
#pragma unroll
        for (int a = 0; a < NS; ++a) {
          float4 tilde = make_float4(0.f, 0.f, 0.f, 0.f);
          if (zok && col_ok[j]) {
            const float4 c4 = cen[j * g::LX + a * g::LX * g::LY];
            const float s[3] = {c4.x, c4.y, c4.z};
            float b[3] = {accp[j][a][0].xy.x, accp[j][a][0].xy.y, accp[j][a][0].z};
            onsite32(p, a, s, b);
            float e0 = 0.f, e1 = 0.f, e2 = 0.f;
            if (p.thermal) {
              const unsigned long long site =
                  a * subvol + (uint32_t)wz * plane + (uint32_t)wy[j] * (uint32_t)p.nx + (uint32_t)wx;
              normals3(p.keys, p.replica, site, p.step, e0, e1, e2);
            }
            const float sg = p.sigma[a], im = p.inv_mm[a];
            const float B[3] = {fmaf(b[0], im, sg * e0), fmaf(b[1], im, sg * e1), fmaf(b[2], im, sg * e2)};
            float f[3];
            rhs32(s, B, p.g, p.alpha, f);
            const float x[3] = {fmaf(p.dt, f[0], s[0]), fmaf(p.dt, f[1], s[1]), fmaf(p.dt, f[2], s[2])};
            const float n2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
            float r = rsqrtf(n2);
            r = r * fmaf(-0.5f * n2, r * r, 1.5f);
            tilde = make_float4(x[0] * r, x[1] * r, x[2] * r, 0.f);
            if (inner[j]) {
              float *fa = fo + a * 6 * g::NI + ii[j];
              fa[0] = f[0];
              fa[g::NI] = f[1];
              fa[2 * g::NI] = f[2];
              fa[3 * g::NI] = e0;
              fa[4 * g::NI] = e1;
              fa[5 * g::NI] = e2;
            }
          }
          out[j * 32 + a * 32 * g::BY] = tilde;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < RY; ++j) shift_acc<F>(accp[j]);
    __syncthreads();

    if (kp >= 0) {
      // corrector field: push the S~ plane just computed (interior rows)
      const float4 *base = st + (kp % Q) * g::ST + ry0 * 32 + tx;
#pragma unroll
      for (int j = 0; j < RY; ++j)
        if (rin[j])
          push_plane<F>(p, base + j * 32, 32 * g::BY, 32, accc[j]);
      if (kc >= 0) {
        const int slot = (kc + R) % Q;
        const float4 *cen = st + slot * g::ST + ry0 * 32 + tx;
        const float *fi = fq + slot * (NS * 6 * g::NI);
        cp_wait<1>();  // this thread's FP64 state copies (all but the newest group)
#pragma unroll
        for (int j = 0; j < RY; ++j) {
          if (!inner[j]) continue;
#pragma unroll
          for (int a = 0; a < NS; ++a) {
            const float4 c4 = cen[j * 32 + a * 32 * g::BY];
            const float s[3] = {c4.x, c4.y, c4.z};
            float b[3] = {accc[j][a][0].xy.x, accc[j][a][0].xy.y, accc[j][a][0].z};
            onsite32(p, a, s, b);
            const float *fa = fi + a * 6 * g::NI + ii[j];
            const float sg = p.sigma[a], im = p.inv_mm[a];
            const float B[3] = {fmaf(b[0], im, sg * fa[3 * g::NI]), fmaf(b[1], im, sg * fa[4 * g::NI]),
                                fmaf(b[2], im, sg * fa[5 * g::NI])};
            float f[3];
            rhs32(s, B, p.g, p.alpha, f);
            const float d[3] = {p.hdt * (fa[0] + f[0]), p.hdt * (fa[g::NI] + f[1]), p.hdt * (fa[2 * g::NI] + f[2])};
            const double S0[3] = {s64[(a * 3 + 0) * g::NI + ii[j]], s64[(a * 3 + 1) * g::NI + ii[j]],
                                  s64[(a * 3 + 2) * g::NI + ii[j]]};
            double o[3];
            report_numeric(p.status, renormalise64(S0, d, o));
            const uint32_t i = a * subvol + (uint32_t)c * plane + (uint32_t)cy[j] * (uint32_t)p.nx + (uint32_t)cx;
            Sout[i] = o[0];
            Sout1[i] = o[1];
            Sout2[i] = o[2];
          }
        }
      }
#pragma unroll
      for (int j = 0; j < RY; ++j) shift_acc<F>(accc[j]);
    }
  }
  cp_wait<0>();
}

// ------------------------------------------------------------------ field only

// Pass-kernel geometry: a CTA of 32 x TYT threads owns a 32 x BY column tile, each thread RY = BY / TYT
// adjacent rows of one column.
// A tile whose load region lies inside the lattice in x and y (interior tiles) stages each plane with one
// tensor copy (TMA) of a box of LXA x LY sites x NS sublattices x 3 components: its x start is rounded
// down to 16 bytes (RA columns of halo instead of R: 2 for FP64 input, 4 for the FP32 S~ of the
// corrector) and the box lands as [component][sublattice][row][LXA].  Other tiles copy site by site.
template <class F>
struct GF {
  static constexpr int NS = F::NSUB, R = F::R, BY = F::BY, TYT = F::TYP, RY = BY / TYT;
  static_assert(RY * TYT == BY, "the tile rows must split evenly over the thread rows");
  static constexpr int NT = 32 * TYT, LX = 32 + 2 * R, LY = BY + 2 * R;
  static constexpr int SN = NS * LY * LX;
  static constexpr int NLOAD = (SN + NT - 1) / NT;
  static constexpr int RA64 = (R + 1) & ~1, LXA64 = 32 + 2 * RA64;  // FP64 box (x start even)
  static constexpr int RA32 = 4, LXA32 = 32 + 2 * RA32;             // FP32 box (x start a multiple of 4)
  static_assert(R <= RA32, "the FP32 box covers halos up to 4 columns");
  static constexpr size_t BOX64 = (size_t)3 * NS * LY * LXA64 * 8, BOX32 = (size_t)3 * NS * LY * LXA32 * 4;
  static constexpr size_t STAGE_BYTES = std::max(std::max((size_t)3 * SN * 8, BOX64), BOX32);
  static constexpr size_t OFF_CQ = 2 * (size_t)SN * 16;
  static constexpr size_t OFF_STAGE = (OFF_CQ + (size_t)(R + 1) * NS * RY * NT * 16 + 127) / 128 * 128;
  static constexpr size_t OFF_MBAR = (OFF_STAGE + STAGE_BYTES + 15) / 16 * 16;  // mbarrier, abort word
  static constexpr size_t SMEM = OFF_MBAR + 16;
};

// One plane-marching pass over 32 x BY output columns: the field of an input
// spin field plus an epilogue per output site.
//  PASS_FIELD: b = field (+ Zeeman and anisotropy when onsite), FP64 out;
//  PASS_PRED:  Heun predictor from S^n (FP64 in): f0 = f(S^n, B), S~ = N[S^n + dt f0],
//              S~ and f0 written as FP32 planes;
//  PASS_CORR:  Heun corrector from S~ (FP32 in): f1 = f(S~, B~),
//              S^{n+1} = N[S^n + dt/2 (f0 + f1)] in FP64 (S^n, f0 and, for a
//              thermal step, the predictor's normals read at the site).
// PASS_PRED followed by PASS_CORR is the two-pass form of the fused Heun step:
// the same FP32 field sums in the same order, the same noise, the same FP64
// renormalisation.
enum PassMode { PASS_FIELD = 0, PASS_PRED = 1, PASS_CORR = 2 };

struct PassIO {
  const double *S;   // FIELD, PRED: input spins; CORR: the FP64 state S^n
  const float *St;   // CORR: S~ (three FP32 planes)
  double *b;         // FIELD: output field (FP64)
  float *bf;         // FIELD: output field in FP32 instead, when set
  float *St_out;     // PRED: S~
  float *f0;         // PRED: written; CORR: read
  float *eta;        // thermal steps: the normals, written by PRED and read by CORR
  double *Sout;      // CORR: S^{n+1}
  int nzc;           // z chunks per image (blockIdx.z = image * nzc + chunk)
  long long istride; // doubles between images (FIELD)
  unsigned long long step;  // noise counter of the step (PRED)
  const int2 *sched; // balanced schedule (one image): CTA k owns column-plane units
                     // [sched[k].x, sched[k].x + sched[k].y) of u = column * nz + z; null: the grid tiles
  int tma;           // 1: interior tiles stage planes with the launch's tensor map (k_stencil_pass only)
  int *werr;         // set when a bounded wait on a tensor copy gives up
  int zc0;           // k_stencil_pass on the grid: first z chunk of the launch (chunk zc0 + blockIdx.z)
};

// ------------------------------------------------------------------ tensor copies of the pass kernels

__device__ __forceinline__ void tma_plane(const CUtensorMap *tm, void *dst, uint64_t *mbar, uint32_t bytes, int x,
                                          int y, int z) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier generic accesses of dst come first
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(0), "r"(0), "r"(smem_addr(mbar))
      : "memory");
}

// Wait for phase `parity` of the plane barrier, about a second at most; a thread whose wait gives up (or
// finds that another one did) sets the CTA's abort word and the error word and returns false.
__device__ __forceinline__ bool tma_wait(uint64_t *mbar, uint32_t parity, volatile int *abort, int *werr) {
  for (long it = 0; it < (1L << 24); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (*abort) return false;
    if (it > 1024) __nanosleep(64);
  }
  *abort = 1;
  if (werr) atomicExch(werr, 1);
  return false;
}

__device__ __forceinline__ void cp_async4(unsigned dst, const void *src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(ok ? 4 : 0) : "memory");
}

// FP32 planes of S~ straight into the float4 ring (4-byte zero-filling copies)
template <int NLOAD, int NT, int SN, class GEO>
__device__ __forceinline__ void issue_plane_f32(const GEO &p, const float *__restrict__ S, int q, int tid,
                                                const uint32_t (&off)[NLOAD], unsigned okmask, float4 *dst) {
  bool zok = true;
  const int gz = wrap_axis(q, p.nz, p.pz, zok);
  const uint32_t zoff = (uint32_t)gz * (uint32_t)p.ny * (uint32_t)p.nx;
  const float *S1 = S + p.nsite, *S2 = S + 2 * p.nsite;
#pragma unroll
  for (int j = 0; j < NLOAD; ++j) {
    const int e = tid + j * NT;
    if (e < SN) {
      const bool ok = zok && ((okmask >> j) & 1u);
      const uint32_t i = off[j] + zoff;
      const unsigned d = smem_addr(dst + e);
      cp_async4(d, S + i, ok);
      cp_async4(d + 4, S1 + i, ok);
      cp_async4(d + 8, S2 + i, ok);
    }
  }
}

// One segment: the output columns of the 32 x BY tile at (x0, y0), planes z0 .. z0 + tzc - 1,
// of image img.  p carries the couplings and constants, gg the lattice geometry (nx .. pz,
// nsite) and the noise replica index: the launch arguments themselves for one system, a
// per-replica record in a batch.
// TMAP: compiled with the tensor-copy staging (otherwise every tile copies site by site and tm is
// ignored); tm: the launch's tensor map over the input planes (S, or S~ for PASS_CORR), or null;
// tphase: the parity of the CTA's next plane-barrier phase (advanced by every tensor-copied plane).
template <int FID, int MODE, bool TMAP = false, class GEO>
__device__ __forceinline__ void pass_segment(const StencilArgs &p, const GEO &gg, int onsite, const PassIO &io,
                                             unsigned char *smem_raw, int img, int x0, int y0, int z0, int tzc,
                                             const CUtensorMap *tm, uint32_t &tphase) {
  using F = Family<FID>;
  using g = GF<F>;
  constexpr int NS = F::NSUB, R = F::R, RY = g::RY;
  float4 *sn = reinterpret_cast<float4 *>(smem_raw);                    // [2][SN]
  float4 *cq = reinterpret_cast<float4 *>(smem_raw + g::OFF_CQ);        // [R+1][NS][RY][NT] centre values
  double *stage = reinterpret_cast<double *>(smem_raw + g::OFF_STAGE);  // [3][SN] (FP64 input) or a tensor box
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw + g::OFF_MBAR);
  volatile int *abort = reinterpret_cast<volatile int *>(smem_raw + g::OFF_MBAR + 8);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  // tensor-copied planes: the box starts RA columns left of the tile (RA >= R, 16-byte aligned)
  constexpr bool F32IN = MODE == PASS_CORR;
  constexpr int RA = F32IN ? g::RA32 : g::RA64, LXA = F32IN ? g::LXA32 : g::LXA64;
  constexpr int CS = NS * g::LY * LXA;  // elements per component in the box
  constexpr uint32_t BOX_BYTES = (uint32_t)(F32IN ? g::BOX32 : g::BOX64);
  const bool tma = TMAP && tm && x0 >= RA && x0 + 32 + RA <= gg.nx && y0 >= R && y0 + F::BY + R <= gg.ny;
  int sidx[g::NLOAD];  // box element of this thread's load-region sites
  if constexpr (TMAP) {
#pragma unroll
    for (int j = 0; j < g::NLOAD; ++j) {
      const int e = tid + j * g::NT;
      const int a = e / (g::LX * g::LY), r = e - a * (g::LX * g::LY), ly = r / g::LX, lx = r - ly * g::LX;
      sidx[j] = (a * g::LY + ly) * LXA + lx + (RA - R);
    }
  }
  auto tma_issue = [&](int q) {
    if (tid == 0 && !*abort) {
      bool zok = true;  // open z faces: out-of-range planes are read as zeros by the copy itself
      const int gz = gg.pz ? wrap_axis(q, gg.nz, 1, zok) : q;
      tma_plane(tm, stage, mbar, BOX_BYTES, x0 - RA, y0 - R, gz);
    }
  };
  const int ry0 = ty * RY;  // first tile row of this thread
  const double *Sin = io.S + img * io.istride;
  double *bout = io.b + img * io.istride;
  const int cx = x0 + tx;
  const uint32_t plane = (uint32_t)gg.ny * (uint32_t)gg.nx, subvol = (uint32_t)gg.nz * plane;
  bool mine[RY];
  uint32_t icol[RY];  // this thread's columns in a plane
#pragma unroll
  for (int j = 0; j < RY; ++j) {
    const int cy = y0 + ry0 + j;
    mine[j] = cx < gg.nx && cy < gg.ny;
    icol[j] = (uint32_t)cy * (uint32_t)gg.nx + (uint32_t)cx;
  }
  const long long N = gg.nsite;
  Acc3 acc[RY][NS][2 * R + 1];
#pragma unroll
  for (int j = 0; j < RY; ++j) zero_acc<F>(acc[j]);
  uint32_t off[g::NLOAD];
  unsigned okmask;
  load_offsets<g::NLOAD, g::NT, g::SN, g::LX, g::LY>(gg, x0 - R, y0 - R, tid, off, okmask);
  const int niter = tzc + 2 * R;
  // corrector: S^n and f0 of the next output plane, loaded one plane ahead so the
  // global-load latency hides behind a plane of field work
  double nS[RY][NS][3];
  float nf[RY][NS][3], ne[RY][NS][3];
  auto prefetch = [&](int cz) {
    if constexpr (MODE == PASS_CORR) {
      if (cz < z0 + tzc) {
#pragma unroll
        for (int j = 0; j < RY; ++j) {
          if (!mine[j]) continue;
#pragma unroll
          for (int a = 0; a < NS; ++a) {
            const uint32_t i = a * subvol + (uint32_t)cz * plane + icol[j];
#pragma unroll
            for (int m = 0; m < 3; ++m) {
              nS[j][a][m] = (io.S + m * N)[i];
              nf[j][a][m] = (io.f0 + m * N)[i];
              ne[j][a][m] = (p.thermal && !p.regen) ? (io.eta + m * N)[i] : 0.0f;
            }
          }
        }
      }
    }
  };
  prefetch(z0);
  if (tma)
    tma_issue(z0 - R);
  else if constexpr (MODE == PASS_CORR)
    issue_plane_f32<g::NLOAD, g::NT, g::SN>(gg, io.St, z0 - R, tid, off, okmask, sn);
  else
    issue_plane<g::NLOAD, g::NT, g::SN>(gg, Sin, z0 - R, tid, off, okmask, stage);
  cp_commit();
  for (int k = 0; k < niter; ++k) {
    const int q = z0 - R + k;
    float4 *buf = sn + (k & 1) * g::SN;
    if (TMAP && tma) {
      // the box of plane q has landed: this thread's sites into the FP32 ring (the same values, and for
      // FP64 input the same integer conversion, as the site-by-site copies)
      tma_wait(mbar, tphase, abort, io.werr);
      tphase ^= 1u;
#pragma unroll
      for (int j = 0; j < g::NLOAD; ++j) {
        const int e = tid + j * g::NT;
        if (e < g::SN) {
          if constexpr (F32IN) {
            const float *sf = reinterpret_cast<const float *>(stage);
            buf[e] = make_float4(sf[sidx[j]], sf[CS + sidx[j]], sf[2 * CS + sidx[j]], 0.0f);
          } else {
            buf[e] = make_float4(f64_to_f32(stage[sidx[j]]), f64_to_f32(stage[CS + sidx[j]]),
                                 f64_to_f32(stage[2 * CS + sidx[j]]), 0.0f);
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // these reads before the next copy's writes
      __syncthreads();  // every site of plane q is in the ring and the box is free again
      if (k + 1 < niter) tma_issue(q + 1);
    } else if constexpr (MODE == PASS_CORR) {
      cp_wait<0>();
      __syncthreads();  // every thread's copies of plane q have landed
      if (k + 1 < niter)
        issue_plane_f32<g::NLOAD, g::NT, g::SN>(gg, io.St, q + 1, tid, off, okmask, sn + ((k + 1) & 1) * g::SN);
    } else {
      cp_wait<0>();
      convert_plane<g::NLOAD, g::NT, g::SN>(stage, buf, tid);
      if (k + 1 < niter) issue_plane<g::NLOAD, g::NT, g::SN>(gg, Sin, q + 1, tid, off, okmask, stage);
    }
    cp_commit();
    if (MODE != PASS_CORR && !tma) __syncthreads();
    const float4 *base = buf + (ry0 + R) * g::LX + (tx + R);
#pragma unroll
    for (int j = 0; j < RY; ++j) push_plane<F>(p, base + j * g::LX, g::LX * g::LY, g::LX, acc[j]);
    // keep this plane's centre values for the epilogue R planes later
#pragma unroll
    for (int j = 0; j < RY; ++j)
#pragma unroll
      for (int a = 0; a < NS; ++a)
        cq[(((k % (R + 1)) * NS + a) * RY + j) * g::NT + tid] = base[j * g::LX + a * g::LX * g::LY];
    const int kc = k - 2 * R;
    if (kc >= 0) {
      const int c = z0 + kc;
#pragma unroll
      for (int j = 0; j < RY; ++j) {
        if (!mine[j]) continue;
#pragma unroll
        for (int a = 0; a < NS; ++a) {
          float v[3] = {acc[j][a][0].xy.x, acc[j][a][0].xy.y, acc[j][a][0].z};
          const float4 c4 = cq[((((k - R) % (R + 1)) * NS + a) * RY + j) * g::NT + tid];
          const float s[3] = {c4.x, c4.y, c4.z};
          const uint32_t i = a * subvol + (uint32_t)c * plane + icol[j];
          if constexpr (MODE == PASS_FIELD) {
            if (onsite) onsite32(p, a, s, v);
            if (io.bf) {
              io.bf[i] = v[0];
              (io.bf + N)[i] = v[1];
              (io.bf + 2 * N)[i] = v[2];
            } else {
              bout[i] = (double)v[0];
              (bout + N)[i] = (double)v[1];
              (bout + 2 * N)[i] = (double)v[2];
            }
          } else {
            onsite32(p, a, s, v);
            float e0 = 0.f, e1 = 0.f, e2 = 0.f;
            if constexpr (MODE == PASS_PRED) {
              if (p.thermal) {
                normals3(p.keys, gg.replica, (unsigned long long)i, io.step, e0, e1, e2);
                if (!p.regen) {
                  io.eta[i] = e0;
                  (io.eta + N)[i] = e1;
                  (io.eta + 2 * N)[i] = e2;
                }
              }
            } else if (p.thermal && p.regen) {
              // the same counter-based normals as the predictor's (a pure function of seed, replica, site, step)
              normals3(p.keys, gg.replica, (unsigned long long)i, io.step, e0, e1, e2);
            } else {
              e0 = ne[j][a][0];
              e1 = ne[j][a][1];
              e2 = ne[j][a][2];
            }
            const float sg = p.sigma[a], im = p.inv_mm[a];
            const float B[3] = {fmaf(v[0], im, sg * e0), fmaf(v[1], im, sg * e1), fmaf(v[2], im, sg * e2)};
            float f[3];
            rhs32(s, B, p.g, p.alpha, f);
            if constexpr (MODE == PASS_PRED) {
              const float x[3] = {fmaf(p.dt, f[0], s[0]), fmaf(p.dt, f[1], s[1]), fmaf(p.dt, f[2], s[2])};
              const float n2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
              float r = rsqrtf(n2);
              r = r * fmaf(-0.5f * n2, r * r, 1.5f);
              io.St_out[i] = x[0] * r;
              (io.St_out + N)[i] = x[1] * r;
              (io.St_out + 2 * N)[i] = x[2] * r;
              io.f0[i] = f[0];
              (io.f0 + N)[i] = f[1];
              (io.f0 + 2 * N)[i] = f[2];
            } else {
              const float d[3] = {p.hdt * (nf[j][a][0] + f[0]), p.hdt * (nf[j][a][1] + f[1]),
                                  p.hdt * (nf[j][a][2] + f[2])};
              double o[3];
              report_numeric(p.status, renormalise64(nS[j][a], d, o));
              io.Sout[i] = o[0];
              (io.Sout + N)[i] = o[1];
              (io.Sout + 2 * N)[i] = o[2];
            }
          }
        }
      }
      prefetch(c + 1);
    }
#pragma unroll
    for (int j = 0; j < RY; ++j) shift_acc<F>(acc[j]);
    // One barrier per plane suffices: the ring slot that iteration k + 1 refills (FP32 conversion of
    // FIELD / PRED, or the S~ copies of CORR issued after that iteration's barrier) was last read in
    // iteration k - 1, which every thread finished before arriving at iteration k's barrier; the
    // staging area and the centre ring are written and read by one thread only.
  }
  cp_wait<0>();
}

// The column-plane units of schedule entry k, segment by segment.
template <int FID, int MODE, bool TMAP = false>
__device__ __forceinline__ void run_scheduled(const StencilArgs &p, int onsite, const PassIO &io,
                                              unsigned char *smem_raw, int k, const CUtensorMap *tm,
                                              uint32_t &tphase) {
  using F = Family<FID>;
  const int2 e = io.sched[k];
  const int ncx = (p.nx + 31) / 32;
  long long u = e.x;
  const long long uend = (long long)e.x + e.y;
  while (u < uend) {  // uniform over the block
    const int col = (int)(u / p.nz), z = (int)(u - (long long)col * p.nz);
    const int len = (int)min((long long)(p.nz - z), uend - u);
    pass_segment<FID, MODE, TMAP>(p, p, onsite, io, smem_raw, 0, (col % ncx) * 32, (col / ncx) * F::BY, z, len,
                                  tm, tphase);
    u += len;
    __syncthreads();  // shared memory is reused by the next segment
  }
}

// TMAP: the instantiation with tensor-copied planes (io.tma set); the other one is the site-by-site
// staging alone, so that the extra registers of the copy path never weigh on it.
template <int FID, int MODE, bool TMAP>
__global__ void __launch_bounds__(GF<Family<FID>>::NT, Family<FID>::MINB)
    k_stencil_pass(const StencilArgs p, int onsite, const PassIO io, const __grid_constant__ CUtensorMap tmap) {
  using F = Family<FID>;
  using g = GF<F>;
  extern __shared__ __align__(128) unsigned char smem_pass[];  // the box of a tensor copy starts 128-byte aligned
  unsigned char *smem_raw = smem_pass;
  const CUtensorMap *tm = TMAP && io.tma ? &tmap : nullptr;
  uint32_t tphase = 0;
  if (TMAP && tm) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(smem_raw + g::OFF_MBAR)));
      *reinterpret_cast<volatile int *>(smem_raw + g::OFF_MBAR + 8) = 0;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
  }
  if (io.sched) {
    run_scheduled<FID, MODE, TMAP>(p, onsite, io, smem_raw, blockIdx.x, tm, tphase);
  } else {
    const int img = blockIdx.z / io.nzc, zc = blockIdx.z - img * io.nzc;
    const int z0 = (io.zc0 + zc) * p.tz;
    pass_segment<FID, MODE, TMAP>(p, p, onsite, io, smem_raw, img, blockIdx.x * 32, blockIdx.y * F::BY, z0,
                                  min(p.tz, p.nz - z0), tm, tphase);
  }
}

// Grid-wide barrier of a cooperative launch (all CTAs resident): arrive on a
// counter, the last arrival resets it and advances the generation; the others
// wait for the generation to change.  The wait is bounded: after about two
// seconds it sets the error word and gives up, and every CTA then leaves the
// step loop at its next barrier.  Returns false once the error word is set.
struct GridBar {
  unsigned count;
  unsigned gen;
  int err;
  int pad;
};

__device__ __forceinline__ bool grid_sync(GridBar *gb, unsigned nblocks) {
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    volatile unsigned *vgen = &gb->gen;
    const unsigned g = *vgen;
    __threadfence();
    if (atomicAdd(&gb->count, 1u) == nblocks - 1) {
      atomicExch(&gb->count, 0u);
      __threadfence();
      atomicAdd(&gb->gen, 1u);
    } else {
      for (long it = 0; *vgen == g; ++it) {
        if (it > (1L << 25)) {
          atomicExch(&gb->err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int *)&gb->err == 0;
}

// nsteps two-pass Heun steps in one cooperative launch (lattices with few tile
// columns, where per-step launches would dominate): step k runs the predictor
// over every CTA's scheduled units, a grid barrier, the corrector, a barrier.
// The state alternates between S0 and S1 (step k reads S_{k mod 2}).  Same
// per-site arithmetic as the separate pass launches, so bit-identical to them.
template <int FID>
__global__ void __launch_bounds__(GF<Family<FID>>::NT, Family<FID>::MINB)
    k_heun_persistent(const StencilArgs p, PassIO io, double *S0, double *S1, int nsteps,
                      unsigned long long step0, GridBar *gb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t tph = 0;  // unused: the persistent launch copies site by site
  for (int k = 0; k < nsteps; ++k) {
    io.S = (k & 1) ? S1 : S0;
    io.Sout = (k & 1) ? S0 : S1;
    io.step = step0 + (unsigned long long)k;
    run_scheduled<FID, PASS_PRED>(p, 1, io, smem_raw, blockIdx.x, nullptr, tph);
    if (!grid_sync(gb, gridDim.x)) return;
    run_scheduled<FID, PASS_CORR>(p, 1, io, smem_raw, blockIdx.x, nullptr, tph);
    if (!grid_sync(gb, gridDim.x)) return;
  }
}

// ------------------------------------------------------------------ overlapped two-pass step

// Codes of the overlapped step's work units (sx_schedule.h): idx = chunk * ncol + column (column =
// cy * ncx + cx of the 32 x BY tiles, chunk = z / tz), plus kUnitCorr for a corrector unit.
using sched::kUnitCorr;

// One two-pass Heun step in a single launch whose CTAs take predictor and corrector units from a queue
// (`order`, built on the host): the predictor is issue-bound and the corrector bound by DRAM and the
// FP64 pipe, so a predictor and a corrector unit resident on one SM share its resources better than
// two passes that each fill the whole device.  A corrector unit (chunk z, column c) reads S~ on its
// halo: it starts once the predictor units of the 3 x 3 neighbouring columns in chunks z - 1 .. z + 1
// (wrapped on periodic axes, absent beyond open faces) have published their done flags; the queue puts
// every corrector unit after those units, so a wait only ever waits for running predictor units, which
// wait for nothing.  Publication: the unit's stores, a CTA barrier, a device fence, the flag; the
// reader: the flag, a device fence, a CTA barrier, the loads.  Each flag wait gives up after about
// two seconds (error word set).  Per-site arithmetic is that of the two pass launches.
template <int FID, bool TMAP>
__global__ void __launch_bounds__(GF<Family<FID>>::NT, Family<FID>::MINB)
    k_heun_overlap(const StencilArgs p, const PassIO io, const int *__restrict__ order, int nunits, int *queue,
                   int *done, const __grid_constant__ CUtensorMap tm_pred, const __grid_constant__ CUtensorMap tm_corr,
                   int tma_pred, int tma_corr) {
  using F = Family<FID>;
  using g = GF<F>;
  extern __shared__ __align__(128) unsigned char smem_ovl[];
  unsigned char *smem_raw = smem_ovl;
  volatile int *abort = reinterpret_cast<volatile int *>(smem_raw + g::OFF_MBAR + 8);
  volatile int *s_unit = reinterpret_cast<volatile int *>(smem_raw + g::OFF_MBAR + 12);
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(smem_raw + g::OFF_MBAR)));
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t tphase = 0;
  const int ncx = (p.nx + 31) / 32, ncy = (p.ny + F::BY - 1) / F::BY, ncol = ncx * ncy;
  const int nchunk = (p.nz + p.tz - 1) / p.tz;
  for (;;) {
    if (tid == 0) {
      const int i = atomicAdd(queue, 1);
      *s_unit = i < nunits ? order[i] : -1;
    }
    __syncthreads();
    const int code = *s_unit;
    __syncthreads();  // s_unit is rewritten only after every thread has read it
    if (code < 0) break;
    const int idx = code & (kUnitCorr - 1), z = idx / ncol, col = idx - z * ncol;
    const int cx = col % ncx, cy = col / ncx, z0 = z * p.tz, len = min(p.tz, p.nz - z0);
    if (code & kUnitCorr) {
      if (tid < 27) {
        bool ok = true;
        const int zz = wrap_axis(z + tid / 9 - 1, nchunk, p.pz, ok);
        const int yy = wrap_axis(cy + (tid / 3) % 3 - 1, ncy, p.py, ok);
        const int xx = wrap_axis(cx + tid % 3 - 1, ncx, p.px, ok);
        if (ok) {
          volatile int *f = done + (long long)zz * ncol + yy * ncx + xx;
          for (long it = 0; *f == 0; ++it) {
            if (*abort || it > (1L << 24)) {
              *abort = 1;
              if (io.werr) atomicExch(io.werr, 1);
              break;
            }
            if (it > 32) __nanosleep(128);
          }
          __threadfence();
        }
      }
      __syncthreads();
      pass_segment<FID, PASS_CORR, TMAP>(p, p, 1, io, smem_raw, 0, cx * 32, cy * F::BY, z0, len,
                                         TMAP && tma_corr ? &tm_corr : nullptr, tphase);
    } else {
      pass_segment<FID, PASS_PRED, TMAP>(p, p, 1, io, smem_raw, 0, cx * 32, cy * F::BY, z0, len,
                                         TMAP && tma_pred ? &tm_pred : nullptr, tphase);
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        *reinterpret_cast<volatile int *>(done + idx) = 1;
      }
    }
    __syncthreads();  // shared memory is reused by the next unit
  }
}

// ------------------------------------------------------------------ batches of replicas

// One unit owner of a batch: a replica (Heun step) or an image of a chain (field only), with its
// geometry, its noise replica index, the first global column-plane unit it owns, its state
// (replicas: S and Sout, swapped on odd steps of a multi-step run) and two-pass workspace, or its
// field output (images).
struct SGeo {
  int nx, ny, nz, px, py, pz;
  long long nsite;
  unsigned replica;
};
struct BatchRep {
  SGeo g;
  long long u0;
  const double *S;
  double *Sout;
  float *St, *f0, *eta;
  double *b;  // images: field output (FP64, on-site terms included)
  int kind;   // 0: replica, 1: image
  int pad;
};

// The units [e.x, e.x + e.y) of one schedule entry, which may span owners (units are owner-major;
// within an owner u = column * nz + z).  Replicas run MODE with the state roles swapped when
// parity is 1; images run the field pass in the predictor phase when `images` is set and are
// skipped otherwise.
template <int FID, int MODE>
__device__ __forceinline__ void batch_units(const StencilArgs &p, const BatchRep *__restrict__ reps, int nrep,
                                            int2 e, unsigned long long step, int parity, bool images,
                                            unsigned char *smem_raw) {
  using F = Family<FID>;
  long long u = e.x;
  const long long uend = (long long)e.x + e.y;
  int lo = 0, hi = nrep - 1;  // last owner with u0 <= u
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (reps[mid].u0 <= u)
      lo = mid;
    else
      hi = mid - 1;
  }
  int r = lo;
  while (u < uend) {  // uniform over the block
    while (r + 1 < nrep && reps[r + 1].u0 <= u) ++r;
    const SGeo gg = reps[r].g;
    const long long ul = u - reps[r].u0;
    const int ncx = (gg.nx + 31) / 32;
    const int col = (int)(ul / gg.nz), z = (int)(ul - (long long)col * gg.nz);
    const int len = (int)min((long long)(gg.nz - z), uend - u);
    PassIO io;
    uint32_t tph = 0;  // unused: batch segments copy site by site
    io.nzc = 1;
    io.istride = 0;
    io.step = step;
    io.tma = 0;
    io.werr = nullptr;
    io.zc0 = 0;
    io.sched = nullptr;
    io.bf = nullptr;
    if (reps[r].kind == 0) {
      io.S = parity ? reps[r].Sout : reps[r].S;
      io.Sout = parity ? const_cast<double *>(reps[r].S) : reps[r].Sout;
      io.St = reps[r].St;
      io.St_out = reps[r].St;
      io.b = nullptr;
      io.f0 = reps[r].f0;
      io.eta = reps[r].eta;
      pass_segment<FID, MODE>(p, gg, 1, io, smem_raw, 0, (col % ncx) * 32, (col / ncx) * F::BY, z, len, nullptr,
                              tph);
    } else if (MODE == PASS_PRED && images) {
      io.S = reps[r].S;
      io.Sout = nullptr;
      io.St = nullptr;
      io.St_out = nullptr;
      io.b = reps[r].b;
      io.f0 = nullptr;
      io.eta = nullptr;
      pass_segment<FID, PASS_FIELD>(p, gg, 1, io, smem_raw, 0, (col % ncx) * 32, (col / ncx) * F::BY, z, len,
                                    nullptr, tph);
    }
    u += len;
    __syncthreads();  // shared memory is reused by the next segment
  }
}

// One two-pass stage over a batch of owners that share the couplings in p: CTA k walks the
// global column-plane units of schedule entry k.
template <int FID, int MODE>
__global__ void __launch_bounds__(GF<Family<FID>>::NT, Family<FID>::MINB)
    k_batch_pass(const StencilArgs p, const BatchRep *__restrict__ reps, int nrep, const int2 *__restrict__ sched,
                 unsigned long long step, int parity, int images) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  batch_units<FID, MODE>(p, reps, nrep, sched[blockIdx.x], step, parity, images != 0, smem_raw);
}

// nsteps Heun steps of every replica and the field of every image in one cooperative launch:
// step k runs the predictor units of all replicas (plus, at k = 0, the field units of all
// images), a grid barrier, the corrector units, a grid barrier.  Replica states alternate
// S -> Sout -> S ...  Same per-site arithmetic as the separate launches, so bit-identical to them.
// Two schedules over the same owner list: `sched_all` (replicas and images) for the first
// predictor phase, `sched_rep` (replicas only, whose units come first) for every other phase, each
// balanced on its own; a CTA past the end of a schedule idles through that phase.
template <int FID>
__global__ void __launch_bounds__(GF<Family<FID>>::NT, Family<FID>::MINB)
    k_batch_persistent(const StencilArgs p, const BatchRep *__restrict__ reps, int nown,
                       const int2 *__restrict__ sched_all, int nall, const int2 *__restrict__ sched_rep, int nrsch,
                       unsigned long long step0, int nsteps, GridBar *gb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 none = make_int2(0, 0);
  const int2 ea = (int)blockIdx.x < nall ? sched_all[blockIdx.x] : none;
  const int2 er = (int)blockIdx.x < nrsch ? sched_rep[blockIdx.x] : none;
  for (int k = 0; k < nsteps; ++k) {
    batch_units<FID, PASS_PRED>(p, reps, nown, k == 0 ? ea : er, step0 + (unsigned long long)k, k & 1, k == 0,
                                smem_raw);
    if (!grid_sync(gb, gridDim.x)) return;
    batch_units<FID, PASS_CORR>(p, reps, nown, er, step0 + (unsigned long long)k, k & 1, false, smem_raw);
    if (!grid_sync(gb, gridDim.x)) return;
  }
}

// ------------------------------------------------------------------ planning

namespace {

// FAM_SC26_SHELL: taps inside the 3x3x3 cube, each distance shell complete (6, 12, 8 taps) or absent,
// diagonal J equal within a shell, off-diagonal entries only the interfacial-DMI ones of the in-plane
// nearest-neighbour bonds.  An absent shell gets J = 0.
bool match_shell26(const sx_ctx *c, StencilArgs &a) {
  if (c->lat.nsub != 1) return false;
  for (int k = 0; k < kMaxIso; ++k) a.Jiso[k] = 0.0f;
  for (int k = 0; k < kMaxTen; ++k)
    for (int m = 0; m < 9; ++m) a.Jt[k][m] = 0.0f;
  double Js[3] = {0.0, 0.0, 0.0};
  int count[3] = {0, 0, 0};
  for (const Tap &t : c->taps[0]) {
    const int dx = t.d[0], dy = t.d[1], dz = t.d[2];
    if (t.b != 0 || dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1) return false;
    const int d2 = dx * dx + dy * dy + dz * dz;
    if (d2 == 0) return false;
    if (t.J[0] != t.J[4] || t.J[4] != t.J[8]) return false;
    if (count[d2 - 1] > 0 && Js[d2 - 1] != t.J[0]) return false;
    Js[d2 - 1] = t.J[0];
    ++count[d2 - 1];
    // permitted off-diagonal entries: xz, zx on (+-1, 0, 0); yz, zy on (0, +-1, 0)
    bool allow[9] = {false, false, false, false, false, false, false, false, false};
    int slot = -1;
    if (d2 == 1 && dz == 0) {
      if (dy == 0) {
        allow[2] = allow[6] = true;
        slot = dx < 0 ? 0 : 1;
      } else {
        allow[5] = allow[7] = true;
        slot = dy < 0 ? 2 : 3;
      }
    }
    for (int m : {1, 2, 3, 5, 6, 7})
      if (!allow[m] && t.J[m] != 0.0) return false;
    if (slot >= 0)
      for (int m = 0; m < 9; ++m) a.Jt[slot][m] = m == 0 || m == 4 || m == 8 ? 0.0f : (float)t.J[m];
  }
  const int full[3] = {6, 12, 8};
  for (int k = 0; k < 3; ++k)
    if (count[k] != 0 && count[k] != full[k]) return false;
  if (count[1] == 0 && count[2] == 0) return false;  // nearest neighbours only: the SC6 families are cheaper
  for (int k = 0; k < 3; ++k) a.Jiso[k] = (float)Js[k];
  return true;
}

template <int FID>
bool match_family(const sx_ctx *c, StencilArgs &a) {
  using F = Family<FID>;
  if (c->lat.nsub != F::NSUB) return false;
  for (int k = 0; k < kMaxIso; ++k) a.Jiso[k] = 0.0f;
  for (int k = 0; k < kMaxTen; ++k)
    for (int m = 0; m < 9; ++m) a.Jt[k][m] = 0.0f;
  for (int s = 0; s < F::NSUB; ++s) {
    for (const Tap &t : c->taps[s]) {
      int hit = -1;
      for (int i = 0; i < F::L.n; ++i) {
        const TapSpec &f = F::L.t[i];
        if (f.a == s && f.b == t.b && f.dx == t.d[0] && f.dy == t.d[1] && f.dz == t.d[2]) {
          hit = i;
          break;
        }
      }
      if (hit < 0) return false;
      const TapSpec &f = F::L.t[hit];
      const bool iso = t.J[1] == 0.0 && t.J[2] == 0.0 && t.J[3] == 0.0 && t.J[5] == 0.0 && t.J[6] == 0.0 &&
                       t.J[7] == 0.0 && t.J[0] == t.J[4] && t.J[4] == t.J[8];
      if (f.tensor) {
        for (int m = 0; m < 9; ++m) a.Jt[f.coef][m] = (float)t.J[m];
      } else {
        if (!iso) return false;
        a.Jiso[f.coef] = (float)t.J[0];
      }
    }
  }
  return true;
}

template <int FID>
cudaError_t set_smem() {
  cudaError_t e = cudaFuncSetAttribute(k_heun_fused<FID>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)G<Family<FID>>::SMEM);
  if (e != cudaSuccess) return e;
  for (auto fn : {k_stencil_pass<FID, PASS_FIELD, false>, k_stencil_pass<FID, PASS_PRED, false>,
                  k_stencil_pass<FID, PASS_CORR, false>, k_stencil_pass<FID, PASS_FIELD, true>,
                  k_stencil_pass<FID, PASS_PRED, true>, k_stencil_pass<FID, PASS_CORR, true>}) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GF<Family<FID>>::SMEM);
    if (e != cudaSuccess) return e;
  }
  for (auto fn : {k_batch_pass<FID, PASS_PRED>, k_batch_pass<FID, PASS_CORR>}) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GF<Family<FID>>::SMEM);
    if (e != cudaSuccess) return e;
  }
  e = cudaFuncSetAttribute(k_batch_persistent<FID>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)GF<Family<FID>>::SMEM);
  if (e != cudaSuccess) return e;
  for (auto fn : {k_heun_overlap<FID, false>, k_heun_overlap<FID, true>}) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GF<Family<FID>>::SMEM);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int FID>
cudaError_t launch_heun(const StencilPlan &sp, StencilArgs a, const double *src, double *dst, cudaStream_t st) {
  using g = G<Family<FID>>;
  a.tz = sp.tz;  // the grid and the kernel take the z chunk from the same place
  const dim3 grid((a.nx + g::TX - 1) / g::TX, (a.ny + g::TY - 1) / g::TY, (a.nz + sp.tz - 1) / sp.tz);
  k_heun_fused<FID><<<grid, dim3(32, g::TYT), g::SMEM, st>>>(a, src, dst);
  return cudaGetLastError();
}

// z chunk of a field launch over `count` images: minimise waves * (chunk + 2R)
// (the field kernel pays 2R warm-up planes per chunk), balanced chunks only.
template <int FID>
int field_tz(const StencilPlan &sp, const StencilArgs &a, int count) {
  const long long txy = (long long)((a.nx + 31) / 32) * ((a.ny + Family<FID>::BY - 1) / Family<FID>::BY) * count;
  const long long slots = (long long)sp.nsm * sp.occ_field;
  int best_tz = a.nz;
  long long best = -1;
  for (int tz = a.nz; tz >= 1; --tz) {
    const int nchunk = (a.nz + tz - 1) / tz;
    if (tz != a.nz && (a.nz + nchunk - 1) / nchunk != tz) continue;
    if ((long long)nchunk * count > 65535) break;
    const long long waves = (txy * nchunk + slots - 1) / slots;
    const long long cost = waves * (tz + 2 * Family<FID>::R);
    if (best < 0 || cost < best) {
      best = cost;
      best_tz = tz;
    }
  }
  return best_tz;
}

// 5-D tensor map (x, y, z, sublattice, component) over a spin-like array [3][nsub][nz][ny][nx] of FP64 (or
// FP32) values, whose box is the load region of a pass-kernel tile with its x start rounded down to 16
// bytes.  False (the pass then copies site by site) without the driver's encoder, for a base address that
// is not 16-byte aligned, or for a layout the encoder rejects.
template <int FID>
bool encode_plane_map(const StencilPlan &sp, const StencilArgs &a, const void *base, bool f32, CUtensorMap *tm) {
  using g = GF<Family<FID>>;
  memset(tm, 0, sizeof(*tm));
  // the FP32 map serves the corrector (S~), the FP64 one the predictor and field passes (S)
  if (!(sp.tma & (f32 ? 2 : 1)) || !sp.tma_ok || !base || ((uintptr_t)base & 15u)) return false;
  const auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encode_fn());
  if (!enc) return false;
  const cuuint64_t es = f32 ? 4 : 8;
  const cuuint64_t nx = (cuuint64_t)a.nx, ny = (cuuint64_t)a.ny, nz = (cuuint64_t)a.nz;
  const cuuint64_t dims[5] = {nx, ny, nz, (cuuint64_t)g::NS, 3};
  const cuuint64_t strides[4] = {nx * es, nx * ny * es, nx * ny * nz * es, (cuuint64_t)a.nsite * es};
  const cuuint32_t box[5] = {(cuuint32_t)(f32 ? g::LXA32 : g::LXA64), (cuuint32_t)g::LY, 1, (cuuint32_t)g::NS, 3};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUresult r = enc(tm, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5,
                         const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int FID>
cudaError_t launch_field(const StencilPlan &sp, const StencilArgs &base, int onsite, const double *S, double *b,
                         int count, long long stride, cudaStream_t st, float *bf = nullptr) {
  using g = GF<Family<FID>>;
  StencilArgs a = base;
  a.tz = count == 1 ? sp.tz : field_tz<FID>(sp, a, count);
  PassIO io;
  memset(&io, 0, sizeof(io));
  io.S = S;
  io.b = b;
  io.bf = bf;
  io.nzc = (a.nz + a.tz - 1) / a.tz;
  io.istride = stride;
  io.werr = sp.d_bar ? &sp.d_bar->err : nullptr;
  if ((long long)io.nzc * count > 65535) return cudaErrorInvalidConfiguration;
  CUtensorMap tm;
  io.tma = count == 1 && encode_plane_map<FID>(sp, a, S, false, &tm) ? 1 : 0;  // one image: a 5-D box
  const dim3 grid((a.nx + 31) / 32, (a.ny + Family<FID>::BY - 1) / Family<FID>::BY, io.nzc * count);
  (io.tma ? k_stencil_pass<FID, PASS_FIELD, true> : k_stencil_pass<FID, PASS_FIELD, false>)
      <<<grid, dim3(32, GF<Family<FID>>::TYT), g::SMEM, st>>>(a, onsite, io, tm);
  return cudaGetLastError();
}

// two-pass Heun step: predictor pass into the S~ / f0 workspace, corrector pass into dst
template <int FID>
cudaError_t launch_heun2(const StencilPlan &sp, StencilArgs a, const double *src, double *dst, cudaStream_t st) {
  using g = GF<Family<FID>>;
  a.tz = sp.tz2;
  PassIO io;
  memset(&io, 0, sizeof(io));
  io.S = src;
  io.St = sp.d_St;
  io.St_out = sp.d_St;
  io.f0 = sp.d_f0;
  io.eta = sp.d_eta;
  io.Sout = dst;
  io.b = nullptr;
  io.sched = sp.d_sched;
  io.step = a.step;
  io.nzc = (a.nz + a.tz - 1) / a.tz;
  io.werr = sp.d_bar ? &sp.d_bar->err : nullptr;
  if (sp.ovl_grid) {
    // one launch: clear the done flags and the queue counter, then the overlapped units
    io.sched = nullptr;
    CUtensorMap tp, tc;
    const int use_p = encode_plane_map<FID>(sp, a, src, false, &tp) ? 1 : 0;
    const int use_c = encode_plane_map<FID>(sp, a, sp.d_St, true, &tc) ? 1 : 0;
    cudaError_t e = cudaMemsetAsync(sp.d_done, 0, (size_t)sp.n_done * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sp.d_queue, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    ((use_p || use_c) ? k_heun_overlap<FID, true> : k_heun_overlap<FID, false>)
        <<<sp.ovl_grid, dim3(32, GF<Family<FID>>::TYT), g::SMEM, st>>>(a, io, sp.d_order, sp.n_order, sp.d_queue,
                                                                       sp.d_done, tp, tc, use_p, use_c);
    return cudaGetLastError();
  }
  const dim3 grid = sp.d_sched ? dim3(sp.nsched)
                               : dim3((a.nx + 31) / 32, (a.ny + Family<FID>::BY - 1) / Family<FID>::BY, io.nzc);
  CUtensorMap tm;
  io.tma = encode_plane_map<FID>(sp, a, src, false, &tm) ? 1 : 0;
  (io.tma ? k_stencil_pass<FID, PASS_PRED, true> : k_stencil_pass<FID, PASS_PRED, false>)
      <<<grid, dim3(32, GF<Family<FID>>::TYT), g::SMEM, st>>>(a, 1, io, tm);
  io.tma = encode_plane_map<FID>(sp, a, sp.d_St, true, &tm) ? 1 : 0;
  (io.tma ? k_stencil_pass<FID, PASS_CORR, true> : k_stencil_pass<FID, PASS_CORR, false>)
      <<<grid, dim3(32, GF<Family<FID>>::TYT), g::SMEM, st>>>(a, 1, io, tm);
  return cudaGetLastError();
}

// One pass (PRED or CORR) of the two-pass step over z chunk zc (a.tz planes) on the grid of tile columns.
template <int FID>
cudaError_t launch_pass_chunk(const StencilPlan &sp, const StencilArgs &a, const double *src, double *dst, int mode,
                              int zc, cudaStream_t st) {
  using g = GF<Family<FID>>;
  PassIO io;
  memset(&io, 0, sizeof(io));
  io.S = src;
  io.St = sp.d_St;
  io.St_out = sp.d_St;
  io.f0 = sp.d_f0;
  io.eta = sp.d_eta;
  io.Sout = dst;
  io.step = a.step;
  io.nzc = 1;
  io.zc0 = zc;
  io.werr = sp.d_bar ? &sp.d_bar->err : nullptr;
  const dim3 grid((a.nx + 31) / 32, (a.ny + Family<FID>::BY - 1) / Family<FID>::BY, 1);
  CUtensorMap tm;
  if (mode == PASS_PRED) {
    io.tma = encode_plane_map<FID>(sp, a, src, false, &tm) ? 1 : 0;
    (io.tma ? k_stencil_pass<FID, PASS_PRED, true> : k_stencil_pass<FID, PASS_PRED, false>)
        <<<grid, dim3(32, GF<Family<FID>>::TYT), g::SMEM, st>>>(a, 1, io, tm);
  } else {
    io.tma = encode_plane_map<FID>(sp, a, sp.d_St, true, &tm) ? 1 : 0;
    (io.tma ? k_stencil_pass<FID, PASS_CORR, true> : k_stencil_pass<FID, PASS_CORR, false>)
        <<<grid, dim3(32, GF<Family<FID>>::TYT), g::SMEM, st>>>(a, 1, io, tm);
  }
  return cudaGetLastError();
}

template <int FID>
cudaError_t launch_persistent(const StencilPlan &sp, const StencilArgs &a, double *S0, double *S1, int nsteps,
                              unsigned long long step0, cudaStream_t st) {
  using g = GF<Family<FID>>;
  PassIO io;
  memset(&io, 0, sizeof(io));
  io.St = sp.d_St;
  io.St_out = sp.d_St;
  io.f0 = sp.d_f0;
  io.eta = sp.d_eta;
  io.sched = sp.d_sched;
  io.nzc = 1;
  StencilArgs pa = a;
  GridBar *gb = sp.d_bar;
  void *args[] = {(void *)&pa, (void *)&io, (void *)&S0, (void *)&S1, (void *)&nsteps, (void *)&step0, (void *)&gb};
  cudaError_t e = cudaMemsetAsync(sp.d_bar, 0, 2 * sizeof(unsigned), st);  // count, gen (err is sticky)
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel((const void *)k_heun_persistent<FID>, dim3(sp.nsched),
                                     dim3(32, GF<Family<FID>>::TYT), args, g::SMEM, st);
}

std::vector<int2> balanced_schedule_multi(const std::vector<long long> &ncol, const std::vector<int> &nz, int R,
                                          long long slots) {
  return sched::balanced_schedule_multi<int2>(ncol, nz, R, slots);
}
std::vector<int2> balanced_schedule(long long ncol, int nz, int R, long long slots) {
  return sched::balanced_schedule<int2>(ncol, nz, R, slots);
}

// z chunk per CTA: each chunk pays 4R warm-up planes, and the grid runs in
// waves of (SMs x resident CTAs); pick the chunk that minimises
// waves * (chunk + 4R), preferring longer chunks (fewer re-read planes) on ties.
template <int FID>
int choose_tz(const sx_ctx *c) {
  using F = Family<FID>;
  using g = G<F>;
  const int txy = ((c->geo.nx + g::TX - 1) / g::TX) * ((c->geo.ny + g::TY - 1) / g::TY);
  int nsm = 152, occ = 1;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_heun_fused<FID>, g::NT, g::SMEM) != cudaSuccess ||
      occ < 1)
    occ = 1;
  const long long slots = (long long)nsm * occ;
  const int nz = c->geo.nz;
  int best_tz = nz;
  long long best = -1;
  for (int tz = nz; tz >= 1; --tz) {
    const int nchunk = (nz + tz - 1) / tz;
    if (tz != nz && (nz + nchunk - 1) / nchunk != tz) continue;  // only balanced chunk lengths
    const long long waves = ((long long)txy * nchunk + slots - 1) / slots;
    const long long cost = waves * (tz + 4 * F::R);
    if (best < 0 || cost < best) {
      best = cost;
      best_tz = tz;
    }
  }
  return best_tz;
}

template <int FID>
cudaError_t persistent_occupancy(int *occ) {
  cudaError_t e = cudaFuncSetAttribute(k_heun_persistent<FID>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)GF<Family<FID>>::SMEM);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_heun_persistent<FID>, GF<Family<FID>>::NT,
                                                       GF<Family<FID>>::SMEM);
}

template <int FID>
cudaError_t overlap_occupancy(int *occ) {
  cudaError_t e = cudaFuncSetAttribute(k_heun_overlap<FID, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)GF<Family<FID>>::SMEM);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_heun_overlap<FID, true>, GF<Family<FID>>::NT,
                                                       GF<Family<FID>>::SMEM);
}

template <int FID>
int field_occupancy() {
  int occ = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_stencil_pass<FID, PASS_CORR, false>, GF<Family<FID>>::NT,
                                                    GF<Family<FID>>::SMEM) != cudaSuccess ||
      occ < 1)
    occ = 1;
  return occ;
}

}  // namespace

int stencil_plan(sx_ctx *c) {
  if (c->prec != SX_PREC_FP32)
    return set_error(SX_ERR_UNSUPPORTED, "the stencil backend computes the field in FP32 (use gather for FP64)");
  if (c->geo.nsite >= (1LL << 32))
    return set_error(SX_ERR_UNSUPPORTED, "the stencil backend indexes sites with 32 bits: nsite must be below 2^32");
  StencilPlan *sp = new (std::nothrow) StencilPlan();
  if (!sp) return set_error(SX_ERR_OOM, "host allocation failed");
  StencilArgs &a = sp->base;
  memset(&a, 0, sizeof(a));
  int fam = -1;
  if (match_family<FAM_SC6_ISO>(c, a))
    fam = FAM_SC6_ISO;
  else if (match_family<FAM_SC6_TEN>(c, a))
    fam = FAM_SC6_TEN;
  else if (match_shell26(c, a))
    fam = FAM_SC26_SHELL;
  else if (match_family<FAM_SC26_ISO>(c, a))
    fam = FAM_SC26_ISO;
  else if (match_family<FAM_SC26_TEN>(c, a))
    fam = FAM_SC26_TEN;
  else if (match_family<FAM_SC32_ISO>(c, a))
    fam = FAM_SC32_ISO;
  else if (match_family<FAM_BCC4>(c, a))
    fam = FAM_BCC4;
  if (fam < 0) {
    delete sp;
    return set_error(SX_ERR_UNSUPPORTED,
                     "no stencil family holds these taps (families: SC nearest neighbours, SC 3x3x3 cube, SC four shells, bcc four "
                     "shells); use the gather backend");
  }
  sp->family = fam;
  a.nx = c->geo.nx;
  a.ny = c->geo.ny;
  a.nz = c->geo.nz;
  a.px = c->geo.px;
  a.py = c->geo.py;
  a.pz = c->geo.pz;
  a.nsite = c->geo.nsite;
  for (int s = 0; s < c->lat.nsub && s < 2; ++s) {
    for (int k = 0; k < 3; ++k) {
      a.zee[s][k] = (float)c->onsite.zee[s][k];
      a.axis[s][k] = (float)c->onsite.axis[s][k];
    }
    a.twoK[s] = (float)c->onsite.twoK[s];
    a.inv_mm[s] = (float)c->onsite.inv_mm[s];
  }
  cudaError_t e;
  switch (fam) {
    case FAM_SC6_ISO: e = set_smem<FAM_SC6_ISO>(); break;
    case FAM_SC6_TEN: e = set_smem<FAM_SC6_TEN>(); break;
    case FAM_SC26_ISO: e = set_smem<FAM_SC26_ISO>(); break;
    case FAM_SC26_TEN: e = set_smem<FAM_SC26_TEN>(); break;
    case FAM_SC26_SHELL: e = set_smem<FAM_SC26_SHELL>(); break;
    case FAM_SC32_ISO: e = set_smem<FAM_SC32_ISO>(); break;
    default: e = set_smem<FAM_BCC4>(); break;
  }
  if (e != cudaSuccess) {
    delete sp;
    return cuda_error(e, "cudaFuncSetAttribute");
  }
  switch (fam) {
    case FAM_SC6_ISO: sp->tz = choose_tz<FAM_SC6_ISO>(c); break;
    case FAM_SC6_TEN: sp->tz = choose_tz<FAM_SC6_TEN>(c); break;
    case FAM_SC26_ISO: sp->tz = choose_tz<FAM_SC26_ISO>(c); break;
    case FAM_SC26_TEN: sp->tz = choose_tz<FAM_SC26_TEN>(c); break;
    case FAM_SC26_SHELL: sp->tz = choose_tz<FAM_SC26_SHELL>(c); break;
    case FAM_SC32_ISO: sp->tz = choose_tz<FAM_SC32_ISO>(c); break;
    default: sp->tz = choose_tz<FAM_BCC4>(c); break;
  }
  a.tz = sp->tz;
  sp->nsm = 152;
  cudaDeviceGetAttribute(&sp->nsm, cudaDevAttrMultiProcessorCount, c->device);
  switch (fam) {
    case FAM_SC6_ISO: sp->occ_field = field_occupancy<FAM_SC6_ISO>(); break;
    case FAM_SC6_TEN: sp->occ_field = field_occupancy<FAM_SC6_TEN>(); break;
    case FAM_SC26_ISO: sp->occ_field = field_occupancy<FAM_SC26_ISO>(); break;
    case FAM_SC26_TEN: sp->occ_field = field_occupancy<FAM_SC26_TEN>(); break;
    case FAM_SC26_SHELL: sp->occ_field = field_occupancy<FAM_SC26_SHELL>(); break;
    case FAM_SC32_ISO: sp->occ_field = field_occupancy<FAM_SC32_ISO>(); break;
    default: sp->occ_field = field_occupancy<FAM_BCC4>(); break;
  }
  switch (fam) {
    case FAM_SC6_ISO: sp->tz2 = field_tz<FAM_SC6_ISO>(*sp, a, 1); break;
    case FAM_SC6_TEN: sp->tz2 = field_tz<FAM_SC6_TEN>(*sp, a, 1); break;
    case FAM_SC26_ISO: sp->tz2 = field_tz<FAM_SC26_ISO>(*sp, a, 1); break;
    case FAM_SC26_TEN: sp->tz2 = field_tz<FAM_SC26_TEN>(*sp, a, 1); break;
    case FAM_SC26_SHELL: sp->tz2 = field_tz<FAM_SC26_SHELL>(*sp, a, 1); break;
    case FAM_SC32_ISO: sp->tz2 = field_tz<FAM_SC32_ISO>(*sp, a, 1); break;
    default: sp->tz2 = field_tz<FAM_BCC4>(*sp, a, 1); break;
  }
  {
    // every family uses 32-wide tiles; R and BY per family
    const int R = family_r(fam), BY = family_by(fam);
    const long long ncol = (long long)((a.nx + 31) / 32) * ((a.ny + BY - 1) / BY);
    // Only when the columns are fewer than the resident CTA slots: then the z-chunked grid
    // leaves SMs idle (e.g. 128 CTAs for 152 SMs) and the balanced schedule fills them.
    // With many columns the hardware's dynamic CTA scheduling balances equal columns
    // well and keeps neighbouring columns (which share halo planes) concurrent in L2.
    const long long slots = (long long)sp->nsm * sp->occ_field;
    std::vector<int2> sch;
    if (ncol < slots && ncol * a.nz < (1LL << 31)) sch = balanced_schedule(ncol, a.nz, R, slots);
    sp->nsched = (int)sch.size();
    if (sch.empty()) {
      sp->d_sched = nullptr;
    } else if (cudaMalloc(&sp->d_sched, sch.size() * sizeof(int2)) != cudaSuccess ||
        cudaMemcpy(sp->d_sched, sch.data(), sch.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(sp->d_sched);
      delete sp;
      return set_error(SX_ERR_OOM, "stencil schedule: device allocation failed");
    }
  }
  // error word of the bounded waits (tensor-copy planes, grid barriers of the persistent launch)
  if (cudaMalloc(&sp->d_bar, sizeof(GridBar)) != cudaSuccess || cudaMemset(sp->d_bar, 0, sizeof(GridBar)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(sp->d_sched);
    cudaFree(sp->d_bar);
    delete sp;
    return set_error(SX_ERR_OOM, "stencil error word: device allocation failed");
  }
  sp->tma_ok = (a.nx % 4 == 0 && tensor_map_encode_fn()) ? 1 : 0;
  sp->tma = 0;  // site-by-site staging unless the autotuner or sx_set_tiles chooses tensor copies
  if (sp->d_sched) {
    int occ = 0;
    cudaError_t e2 = cudaSuccess;
    if (e2 == cudaSuccess) {
      switch (fam) {
        case FAM_SC6_ISO: e2 = persistent_occupancy<FAM_SC6_ISO>(&occ); break;
        case FAM_SC6_TEN: e2 = persistent_occupancy<FAM_SC6_TEN>(&occ); break;
        case FAM_SC26_ISO: e2 = persistent_occupancy<FAM_SC26_ISO>(&occ); break;
        case FAM_SC26_TEN: e2 = persistent_occupancy<FAM_SC26_TEN>(&occ); break;
        case FAM_SC26_SHELL: e2 = persistent_occupancy<FAM_SC26_SHELL>(&occ); break;
        case FAM_SC32_ISO: e2 = persistent_occupancy<FAM_SC32_ISO>(&occ); break;
        default: e2 = persistent_occupancy<FAM_BCC4>(&occ); break;
      }
    }
    if (e2 != cudaSuccess) {
      cudaGetLastError();
      occ = 0;
    }
    sp->occ_persist = occ;
    sp->persistent = sp->d_bar && (long long)occ * sp->nsm >= sp->nsched ? 1 : 0;
  }
  sp->sched_factor = sp->d_sched ? 1 : 0;
  c->stencil = sp;
  const int rc = stencil_set_scheme(c, c->opt_scheme);
  if (rc != SX_OK) {
    stencil_free(c);
    return rc;
  }
  return SX_OK;
}

int stencil_set_scheme(sx_ctx *c, int scheme) {
  StencilPlan *sp = c->stencil;
  if (scheme == SX_STENCIL_AUTO) scheme = SX_STENCIL_TWO_PASS;
  if (scheme == SX_STENCIL_TWO_PASS && !sp->d_St) {
    const size_t bytes = 3 * (size_t)c->geo.nsite * sizeof(float);
    if (cudaMalloc(&sp->d_St, bytes) != cudaSuccess || cudaMalloc(&sp->d_f0, bytes) != cudaSuccess ||
        cudaMalloc(&sp->d_eta, bytes) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(sp->d_St);
      cudaFree(sp->d_f0);
      sp->d_St = sp->d_f0 = sp->d_eta = nullptr;
      if (c->opt_scheme == SX_STENCIL_TWO_PASS)
        return set_error(SX_ERR_OOM, "two-pass stencil workspace (36 B per site): out of device memory");
      scheme = SX_STENCIL_FUSED;
    }
  }
  if (scheme == SX_STENCIL_FUSED && sp->d_St) {
    cudaFree(sp->d_St);
    cudaFree(sp->d_f0);
    cudaFree(sp->d_eta);
    sp->d_St = sp->d_f0 = sp->d_eta = nullptr;
  }
  if (sp->scheme != scheme) ++c->plan_gen;  // workspace allocated or freed
  sp->scheme = scheme;
  c->launches_per_step = scheme == SX_STENCIL_TWO_PASS && !sp->ovl_grid ? 2 : 1;
  return SX_OK;
}

int stencil_scheme(const sx_ctx *c) { return c->stencil ? c->stencil->scheme : -1; }

bool stencil_persistent_ok(const sx_ctx *c) {
  return c->stencil && c->stencil->scheme == SX_STENCIL_TWO_PASS && c->stencil->persistent;
}

// 1 if a bounded wait of the persistent kernel gave up since the last check (clears it)
int stencil_check_error(const sx_ctx *c) {
  if (!c->stencil || !c->stencil->d_bar) return 0;
  GridBar h;
  if (cudaMemcpy(&h, c->stencil->d_bar, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return 0;
  if (h.err) cudaMemset(c->stencil->d_bar, 0, sizeof(GridBar));
  return h.err;
}

void stencil_free(sx_ctx *c) {
  if (c->stencil) {
    cudaFree(c->stencil->d_St);
    cudaFree(c->stencil->d_f0);
    cudaFree(c->stencil->d_eta);
    cudaFree(c->stencil->d_sched);
    cudaFree(c->stencil->d_bar);
    cudaFree(c->stencil->d_order);
    cudaFree(c->stencil->d_done);
    cudaFree(c->stencil->d_queue);
  }
  delete c->stencil;
  c->stencil = nullptr;
}

int stencil_family(const sx_ctx *c) { return c->stencil ? c->stencil->family : -1; }

cudaError_t stencil_field_batch(const sx_ctx *c, const double *S, double *b, int count, long long stride,
                                bool onsite, cudaStream_t st) {
  const StencilPlan &sp = *c->stencil;
  switch (sp.family) {
    case FAM_SC6_ISO: return launch_field<FAM_SC6_ISO>(sp, sp.base, onsite, S, b, count, stride, st);
    case FAM_SC6_TEN: return launch_field<FAM_SC6_TEN>(sp, sp.base, onsite, S, b, count, stride, st);
    case FAM_SC26_ISO: return launch_field<FAM_SC26_ISO>(sp, sp.base, onsite, S, b, count, stride, st);
    case FAM_SC26_TEN: return launch_field<FAM_SC26_TEN>(sp, sp.base, onsite, S, b, count, stride, st);
    case FAM_SC26_SHELL: return launch_field<FAM_SC26_SHELL>(sp, sp.base, onsite, S, b, count, stride, st);
    case FAM_SC32_ISO: return launch_field<FAM_SC32_ISO>(sp, sp.base, onsite, S, b, count, stride, st);
    default: return launch_field<FAM_BCC4>(sp, sp.base, onsite, S, b, count, stride, st);
  }
}

cudaError_t stencil_field(const sx_ctx *c, const double *S, double *b, bool onsite, cudaStream_t st) {
  return stencil_field_batch(c, S, b, 1, 0, onsite, st);
}

cudaError_t stencil_field_f32(const sx_ctx *c, const double *S, float *b, bool onsite, cudaStream_t st) {
  const StencilPlan &sp = *c->stencil;
  const int on = onsite ? 1 : 0;
  switch (sp.family) {
    case FAM_SC6_ISO: return launch_field<FAM_SC6_ISO>(sp, sp.base, on, S, nullptr, 1, 0, st, b);
    case FAM_SC6_TEN: return launch_field<FAM_SC6_TEN>(sp, sp.base, on, S, nullptr, 1, 0, st, b);
    case FAM_SC26_ISO: return launch_field<FAM_SC26_ISO>(sp, sp.base, on, S, nullptr, 1, 0, st, b);
    case FAM_SC26_TEN: return launch_field<FAM_SC26_TEN>(sp, sp.base, on, S, nullptr, 1, 0, st, b);
    case FAM_SC26_SHELL: return launch_field<FAM_SC26_SHELL>(sp, sp.base, on, S, nullptr, 1, 0, st, b);
    case FAM_SC32_ISO: return launch_field<FAM_SC32_ISO>(sp, sp.base, on, S, nullptr, 1, 0, st, b);
    default: return launch_field<FAM_BCC4>(sp, sp.base, on, S, nullptr, 1, 0, st, b);
  }
}

namespace {
StencilArgs heun_args(const sx_ctx *c, const HeunConst &h, uint64_t step) {
  StencilArgs a = c->stencil->base;
  a.g = (float)h.g;
  a.alpha = (float)h.alpha;
  a.dt = (float)h.dt;
  a.hdt = (float)(0.5 * h.dt);
  a.thermal = h.thermal;
  for (int s = 0; s < c->lat.nsub && s < 2; ++s) a.sigma[s] = (float)h.sigma[s];
  a.seed = h.seed;
  a.keys = philox_keys(h.seed);
  a.replica = h.replica;
  a.step = step;
  a.status = c->d_status;
  return a;
}
}  // namespace

namespace {
cudaError_t pass_chunk(const StencilPlan &sp, const StencilArgs &a, const double *src, double *dst, int mode, int zc,
                       cudaStream_t st) {
  switch (sp.family) {
    case FAM_SC6_ISO: return launch_pass_chunk<FAM_SC6_ISO>(sp, a, src, dst, mode, zc, st);
    case FAM_SC6_TEN: return launch_pass_chunk<FAM_SC6_TEN>(sp, a, src, dst, mode, zc, st);
    case FAM_SC26_ISO: return launch_pass_chunk<FAM_SC26_ISO>(sp, a, src, dst, mode, zc, st);
    case FAM_SC26_TEN: return launch_pass_chunk<FAM_SC26_TEN>(sp, a, src, dst, mode, zc, st);
    case FAM_SC26_SHELL: return launch_pass_chunk<FAM_SC26_SHELL>(sp, a, src, dst, mode, zc, st);
    case FAM_SC32_ISO: return launch_pass_chunk<FAM_SC32_ISO>(sp, a, src, dst, mode, zc, st);
    default: return launch_pass_chunk<FAM_BCC4>(sp, a, src, dst, mode, zc, st);
  }
}
}  // namespace

// Steps on a host array with the transfers pipelined against the two passes.  The state is cut into K
// z chunks (up to 64, each at least max(r, 4) planes: the upload-only head and download-only tail of the
// step shrink with the chunk, 16 chunks took 186 ms at 1024^3 and 64 took 161) and goes up chunk by
// chunk on a copy stream.  In the
// first step the predictor of chunk c waits only for the chunks holding its planes and their halo (c - 1 ..
// c + 1, wrapped on a periodic z axis), so it runs while later chunks are still in flight.  In the last
// step each corrector chunk is launched as soon as the predictor chunks of its S~ halo have been, and
// goes down on a second copy stream right after it, overlapping the uploads (the link is full duplex)
// and the remaining passes.  The per-site arithmetic is that of the two-pass step on any z chunk, so the
// results equal those of whole copies and sx_llg_heun_step.  cudaErrorNotSupported when the plan does
// not take this path (not the two-pass scheme, too few planes); the caller then copies whole arrays.
cudaError_t stencil_heun_host(const sx_ctx *c, double *S_host, double *dA, double *dB, const HeunConst &h,
                              uint64_t step0, int nsteps, cudaStream_t st) {
  const StencilPlan &sp = *c->stencil;
  if (sp.scheme != SX_STENCIL_TWO_PASS || nsteps < 1) return cudaErrorNotSupported;
  const int R = family_r(sp.family), nz = c->geo.nz;
  int K = std::min(64, nz / std::max(R, 4));
  if (K < 4) return cudaErrorNotSupported;
  const int tzh = (nz + K - 1) / K;
  K = (nz + tzh - 1) / tzh;
  if (nz - (K - 1) * tzh < R) return cudaErrorNotSupported;
  const bool pz = c->geo.pz != 0;
  const long long plane = (long long)c->geo.nx * c->geo.ny, subvol = plane * nz, nsite = c->geo.nsite;
  const int nsub = c->lat.nsub;
  auto copy_chunk = [&](double *dev, int z, bool up, cudaStream_t cs) {
    const long long z0 = (long long)z * tzh, len = std::min<long long>(tzh, nz - z0);
    cudaError_t e = cudaSuccess;
    for (int m = 0; m < 3 && e == cudaSuccess; ++m)
      for (int a = 0; a < nsub && e == cudaSuccess; ++a) {
        const long long off = m * nsite + a * subvol + z0 * plane;
        e = up ? cudaMemcpyAsync(dev + off, S_host + off, len * plane * sizeof(double), cudaMemcpyHostToDevice, cs)
               : cudaMemcpyAsync(S_host + off, dev + off, len * plane * sizeof(double), cudaMemcpyDeviceToHost, cs);
      }
    return e;
  };
  cudaStream_t sin = nullptr, sout = nullptr;
  std::vector<cudaEvent_t> ev(2 * K + 2, nullptr);  // [0, K): chunk uploaded, [K, 2K): chunk corrected, start, end
  cudaError_t e = cudaStreamCreateWithFlags(&sin, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sout, cudaStreamNonBlocking);
  for (auto &x : ev)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
  cudaEvent_t &start = ev[2 * K], &done = ev[2 * K + 1];
  if (e == cudaSuccess) e = cudaEventRecord(start, st);  // after the caller's earlier work on st
  if (e == cudaSuccess) e = cudaStreamWaitEvent(sin, start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(sout, start, 0);
  for (int z = 0; z < K && e == cudaSuccess; ++z) {
    e = copy_chunk(dA, z, true, sin);
    if (e == cudaSuccess) e = cudaEventRecord(ev[z], sin);
  }
  double *src = dA, *dst = dB;
  for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
    StencilArgs a = heun_args(c, h, step0 + (uint64_t)k);
    a.tz = tzh;
    const bool last = k == nsteps - 1;
    for (const sched::ChunkOp &op : sched::host_step_ops(K, pz, k == 0, last)) {
      if (e != cudaSuccess) break;
      if (!op.corr) {
        if (op.wait >= 0) e = cudaStreamWaitEvent(st, ev[op.wait], 0);
        if (e == cudaSuccess) e = pass_chunk(sp, a, src, dst, PASS_PRED, op.z, st);
        continue;
      }
      e = pass_chunk(sp, a, src, dst, PASS_CORR, op.z, st);
      if (e == cudaSuccess && last) {  // this corrector chunk goes down while the rest of the step runs
        e = cudaEventRecord(ev[K + op.z], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sout, ev[K + op.z], 0);
        if (e == cudaSuccess) e = copy_chunk(dst, op.z, false, sout);
      }
    }
    std::swap(src, dst);
  }
  if (e == cudaSuccess) e = cudaEventRecord(done, sout);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, done, 0);
  for (auto &x : ev)
    if (x) cudaEventDestroy(x);
  if (sin) cudaStreamDestroy(sin);
  if (sout) cudaStreamDestroy(sout);
  return e;
}

// nsteps steps in one persistent launch, S0 -> S1 -> S0 ...; the result is in S_{nsteps mod 2}
cudaError_t stencil_heun_steps_persistent(const sx_ctx *c, double *S0, double *S1, const HeunConst &h,
                                          uint64_t step0, int nsteps, cudaStream_t st) {
  const StencilPlan &sp = *c->stencil;
  StencilArgs a = heun_args(c, h, step0);
  a.tz = sp.tz2;
  switch (sp.family) {
    case FAM_SC6_ISO: return launch_persistent<FAM_SC6_ISO>(sp, a, S0, S1, nsteps, step0, st);
    case FAM_SC6_TEN: return launch_persistent<FAM_SC6_TEN>(sp, a, S0, S1, nsteps, step0, st);
    case FAM_SC26_ISO: return launch_persistent<FAM_SC26_ISO>(sp, a, S0, S1, nsteps, step0, st);
    case FAM_SC26_TEN: return launch_persistent<FAM_SC26_TEN>(sp, a, S0, S1, nsteps, step0, st);
    case FAM_SC26_SHELL: return launch_persistent<FAM_SC26_SHELL>(sp, a, S0, S1, nsteps, step0, st);
    case FAM_SC32_ISO: return launch_persistent<FAM_SC32_ISO>(sp, a, S0, S1, nsteps, step0, st);
    default: return launch_persistent<FAM_BCC4>(sp, a, S0, S1, nsteps, step0, st);
  }
}

// ------------------------------------------------------------------ batches (host)

struct StencilBatch {
  int nrep = 0, nimg = 0, family = -1;
  const sx_ctx *proto = nullptr;
  std::vector<BatchRep> h_reps;  // replicas (the per-step schedule)
  BatchRep *d_reps = nullptr;
  int2 *d_sched = nullptr;
  int nsched = 0;
  // sx_batch_run: replicas then images, bound once; own schedule sized for the persistent kernel
  std::vector<BatchRep> h_run;
  BatchRep *d_run = nullptr;
  int2 *d_rsched = nullptr;      // replicas and images (first predictor phase)
  int nrsched = 0;
  int2 *d_rsched_rep = nullptr;  // replicas only (every other phase)
  int nrsched_rep = 0;
  int persistent = 0;  // 1: the nrsched CTAs of the persistent kernel are resident at once
  int bound = 0;
  GridBar *d_bar = nullptr;
};

namespace {
bool same_couplings(const StencilArgs &a, const StencilArgs &b) {
  return memcmp(a.Jiso, b.Jiso, sizeof(a.Jiso)) == 0 && memcmp(a.Jt, b.Jt, sizeof(a.Jt)) == 0 &&
         memcmp(a.zee, b.zee, sizeof(a.zee)) == 0 && memcmp(a.twoK, b.twoK, sizeof(a.twoK)) == 0 &&
         memcmp(a.axis, b.axis, sizeof(a.axis)) == 0 && memcmp(a.inv_mm, b.inv_mm, sizeof(a.inv_mm)) == 0;
}

template <int FID>
cudaError_t launch_batch(const StencilBatch &b, const StencilArgs &a, unsigned long long step, cudaStream_t st) {
  using g = GF<Family<FID>>;
  const dim3 grid(b.nsched), block(32, GF<Family<FID>>::TYT);
  k_batch_pass<FID, PASS_PRED><<<grid, block, g::SMEM, st>>>(a, b.d_reps, b.nrep, b.d_sched, step, 0, 0);
  k_batch_pass<FID, PASS_CORR><<<grid, block, g::SMEM, st>>>(a, b.d_reps, b.nrep, b.d_sched, step, 0, 0);
  return cudaGetLastError();
}

template <int FID>
cudaError_t launch_batch_run(const StencilBatch &b, const StencilArgs &a, unsigned long long step0, int nsteps,
                             cudaStream_t st) {
  using g = GF<Family<FID>>;
  const dim3 block(32, GF<Family<FID>>::TYT);
  const int nown = b.nrep + b.nimg;
  if (b.persistent) {
    cudaError_t e = cudaMemsetAsync(b.d_bar, 0, 2 * sizeof(unsigned), st);  // count, gen (err is sticky)
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(std::max(b.nrsched, b.nrsched_rep));
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = g::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch_persistent<FID>, a, (const BatchRep *)b.d_run, nown,
                              (const int2 *)b.d_rsched, b.nrsched, (const int2 *)b.d_rsched_rep, b.nrsched_rep, step0,
                              nsteps, b.d_bar);
  }
  for (int k = 0; k < nsteps; ++k) {
    if (k == 0)
      k_batch_pass<FID, PASS_PRED><<<dim3(b.nrsched), block, g::SMEM, st>>>(a, b.d_run, nown, b.d_rsched, step0, 0, 1);
    else
      k_batch_pass<FID, PASS_PRED><<<dim3(b.nrsched_rep), block, g::SMEM, st>>>(a, b.d_run, nown, b.d_rsched_rep,
                                                                               step0 + k, k & 1, 0);
    k_batch_pass<FID, PASS_CORR><<<dim3(b.nrsched_rep), block, g::SMEM, st>>>(a, b.d_run, nown, b.d_rsched_rep,
                                                                             step0 + k, k & 1, 0);
  }
  return cudaGetLastError();
}

template <int FID>
cudaError_t batch_persistent_occupancy(int *occ) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_batch_persistent<FID>, GF<Family<FID>>::NT,
                                                       GF<Family<FID>>::SMEM);
}

BatchRep owner_of(const sx_ctx *c, int kind) {
  BatchRep rep;
  memset(&rep, 0, sizeof(rep));
  rep.g.nx = c->geo.nx;
  rep.g.ny = c->geo.ny;
  rep.g.nz = c->geo.nz;
  rep.g.px = c->geo.px;
  rep.g.py = c->geo.py;
  rep.g.pz = c->geo.pz;
  rep.g.nsite = c->geo.nsite;
  rep.kind = kind;
  if (kind == 0) {
    rep.St = c->stencil->d_St;
    rep.f0 = c->stencil->d_f0;
    rep.eta = c->stencil->d_eta;
  }
  return rep;
}
}  // namespace

int stencil_batch_create(StencilBatch **out, sx_ctx *const *ctxs, int nrep, const sx_ctx *img_ctx, int nimg) {
  StencilBatch *b = new (std::nothrow) StencilBatch();
  if (!b) return set_error(SX_ERR_OOM, "host allocation failed");
  b->nrep = nrep;
  b->nimg = img_ctx ? nimg : 0;
  b->proto = ctxs[0];
  b->family = ctxs[0]->stencil->family;
  const int BY = family_by(b->family), R = family_r(b->family);
  std::vector<long long> ncol, rcol;
  std::vector<int> nz, rnz;
  long long u0 = 0;
  auto columns = [&](const sx_ctx *c) { return (long long)((c->geo.nx + 31) / 32) * ((c->geo.ny + BY - 1) / BY); };
  for (int r = 0; r < nrep; ++r) {
    const sx_ctx *c = ctxs[r];
    if (c->stencil->family != b->family || !same_couplings(c->stencil->base, ctxs[0]->stencil->base)) {
      delete b;
      return set_error(SX_ERR_ARG, "batched replicas must share the lattice family and every coupling");
    }
    if (c->device != ctxs[0]->device) {
      delete b;
      return set_error(SX_ERR_ARG, "batched replicas must be planned on one device");
    }
    BatchRep rep = owner_of(c, 0);
    rep.u0 = u0;
    ncol.push_back(columns(c));
    nz.push_back(c->geo.nz);
    u0 += ncol.back() * nz.back();
    b->h_reps.push_back(rep);
  }
  long long ru0 = u0;
  b->h_run = b->h_reps;
  rcol = ncol;
  rnz = nz;
  if (b->nimg > 0) {
    if (img_ctx->stencil->family != b->family || !same_couplings(img_ctx->stencil->base, ctxs[0]->stencil->base) ||
        img_ctx->device != ctxs[0]->device) {
      delete b;
      return set_error(SX_ERR_ARG, "the images must share the batch's lattice family, couplings and device");
    }
    for (int k = 0; k < b->nimg; ++k) {
      BatchRep rep = owner_of(img_ctx, 1);
      rep.u0 = ru0;
      rcol.push_back(columns(img_ctx));
      rnz.push_back(img_ctx->geo.nz);
      ru0 += rcol.back() * rnz.back();
      b->h_run.push_back(rep);
    }
  }
  if (ru0 >= (1LL << 31)) {
    delete b;
    return set_error(SX_ERR_UNSUPPORTED, "batch too large for one schedule (2^31 column-plane units)");
  }
  const StencilPlan &sp0 = *ctxs[0]->stencil;
  std::vector<int2> sch = balanced_schedule_multi(ncol, nz, R, (long long)sp0.nsm * sp0.occ_field);
  b->nsched = (int)sch.size();
  // the run schedule: as many CTAs as the persistent kernel keeps resident
  int occ = 0;
  cudaError_t e = cudaSuccess;
  switch (b->family) {
    case FAM_SC6_ISO: e = batch_persistent_occupancy<FAM_SC6_ISO>(&occ); break;
    case FAM_SC6_TEN: e = batch_persistent_occupancy<FAM_SC6_TEN>(&occ); break;
    case FAM_SC26_ISO: e = batch_persistent_occupancy<FAM_SC26_ISO>(&occ); break;
    case FAM_SC26_TEN: e = batch_persistent_occupancy<FAM_SC26_TEN>(&occ); break;
    case FAM_SC26_SHELL: e = batch_persistent_occupancy<FAM_SC26_SHELL>(&occ); break;
    case FAM_SC32_ISO: e = batch_persistent_occupancy<FAM_SC32_ISO>(&occ); break;
    default: e = batch_persistent_occupancy<FAM_BCC4>(&occ); break;
  }
  if (e != cudaSuccess || occ < 1) occ = 0;
  const long long rslots = (long long)sp0.nsm * (occ > 0 ? occ : sp0.occ_field);
  std::vector<int2> rsch = balanced_schedule_multi(rcol, rnz, R, rslots);
  std::vector<int2> rsch_rep = balanced_schedule_multi(ncol, nz, R, rslots);
  b->nrsched = (int)rsch.size();
  b->nrsched_rep = (int)rsch_rep.size();
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctxs[0]->device);
  b->persistent = coop && occ > 0 && std::max(b->nrsched, b->nrsched_rep) <= rslots ? 1 : 0;
  e = cudaMalloc(&b->d_reps, nrep * sizeof(BatchRep));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_sched, sch.size() * sizeof(int2));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_sched, sch.data(), sch.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_run, b->h_run.size() * sizeof(BatchRep));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_rsched, rsch.size() * sizeof(int2));
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_rsched, rsch.data(), rsch.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_rsched_rep, rsch_rep.size() * sizeof(int2));
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_rsched_rep, rsch_rep.data(), rsch_rep.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_bar, sizeof(GridBar));
  if (e == cudaSuccess) e = cudaMemset(b->d_bar, 0, sizeof(GridBar));
  if (e != cudaSuccess) {
    stencil_batch_free(b);
    return cuda_error(e, "batch plan");
  }
  *out = b;
  return SX_OK;
}

void stencil_batch_free(StencilBatch *b) {
  if (!b) return;
  cudaFree(b->d_reps);
  cudaFree(b->d_sched);
  cudaFree(b->d_run);
  cudaFree(b->d_rsched);
  cudaFree(b->d_rsched_rep);
  cudaFree(b->d_bar);
  delete b;
}

cudaError_t stencil_batch_step(StencilBatch *b, const double *const *S_in, double *const *S_out, const HeunConst &h,
                               uint64_t step, cudaStream_t st) {
  for (int r = 0; r < b->nrep; ++r) {
    b->h_reps[r].S = S_in[r];
    b->h_reps[r].Sout = S_out[r];
    b->h_reps[r].g.replica = h.replica + (uint32_t)r;
  }
  // pageable source: staged by the CUDA driver before this call returns, ordered on the stream
  cudaError_t e =
      cudaMemcpyAsync(b->d_reps, b->h_reps.data(), b->nrep * sizeof(BatchRep), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  const StencilArgs a = heun_args(b->proto, h, step);
  switch (b->family) {
    case FAM_SC6_ISO: return launch_batch<FAM_SC6_ISO>(*b, a, step, st);
    case FAM_SC6_TEN: return launch_batch<FAM_SC6_TEN>(*b, a, step, st);
    case FAM_SC26_ISO: return launch_batch<FAM_SC26_ISO>(*b, a, step, st);
    case FAM_SC26_TEN: return launch_batch<FAM_SC26_TEN>(*b, a, step, st);
    case FAM_SC26_SHELL: return launch_batch<FAM_SC26_SHELL>(*b, a, step, st);
    case FAM_SC32_ISO: return launch_batch<FAM_SC32_ISO>(*b, a, step, st);
    default: return launch_batch<FAM_BCC4>(*b, a, step, st);
  }
}

int stencil_batch_bind(StencilBatch *b, double *const *S_a, double *const *S_b, const double *images,
                       double *fields, uint32_t replica0) {
  for (int r = 0; r < b->nrep; ++r) {
    b->h_run[r].S = S_a[r];
    b->h_run[r].Sout = S_b[r];
    b->h_run[r].g.replica = replica0 + (uint32_t)r;
  }
  for (int k = 0; k < b->nimg; ++k) {
    BatchRep &o = b->h_run[b->nrep + k];
    const long long n3 = 3 * o.g.nsite;
    o.S = images + n3 * k;
    o.b = fields + n3 * k;
  }
  const cudaError_t e =
      cudaMemcpy(b->d_run, b->h_run.data(), b->h_run.size() * sizeof(BatchRep), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_error(e, "batch bind");
  b->bound = 1;
  return SX_OK;
}

int stencil_batch_bound(const StencilBatch *b) { return b->bound; }
int stencil_batch_persistent(const StencilBatch *b) { return b->persistent; }

cudaError_t stencil_batch_run(StencilBatch *b, const HeunConst &h, uint64_t step0, int nsteps, cudaStream_t st) {
  const StencilArgs a = heun_args(b->proto, h, step0);
  switch (b->family) {
    case FAM_SC6_ISO: return launch_batch_run<FAM_SC6_ISO>(*b, a, step0, nsteps, st);
    case FAM_SC6_TEN: return launch_batch_run<FAM_SC6_TEN>(*b, a, step0, nsteps, st);
    case FAM_SC26_ISO: return launch_batch_run<FAM_SC26_ISO>(*b, a, step0, nsteps, st);
    case FAM_SC26_TEN: return launch_batch_run<FAM_SC26_TEN>(*b, a, step0, nsteps, st);
    case FAM_SC26_SHELL: return launch_batch_run<FAM_SC26_SHELL>(*b, a, step0, nsteps, st);
    case FAM_SC32_ISO: return launch_batch_run<FAM_SC32_ISO>(*b, a, step0, nsteps, st);
    default: return launch_batch_run<FAM_BCC4>(*b, a, step0, nsteps, st);
  }
}

// 1 if a grid barrier of sx_batch_run gave up since the last check (clears it)
int stencil_batch_check_error(StencilBatch *b) {
  GridBar h;
  if (cudaMemcpy(&h, b->d_bar, sizeof(GridBar), cudaMemcpyDeviceToHost) != cudaSuccess) return 0;
  if (h.err) cudaMemset(b->d_bar, 0, sizeof(GridBar));
  return h.err ? 1 : 0;
}

// ------------------------------------------------------------------ tile shapes (autotuner)

namespace {
template <int FID>
void fused_tile(int *tx, int *ty) {
  *tx = G<Family<FID>>::TX;
  *ty = G<Family<FID>>::TY;
}
void fused_tile_of(int fam, int *tx, int *ty) {
  switch (fam) {
    case FAM_SC6_ISO: fused_tile<FAM_SC6_ISO>(tx, ty); break;
    case FAM_SC6_TEN: fused_tile<FAM_SC6_TEN>(tx, ty); break;
    case FAM_SC26_ISO: fused_tile<FAM_SC26_ISO>(tx, ty); break;
    case FAM_SC26_TEN: fused_tile<FAM_SC26_TEN>(tx, ty); break;
    case FAM_SC26_SHELL: fused_tile<FAM_SC26_SHELL>(tx, ty); break;
    case FAM_SC32_ISO: fused_tile<FAM_SC32_ISO>(tx, ty); break;
    default: fused_tile<FAM_BCC4>(tx, ty); break;
  }
}
// balanced z-chunk lengths near nz / k
std::vector<int> chunk_lengths(int nz, int around) {
  std::vector<int> out;
  auto add = [&](int tz) {
    if (tz < 1 || tz > nz) return;
    const int nchunk = (nz + tz - 1) / tz;
    tz = (nz + nchunk - 1) / nchunk;  // the balanced length of that chunk count
    if (std::find(out.begin(), out.end(), tz) == out.end()) out.push_back(tz);
  };
  add(around);
  for (int k : {1, 2, 3, 4, 6, 8}) add((nz + k - 1) / k);
  for (int tz : {8, 16, 32, 64}) add(tz);
  return out;
}

void overlap_free(StencilPlan &sp) {
  cudaFree(sp.d_order);
  cudaFree(sp.d_done);
  cudaFree(sp.d_queue);
  sp.d_order = sp.d_done = sp.d_queue = nullptr;
  sp.n_order = sp.n_done = sp.ovl_grid = 0;
}

// The overlapped launch needs every halo inside the neighbouring units: edge tile columns, rows and
// the last z chunk at least R wide.
bool overlap_fits(const sx_ctx *c, const StencilPlan &sp, int tz) {
  const int R = family_r(sp.family), BY = family_by(sp.family);
  const int nx = c->geo.nx, ny = c->geo.ny, nz = c->geo.nz;
  const long long units = (long long)((nx + 31) / 32) * ((ny + BY - 1) / BY) * ((nz + tz - 1) / tz);
  return tz >= R && (nx % 32 == 0 || nx % 32 >= R) && (ny % BY == 0 || ny % BY >= R) &&
         nz - (nz + tz - 1) / tz * tz + tz >= R && units < (1LL << 29);
}

int overlap_setup(sx_ctx *c, StencilPlan &sp, int tz) {
  overlap_free(sp);
  if (!overlap_fits(c, sp, tz))
    return set_error(SX_ERR_ARG, "overlapped launch: an edge tile or the last z chunk is narrower than the halo");
  int occ = 0;
  cudaError_t e;
  switch (sp.family) {
    case FAM_SC6_ISO: e = overlap_occupancy<FAM_SC6_ISO>(&occ); break;
    case FAM_SC6_TEN: e = overlap_occupancy<FAM_SC6_TEN>(&occ); break;
    case FAM_SC26_ISO: e = overlap_occupancy<FAM_SC26_ISO>(&occ); break;
    case FAM_SC26_TEN: e = overlap_occupancy<FAM_SC26_TEN>(&occ); break;
    case FAM_SC26_SHELL: e = overlap_occupancy<FAM_SC26_SHELL>(&occ); break;
    case FAM_SC32_ISO: e = overlap_occupancy<FAM_SC32_ISO>(&occ); break;
    default: e = overlap_occupancy<FAM_BCC4>(&occ); break;
  }
  if (e != cudaSuccess || occ < 1) {
    cudaGetLastError();
    return set_error(SX_ERR_CUDA, "overlapped launch: no resident CTA");
  }
  const int BY = family_by(sp.family);
  const int ncx = (c->geo.nx + 31) / 32, ncy = (c->geo.ny + BY - 1) / BY, nchunk = (c->geo.nz + tz - 1) / tz;
  const int grid = occ * sp.nsm;
  const std::vector<int> order = sched::overlap_order(ncx, ncy, nchunk, c->geo.px, c->geo.py, c->geo.pz, grid);
  const int ndone = ncx * ncy * nchunk;
  if (cudaMalloc(&sp.d_order, order.size() * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&sp.d_done, (size_t)ndone * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&sp.d_queue, sizeof(int)) != cudaSuccess ||
      cudaMemcpy(sp.d_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    overlap_free(sp);
    return set_error(SX_ERR_OOM, "overlapped launch: device allocation failed");
  }
  sp.n_order = (int)order.size();
  sp.n_done = ndone;
  sp.ovl_grid = grid;
  return SX_OK;
}
}  // namespace

std::vector<TileChoice> stencil_tile_candidates(const sx_ctx *c, bool thermal) {
  const StencilPlan &sp = *c->stencil;
  std::vector<TileChoice> out;
  const int tma0 = 0;  // the autotuner tries the tensor-copy stagings at its best shape
  for (int tz : chunk_lengths(c->geo.nz, sp.tz)) out.push_back({SX_STENCIL_FUSED, tz, 0, 0, tma0});
  // two-pass: normals stored by the predictor, and (thermal steps) regenerated by the corrector
  for (int regen = 0; regen <= (thermal ? 1 : 0); ++regen) {
    for (int tz : chunk_lengths(c->geo.nz, sp.tz2)) out.push_back({SX_STENCIL_TWO_PASS, tz, 0, regen, tma0});
    const int BY = family_by(sp.family);
    const long long ncol = (long long)((c->geo.nx + 31) / 32) * ((c->geo.ny + BY - 1) / BY);
    if (ncol * c->geo.nz < (1LL << 31))
      for (int f : {1, 2}) out.push_back({SX_STENCIL_TWO_PASS, sp.tz2, f, regen, tma0});
    // one overlapped launch, z chunks of about nz/4 .. nz/16 planes, when the predictor units are at least
    // four times the resident CTA slots
    std::vector<int> otz;
    for (int k : {4, 8, 16}) {
      const int nch = std::min(k, c->geo.nz), tz = (c->geo.nz + nch - 1) / nch;
      if (std::find(otz.begin(), otz.end(), tz) == otz.end() && overlap_fits(c, sp, tz) &&
          ncol * ((c->geo.nz + tz - 1) / tz) >= 4LL * sp.nsm * std::max(sp.occ_field, 1))
        otz.push_back(tz);
    }
    for (int tz : otz) out.push_back({SX_STENCIL_TWO_PASS, tz, kSchedOverlap, regen, tma0});
  }
  return out;
}

int stencil_apply_tiles(sx_ctx *c, const TileChoice &t) {
  StencilPlan &sp = *c->stencil;
  if (t.tma < 0 || t.tma > 3) return set_error(SX_ERR_ARG, "plane staging mask must be in 0 .. 3");
  if (t.tma && !sp.tma_ok)
    return set_error(SX_ERR_UNSUPPORTED, "tensor-copied planes need n[0] a multiple of 4 and the driver's encoder");
  sp.tma = t.tma;
  int rc = stencil_set_scheme(c, t.scheme);
  if (rc != SX_OK) return rc;
  if (stencil_scheme(c) != t.scheme) return set_error(SX_ERR_OOM, "two-pass workspace unavailable");
  if (t.scheme == SX_STENCIL_FUSED) {
    sp.tz = t.tz;
    sp.base.tz = t.tz;
    return SX_OK;
  }
  sp.tz2 = t.tz;
  sp.base.regen = t.regen;
  if (t.sched == kSchedOverlap) {
    cudaFree(sp.d_sched);
    sp.d_sched = nullptr;
    sp.nsched = 0;
    sp.persistent = 0;
    sp.sched_factor = 0;
    c->launches_per_step = 2;
    if ((rc = overlap_setup(c, sp, t.tz)) != SX_OK) return rc;
    sp.sched_factor = kSchedOverlap;
    c->launches_per_step = 1;
    return SX_OK;
  }
  if (sp.ovl_grid) {
    overlap_free(sp);
    sp.sched_factor = 0;
    c->launches_per_step = 2;
  }
  if (t.sched == sp.sched_factor && (t.sched == 0 || sp.d_sched)) return SX_OK;
  cudaFree(sp.d_sched);
  sp.d_sched = nullptr;
  sp.nsched = 0;
  sp.persistent = 0;
  sp.sched_factor = 0;
  if (t.sched > 0) {
    const int R = family_r(sp.family), BY = family_by(sp.family);
    const long long ncol = (long long)((c->geo.nx + 31) / 32) * ((c->geo.ny + BY - 1) / BY);
    if (ncol * c->geo.nz >= (1LL << 31)) return set_error(SX_ERR_ARG, "lattice too large for a balanced schedule");
    const std::vector<int2> sch =
        balanced_schedule(ncol, c->geo.nz, R, (long long)t.sched * sp.nsm * std::max(sp.occ_field, 1));
    if (cudaMalloc(&sp.d_sched, sch.size() * sizeof(int2)) != cudaSuccess ||
        cudaMemcpy(sp.d_sched, sch.data(), sch.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(sp.d_sched);
      sp.d_sched = nullptr;
      return set_error(SX_ERR_OOM, "stencil schedule: device allocation failed");
    }
    sp.nsched = (int)sch.size();
    sp.sched_factor = t.sched;
    sp.persistent = sp.d_bar && sp.occ_persist > 0 && (long long)sp.occ_persist * sp.nsm >= sp.nsched ? 1 : 0;
  }
  return SX_OK;
}

int stencil_fused_tz(const sx_ctx *c) { return c->stencil->tz; }
void stencil_restore_fused_tz(sx_ctx *c, int tz) {
  c->stencil->tz = tz;
  c->stencil->base.tz = tz;
}

TileChoice stencil_current_tiles(const sx_ctx *c) {
  const StencilPlan &sp = *c->stencil;
  if (sp.scheme == SX_STENCIL_FUSED) return {SX_STENCIL_FUSED, sp.tz, 0, 0, sp.tma};
  return {SX_STENCIL_TWO_PASS, sp.tz2, (sp.d_sched || sp.ovl_grid) ? sp.sched_factor : 0, sp.base.regen, sp.tma};
}

void stencil_tiles_info(const sx_ctx *c, int64_t out[8]) {
  const StencilPlan &sp = *c->stencil;
  const int BY = family_by(sp.family), nz = c->geo.nz;
  const long long cx = (c->geo.nx + 31) / 32, cy = (c->geo.ny + BY - 1) / BY;
  out[0] = sp.scheme;
  if (sp.scheme == SX_STENCIL_FUSED) {
    int tx = 0, ty = 0;
    fused_tile_of(sp.family, &tx, &ty);
    out[1] = tx;
    out[2] = ty;
    out[3] = sp.tz;
    out[4] = (long long)((c->geo.nx + tx - 1) / tx) * ((c->geo.ny + ty - 1) / ty) * ((nz + sp.tz - 1) / sp.tz);
    out[5] = 0;
  } else {
    out[1] = 32;
    out[2] = BY;
    out[3] = sp.d_sched ? 0 : sp.tz2;
    out[4] = sp.d_sched ? sp.nsched : sp.ovl_grid ? sp.ovl_grid : cx * cy * ((nz + sp.tz2 - 1) / sp.tz2);
    out[5] = (sp.d_sched || sp.ovl_grid) ? sp.sched_factor : 0;
    out[6] = sp.base.regen;
  }
  out[7] = sp.tma;
}

cudaError_t stencil_heun_step(const sx_ctx *c, const double *src, double *dst, const HeunConst &h, uint64_t step,
                              cudaStream_t st) {
  const StencilPlan &sp = *c->stencil;
  const StencilArgs a = heun_args(c, h, step);
  if (sp.scheme == SX_STENCIL_TWO_PASS) {
    switch (sp.family) {
      case FAM_SC6_ISO: return launch_heun2<FAM_SC6_ISO>(sp, a, src, dst, st);
      case FAM_SC6_TEN: return launch_heun2<FAM_SC6_TEN>(sp, a, src, dst, st);
      case FAM_SC26_ISO: return launch_heun2<FAM_SC26_ISO>(sp, a, src, dst, st);
      case FAM_SC26_TEN: return launch_heun2<FAM_SC26_TEN>(sp, a, src, dst, st);
      case FAM_SC26_SHELL: return launch_heun2<FAM_SC26_SHELL>(sp, a, src, dst, st);
      case FAM_SC32_ISO: return launch_heun2<FAM_SC32_ISO>(sp, a, src, dst, st);
      default: return launch_heun2<FAM_BCC4>(sp, a, src, dst, st);
    }
  }
  switch (sp.family) {
    case FAM_SC6_ISO: return launch_heun<FAM_SC6_ISO>(sp, a, src, dst, st);
    case FAM_SC6_TEN: return launch_heun<FAM_SC6_TEN>(sp, a, src, dst, st);
    case FAM_SC26_ISO: return launch_heun<FAM_SC26_ISO>(sp, a, src, dst, st);
    case FAM_SC26_TEN: return launch_heun<FAM_SC26_TEN>(sp, a, src, dst, st);
    case FAM_SC26_SHELL: return launch_heun<FAM_SC26_SHELL>(sp, a, src, dst, st);
    case FAM_SC32_ISO: return launch_heun<FAM_SC32_ISO>(sp, a, src, dst, st);
    default: return launch_heun<FAM_BCC4>(sp, a, src, dst, st);
  }
}

}  // namespace sx
