// Minimum-energy paths ("Static optimization and minimum-energy paths"), batched
// over the images of a chain.  An image is a whole spin field; the chain is
// nimg images back to back, image n at X + 3 N n.  Endpoints stay fixed.
//
// Geodesic image distance d(Y_n, Y_m) = [sum_i arccos^2(S_i^n . S_i^m)]^(1/2);
// the per-site angle is taken as atan2(|S x T|, S . T), which equals arccos(S.T)
// for unit vectors and stays accurate for nearly parallel spins.
//
// GNEB (Bessarab et al., geodesic NEB): with f = b - (b.S) S the tangent force
// and t+ = P(S_{n+1} - S_n), t- = P(S_n - S_{n-1}) the projected differences,
// the path tangent is tau = a t+ + c t- (energy-weighted upwind choice of
// Henkelman and Jonsson) normalised over the whole image, and
//   F = f - (f.tau^) tau^ + k (d_{n,n+1} - d_{n-1,n}) tau^      (GNEB)
//   F = f - 2 (f.tau^) tau^                                     (climbing image)
// followed by S <- R_exp(S, dt F).  Because tau is linear in t+ and t-, one
// pass over the chain reduces the five inner products t+.t+, t+.t-, t-.t-,
// f.t+, f.t- per image (together with the image energy and the geodesic
// distance to the next image); a one-block kernel then turns them into two
// coefficients per image, F = f + A t+ + C t-, and a second pass moves the
// images.  The fields of all interior images come from one batched launch
// where the backend has one.  No host synchronisation inside an iteration.
//
// String method: every interior image steps S <- R_exp(S, dt f); then the
// images are placed at equal geodesic arc length by per-site spherical
// interpolation between the two neighbouring old images.
//
// Buffers: the caller's chain X and a library chain W alternate.  The fields of
// the interior images of X are written into the interior slots of the other
// chain, and each update thread overwrites the field values it has just read
// at its own site with the new spins, so one extra chain suffices.
//
// Precision: FP64 plans do every step in FP64 (libm-style trig).  Other plans
// (FP32 field) do the path arithmetic in FP32 on FP32-rounded spins with the
// state kept in FP64: the update S + d is formed and renormalised in FP64, the
// energies are summed in FP64.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "sx_device.cuh"
#include "sx_internal.h"

namespace sx {

namespace {

constexpr int kPT = 256;     // threads per block
constexpr int kNS = 8;       // partial sums per (image, block)
constexpr int kMaxImg = 4096;

// partial slots: 0 energy, 1 t+.t+, 2 t+.t-, 3 t-.t-, 4 f.t+, 5 f.t-, 6 theta^2 to the next image
enum { P_E = 0, P_PP, P_PM, P_MM, P_FP, P_FM, P_D2 };

__device__ __forceinline__ double block_sum(double v, double *sm) {
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int s = kPT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sm[0];
  __syncthreads();
  return r;
}

template <typename R>
__device__ __forceinline__ R to_r(double v);
template <>
__device__ __forceinline__ double to_r<double>(double v) {
  return v;
}
template <>
__device__ __forceinline__ float to_r<float>(double v) {
  return f64_to_f32(v);
}

__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return f32_to_f64(v); }

// sublattice of site i (sites are sublattice-major, ncell sites each; nsub <= 8)
__device__ __forceinline__ int sublattice(long long i, long long ncell, int nsub) {
  int a = 0;
  while (a + 1 < nsub && i >= (a + 1) * ncell) ++a;
  return a;
}

template <typename R>
__device__ __forceinline__ void load3(const double *__restrict__ p, long long N, long long i, R s[3]) {
  s[0] = to_r<R>(p[i]);
  s[1] = to_r<R>(p[N + i]);
  s[2] = to_r<R>(p[2 * N + i]);
}

template <typename R>
__device__ __forceinline__ R dot3(const R a[3], const R b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// x <- x - (x.s) s
template <typename R>
__device__ __forceinline__ void project(const R s[3], R x[3]) {
  const R d = dot3(x, s);
  x[0] -= d * s[0];
  x[1] -= d * s[1];
  x[2] -= d * s[2];
}

__device__ __forceinline__ double r_atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float r_atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double r_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float r_sqrt(float x) { return sqrtf(x); }

// angle between unit vectors s and t = s + dl: |s x t| = |s x dl|, s.t = 1 - |dl|^2/2
template <typename R>
__device__ __forceinline__ R site_angle(const R s[3], const R dl[3]) {
  const R c0 = s[1] * dl[2] - s[2] * dl[1];
  const R c1 = s[2] * dl[0] - s[0] * dl[2];
  const R c2 = s[0] * dl[1] - s[1] * dl[0];
  return r_atan2(r_sqrt(c0 * c0 + c1 * c1 + c2 * c2), R(1) - R(0.5) * dot3(dl, dl));
}

// S <- R_exp(S, u) for a tangent u; s64 is the FP64 state, sr its copy in R.  Returns true when
// the result is not finite or has zero length (a numeric error).
__device__ __forceinline__ bool retract(const double s64[3], const double sr[3], const double u[3], double out[3]) {
  (void)sr;
  const double a = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  if (a == 0.0) {
    out[0] = s64[0];
    out[1] = s64[1];
    out[2] = s64[2];
    return !(fabs(s64[0]) + fabs(s64[1]) + fabs(s64[2]) < 1e300);
  }
  const double c = cos(a), sn = sin(a) / a;
  for (int k = 0; k < 3; ++k) out[k] = c * s64[k] + sn * u[k];
  return unit64_checked(out);
}

// FP32 arithmetic, FP64 state: d = (cos a - 1) s + (sin a / a) u with
// cos a - 1 = -2 sin^2(a/2), then S' = N[S + d] in FP64.
__device__ __forceinline__ bool retract(const double s64[3], const float sr[3], const float u[3], double out[3]) {
  const float a = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  const float h = sinf(0.5f * a);
  const float c1 = -2.0f * h * h;
  const float sc = a > 0.0f ? sinf(a) / a : 1.0f;
  const float d[3] = {c1 * sr[0] + sc * u[0], c1 * sr[1] + sc * u[1], c1 * sr[2] + sc * u[2]};
  return renormalise64(s64, d, out);
}

// Zeeman term mu mu_B B per sublattice in the arithmetic type of the path kernels
template <typename R>
struct ZeeR {
  R z[SX_MAX_SUB][3];
};

// Sum NV per-thread values of type R over the block: a shuffle tree in R inside
// each warp, then the warp sums widened and added in FP64 by thread 0, which
// writes out[slot[k]].  All threads must call it.
template <typename R, int NV>
__device__ __forceinline__ void block_reduce_store(R (&v)[NV], const int (&slot)[NV], double *__restrict__ out) {
  __shared__ R red[NV][kPT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    R x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[k][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double acc = 0.0;
      for (int w = 0; w < kPT / 32; ++w) acc += to_d(red[k][w]);
      out[slot[k]] = acc;
    }
  }
}

enum { MODE_GEO = 0, MODE_FULL = 1, MODE_ENERGY = 2 };

// Per (image slot, block) partial sums; image n = n0 + blockIdx.y * nstep.
//  MODE_GEO:    theta^2 to image n+1 (n in 0 .. nimg-2);
//  MODE_FULL:   as MODE_GEO, and for n >= 1 the energy sum S.(b + zee) and the
//               five tangent inner products of image n;
//  MODE_ENERGY: the energy sum of image n only.
// B holds the field of image n in slot n.  Slot layout: partial[(y nb + block) kNS + k].
template <typename R, int MODE>
__global__ void __launch_bounds__(kPT) k_path_reduce(const double *__restrict__ X, const double *__restrict__ B,
                                                     long long N, long long ncell, int nsub, ZeeR<R> zee, int n0,
                                                     int nstep, double *__restrict__ partial) {
  const int n = n0 + blockIdx.y * nstep;
  const double *S = X + 3 * N * (long long)n;
  const double *Sp = S + 3 * N;
  R acc[7] = {0, 0, 0, 0, 0, 0, 0};
  const bool geo = MODE != MODE_ENERGY;
  const bool tangent = MODE == MODE_FULL && n >= 1;
  const bool energy = MODE == MODE_ENERGY || tangent;
  for (long long i = (long long)blockIdx.x * kPT + threadIdx.x; i < N; i += (long long)gridDim.x * kPT) {
    R s[3];
    load3<R>(S, N, i, s);
    R tp[3];
    if (geo) {
      R sp[3];
      load3<R>(Sp, N, i, sp);
      tp[0] = sp[0] - s[0];
      tp[1] = sp[1] - s[1];
      tp[2] = sp[2] - s[2];
      const R th = site_angle<R>(s, tp);
      acc[P_D2] += th * th;
    }
    if (energy) {
      R br[3];
      load3<R>(B + 3 * N * (long long)n, N, i, br);
      const int a = sublattice(i, ncell, nsub);
      acc[P_E] += s[0] * (br[0] + zee.z[a][0]) + s[1] * (br[1] + zee.z[a][1]) + s[2] * (br[2] + zee.z[a][2]);
      if (tangent) {
        R sm_[3];
        load3<R>(S - 3 * N, N, i, sm_);
        R tm[3] = {s[0] - sm_[0], s[1] - sm_[1], s[2] - sm_[2]};
        project<R>(s, tp);
        project<R>(s, tm);
        project<R>(s, br);
        acc[P_PP] += dot3(tp, tp);
        acc[P_PM] += dot3(tp, tm);
        acc[P_MM] += dot3(tm, tm);
        acc[P_FP] += dot3(br, tp);
        acc[P_FM] += dot3(br, tm);
      }
    }
  }
  double *out = partial + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * kNS;
  if (MODE == MODE_GEO) {
    R v[1] = {acc[P_D2]};
    const int sl[1] = {P_D2};
    block_reduce_store<R, 1>(v, sl, out);
  } else if (MODE == MODE_ENERGY) {
    R v[1] = {acc[P_E]};
    const int sl[1] = {P_E};
    block_reduce_store<R, 1>(v, sl, out);
  } else {
    const int sl[7] = {0, 1, 2, 3, 4, 5, 6};
    block_reduce_store<R, 7>(acc, sl, out);  // slot 0 etc. hold zeros for n = 0
  }
}

// sums[y][k] = sum over the blocks of image slot y (fixed order: deterministic);
// the energy slot is scaled by -1/2 (E = -1/2 sum S.(b + zee)).  nv: the
// number of leading slots to reduce (7, or 1 for energies only); with
// geo_only only the geodesic slot is reduced and the others are set to 0.
__global__ void __launch_bounds__(kPT) k_path_sum(const double *__restrict__ partial, int nb, int geo_only,
                                                  double *__restrict__ sums) {
  __shared__ double sm[kPT];
  const int y = blockIdx.x;
  const double *p = partial + (long long)y * nb * kNS;
  for (int k = 0; k < 7; ++k) {
    if (geo_only && k != P_D2) {
      if (threadIdx.x == 0) sums[y * kNS + k] = 0.0;
      continue;
    }
    double acc = 0.0;
    for (int j = threadIdx.x; j < nb; j += kPT) acc += p[(long long)j * kNS + k];
    acc = block_sum(acc, sm);
    if (threadIdx.x == 0) sums[y * kNS + k] = k == P_E ? -0.5 * acc : acc;
  }
}

// Per-image coefficients (one block; nimg <= kMaxImg).
//  GNEB / CI: coef[n] = {A, C, 0, 0} with F = f + A t+ + C t-.
//  string:    coef[n] = {0, 0, j, w}: image n becomes slerp(old_j, old_j+1; w).
// coeff holds the same numbers in FP32.  E[n] receives the image energies
// (endpoints from the energy slots of eend[0 .. kNS) and eend[kNS .. 2 kNS)).
__global__ void __launch_bounds__(kPT) k_path_coef(const double *__restrict__ sums, const double *__restrict__ eend,
                                                   int nimg, int method, double kspring, double *__restrict__ coef,
                                                   float *__restrict__ coeff, double *__restrict__ E,
                                                   double *__restrict__ L) {
  __shared__ int top_s;
  const int M = nimg;
  for (int n = threadIdx.x; n < M; n += blockDim.x)
    E[n] = n == 0 ? eend[P_E] : n == M - 1 ? eend[kNS + P_E] : sums[n * kNS + P_E];
  __syncthreads();
  if (method == SX_PATH_STRING) {
    if (threadIdx.x == 0) {
      L[0] = 0.0;
      for (int n = 0; n < M - 1; ++n) L[n + 1] = L[n] + sqrt(sums[n * kNS + P_D2]);
    }
    __syncthreads();
    for (int n = 1 + threadIdx.x; n < M - 1; n += blockDim.x) {
      const double target = L[M - 1] * n / (M - 1);
      int j = 0;
      while (j < M - 2 && L[j + 1] < target) ++j;
      const double seg = L[j + 1] - L[j];
      const double w = seg > 0.0 ? (target - L[j]) / seg : 0.0;
      coef[4 * n + 0] = 0.0;
      coef[4 * n + 1] = 0.0;
      coef[4 * n + 2] = (double)j;
      coef[4 * n + 3] = w;
      coeff[4 * n + 0] = 0.0f;
      coeff[4 * n + 1] = 0.0f;
      coeff[4 * n + 2] = (float)j;
      coeff[4 * n + 3] = (float)w;
    }
    return;
  }
  if (threadIdx.x == 0) {
    int top = 1;
    for (int n = 2; n < M - 1; ++n)
      if (E[n] > E[top]) top = n;
    top_s = top;
  }
  __syncthreads();
  const int top = top_s;
  for (int n = 1 + threadIdx.x; n < M - 1; n += blockDim.x) {
    const double *s = sums + n * kNS;
    const double dEp = E[n + 1] - E[n], dEm = E[n - 1] - E[n];
    double a, c;
    if (E[n + 1] > E[n] && E[n] > E[n - 1]) {
      a = 1.0;
      c = 0.0;
    } else if (E[n + 1] < E[n] && E[n] < E[n - 1]) {
      a = 0.0;
      c = 1.0;
    } else {
      const double hi = fmax(fabs(dEp), fabs(dEm)), lo = fmin(fabs(dEp), fabs(dEm));
      if (E[n + 1] > E[n - 1]) {
        a = hi;
        c = lo;
      } else {
        a = lo;
        c = hi;
      }
    }
    const double tt = a * a * s[P_PP] + 2.0 * a * c * s[P_PM] + c * c * s[P_MM];
    const double tn = sqrt(fmax(tt, 0.0));
    const double ftau = tn > 0.0 ? (a * s[P_FP] + c * s[P_FM]) / tn : 0.0;
    const bool ci = method == SX_PATH_CI_GNEB && n == top;
    const double dplus = sqrt(sums[n * kNS + P_D2]), dminus = sqrt(sums[(n - 1) * kNS + P_D2]);
    const double ks = ci ? 0.0 : kspring * (dplus - dminus);
    const double cc = tn > 0.0 ? (ks - (ci ? 2.0 : 1.0) * ftau) / tn : 0.0;
    coef[4 * n + 0] = cc * a;
    coef[4 * n + 1] = cc * c;
    coef[4 * n + 2] = 0.0;
    coef[4 * n + 3] = 0.0;
    coeff[4 * n + 0] = (float)(cc * a);
    coeff[4 * n + 1] = (float)(cc * c);
    coeff[4 * n + 2] = 0.0f;
    coeff[4 * n + 3] = 0.0f;
  }
}

// larger of two non-negative values, NaN from either operand kept (a non-finite force must not read as converged)
template <typename R>
__device__ __forceinline__ R max_keep_nan(R a, R b) {
  return (a > b || a != a) ? a : b;
}

template <typename R>
__device__ __forceinline__ void record_max(R v, unsigned long long *slot) {
  __shared__ R red[kPT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max_keep_nan(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0 && slot) {
    for (int w = 1; w < kPT / 32; ++w) v = max_keep_nan(v, red[w]);
    // non-negative doubles order like their bit patterns; a positive NaN orders above every finite value
    double d = to_d(v);
    if (d != d) d = __longlong_as_double(0x7FF8000000000000ll);
    atomicMax(slot, (unsigned long long)__double_as_longlong(d));
  }
}

// GNEB / CI-GNEB update of interior image n = blockIdx.y + 1: reads the chain X
// and the field of image n in slot n of Y, writes the new image into slot n of Y.
template <typename R>
__global__ void __launch_bounds__(kPT) k_gneb_update(const double *__restrict__ X, double *__restrict__ Y, long long N,
                                                     const R *__restrict__ coef, R dt,
                                                     unsigned long long *__restrict__ fmax_slot,
                                                     int *__restrict__ status) {
  const int n = blockIdx.y + 1;
  const long long i = (long long)blockIdx.x * kPT + threadIdx.x;
  R fm = 0;
  if (i < N) {
    const double *S = X + 3 * N * (long long)n;
    double *Yn = Y + 3 * N * (long long)n;
    R s[3], sp[3], smn[3], b[3];
    load3<R>(S, N, i, s);
    load3<R>(S + 3 * N, N, i, sp);
    load3<R>(S - 3 * N, N, i, smn);
    load3<R>(Yn, N, i, b);
    const double s64[3] = {S[i], S[N + i], S[2 * N + i]};
    R tp[3] = {sp[0] - s[0], sp[1] - s[1], sp[2] - s[2]};
    R tm[3] = {s[0] - smn[0], s[1] - smn[1], s[2] - smn[2]};
    project<R>(s, tp);
    project<R>(s, tm);
    project<R>(s, b);
    const R A = coef[4 * n], C = coef[4 * n + 1];
    R u[3];
    for (int k = 0; k < 3; ++k) u[k] = b[k] + A * tp[k] + C * tm[k];
    fm = r_sqrt(dot3(u, u));
    for (int k = 0; k < 3; ++k) u[k] *= dt;
    double out[3];
    report_numeric(status, retract(s64, s, u, out));
    Yn[i] = out[0];
    Yn[N + i] = out[1];
    Yn[2 * N + i] = out[2];
  }
  record_max<R>(fm, fmax_slot);
}

// Velocity projection on the GNEB force, pass 1: the force F of interior image n = blockIdx.y + 1 at every
// site (as k_gneb_update forms it), v' = v + dt/2 (F_prev + F) (0 when first) with the velocity of the previous
// update v = c_prev F_prev (c_prev still in cvp, F_prev in Fp), per-block sums of v'.F and F.F into
// partial[2 * (blockIdx.y * gridDim.x + blockIdx.x) + {0, 1}], and F stored over F_prev.
template <typename R>
__global__ void __launch_bounds__(kPT) k_gneb_vp_force(const double *__restrict__ X, const double *__restrict__ Y,
                                                       long long N, const R *__restrict__ coef, R dt,
                                                       const double *__restrict__ cvp, R *__restrict__ Fp, int first,
                                                       double *__restrict__ partial,
                                                       unsigned long long *__restrict__ fmax_slot) {
  const int n = blockIdx.y + 1;
  const long long i = (long long)blockIdx.x * kPT + threadIdx.x;
  R fm = 0;
  R vf[2] = {0, 0};  // v'.F and F.F of this thread's site
  if (i < N) {
    const double *S = X + 3 * N * (long long)n;
    R s[3], sp[3], smn[3], b[3];
    load3<R>(S, N, i, s);
    load3<R>(S + 3 * N, N, i, sp);
    load3<R>(S - 3 * N, N, i, smn);
    load3<R>(Y + 3 * N * (long long)n, N, i, b);
    R tp[3] = {sp[0] - s[0], sp[1] - s[1], sp[2] - s[2]};
    R tm[3] = {s[0] - smn[0], s[1] - smn[1], s[2] - smn[2]};
    project<R>(s, tp);
    project<R>(s, tm);
    project<R>(s, b);
    const R A = coef[4 * n], C = coef[4 * n + 1];
    R F[3];
    for (int k = 0; k < 3; ++k) F[k] = b[k] + A * tp[k] + C * tm[k];
    fm = r_sqrt(dot3(F, F));
    const long long base = 3 * N * (long long)n + i;
    // the velocity left by the previous update is c_prev F_prev, F_prev the force stored in Fp
    const R cprev = sizeof(R) == 8 ? (R)cvp[0] : (R)reinterpret_cast<const float *>(cvp + 1)[0];
    // all three loads before the stores: F_prev is overwritten through the same pointer, and interleaved
    // loads and stores would have to wait on one another
    R fp[3] = {0, 0, 0};
    if (!first)
      for (int k = 0; k < 3; ++k) fp[k] = Fp[base + k * N];
    for (int k = 0; k < 3; ++k) {
      const R v = first ? (R)0 : cprev * fp[k] + (R)0.5 * dt * (fp[k] + F[k]);
      vf[0] += v * F[k];
      vf[1] += F[k] * F[k];
    }
    for (int k = 0; k < 3; ++k) Fp[base + k * N] = F[k];
  }
  record_max<R>(fm, fmax_slot);
  // warp sums in R, the block's eight warp sums in FP64 (as the other path reductions)
  const int sl[2] = {0, 1};
  block_reduce_store<R, 2>(vf, sl, partial + 2 * ((long long)blockIdx.y * gridDim.x + blockIdx.x));
}

// pass 2: c = max(sum v'.F, 0) / sum F.F over all blocks (fixed order), as cvp[0] (FP64) and cvp[1] (FP32 bits)
__global__ void __launch_bounds__(kPT) k_gneb_vp_coef(const double *__restrict__ partial, long long nblk,
                                                      double *__restrict__ cvp) {
  __shared__ double sm[kPT];
  double pv = 0.0, ff = 0.0;
  for (long long j = threadIdx.x; j < nblk; j += kPT) {
    pv += partial[2 * j];
    ff += partial[2 * j + 1];
  }
  pv = block_sum(pv, sm);
  ff = block_sum(ff, sm);
  if (threadIdx.x == 0) {
    const double c = (pv > 0.0 && ff > 0.0) ? pv / ff : 0.0;
    cvp[0] = c;
    reinterpret_cast<float *>(cvp + 1)[0] = (float)c;
  }
}

// pass 3: S <- R_exp(S, dt c F + dt^2/2 F) from slot n of X into slot n of Y (the velocity c F is kept as c and
// F, which the next force pass reads)
template <typename R>
__global__ void __launch_bounds__(kPT) k_gneb_vp_update(const double *__restrict__ X, double *__restrict__ Y,
                                                        long long N, const R *__restrict__ Fp,
                                                        const double *__restrict__ cvp, R dt,
                                                        int *__restrict__ status) {
  const int n = blockIdx.y + 1;
  const long long i = (long long)blockIdx.x * kPT + threadIdx.x;
  if (i >= N) return;
  const R c = sizeof(R) == 8 ? (R)cvp[0] : (R)reinterpret_cast<const float *>(cvp + 1)[0];
  const double *S = X + 3 * N * (long long)n;
  double *Yn = Y + 3 * N * (long long)n;
  R s[3];
  load3<R>(S, N, i, s);
  const double s64[3] = {S[i], S[N + i], S[2 * N + i]};
  const long long base = 3 * N * (long long)n + i;
  R u[3];
  const R h = (R)0.5 * dt * dt;
  for (int k = 0; k < 3; ++k) {
    const R f = Fp[base + k * N];
    u[k] = dt * c * f + h * f;
  }
  double out[3];
  report_numeric(status, retract(s64, s, u, out));
  Yn[i] = out[0];
  Yn[N + i] = out[1];
  Yn[2 * N + i] = out[2];
}

// string step, in place on interior image n = blockIdx.y + 1 of X (field in slot n of Y)
template <typename R>
__global__ void __launch_bounds__(kPT) k_string_step(double *__restrict__ X, const double *__restrict__ Y, long long N,
                                                     R dt, unsigned long long *__restrict__ fmax_slot,
                                                     int *__restrict__ status) {
  const int n = blockIdx.y + 1;
  const long long i = (long long)blockIdx.x * kPT + threadIdx.x;
  R fm = 0;
  if (i < N) {
    double *S = X + 3 * N * (long long)n;
    R s[3], b[3];
    load3<R>(S, N, i, s);
    load3<R>(Y + 3 * N * (long long)n, N, i, b);
    const double s64[3] = {S[i], S[N + i], S[2 * N + i]};
    project<R>(s, b);
    fm = r_sqrt(dot3(b, b));
    R u[3] = {dt * b[0], dt * b[1], dt * b[2]};
    double out[3];
    report_numeric(status, retract(s64, s, u, out));
    S[i] = out[0];
    S[N + i] = out[1];
    S[2 * N + i] = out[2];
  }
  record_max<R>(fm, fmax_slot);
}

// slerp(a, c; w) on one site, FP64
__device__ __forceinline__ bool slerp_site(const double a[3], const double c[3], double w, double out[3]) {
  const double c0 = a[1] * c[2] - a[2] * c[1], c1 = a[2] * c[0] - a[0] * c[2], c2 = a[0] * c[1] - a[1] * c[0];
  const double th = atan2(sqrt(c0 * c0 + c1 * c1 + c2 * c2), a[0] * c[0] + a[1] * c[1] + a[2] * c[2]);
  double x[3];
  if (th < 1e-12) {
    for (int k = 0; k < 3; ++k) x[k] = a[k];
  } else {
    const double st = sin(th), p = sin((1.0 - w) * th) / st, q = sin(w * th) / st;
    for (int k = 0; k < 3; ++k) x[k] = p * a[k] + q * c[k];
  }
  for (int k = 0; k < 3; ++k) out[k] = x[k];
  return unit64_checked(out);
}

// FP32 arithmetic, FP64 state: out = N[a + d], d = (p + q - 1) a + q (c - a)
__device__ __forceinline__ bool slerp_site_f(const double a64[3], const float a[3], const float c[3], float w,
                                             double out[3]) {
  const float dl[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  const float th = site_angle<float>(a, dl);
  float pq1, q;
  if (th < 1e-6f) {
    pq1 = 0.0f;
    q = w;
  } else {
    const float st = sinf(th);
    const float p = sinf((1.0f - w) * th) / st;
    q = sinf(w * th) / st;
    pq1 = (p - 1.0f) + q;
  }
  const float d[3] = {pq1 * a[0] + q * dl[0], pq1 * a[1] + q * dl[1], pq1 * a[2] + q * dl[2]};
  return renormalise64(a64, d, out);
}

// string redistribution: interior image n = blockIdx.y + 1 of Y from images j, j+1 of X
template <typename R>
__global__ void __launch_bounds__(kPT) k_string_redistribute(const double *__restrict__ X, double *__restrict__ Y,
                                                             long long N, const R *__restrict__ coef,
                                                             int *__restrict__ status) {
  const int n = blockIdx.y + 1;
  const long long i = (long long)blockIdx.x * kPT + threadIdx.x;
  if (i >= N) return;
  const int j = (int)coef[4 * n + 2];
  const R w = coef[4 * n + 3];
  const double *A = X + 3 * N * (long long)j, *Cn = A + 3 * N;
  const double a64[3] = {A[i], A[N + i], A[2 * N + i]};
  double out[3];
  if constexpr (sizeof(R) == 8) {
    const double c64[3] = {Cn[i], Cn[N + i], Cn[2 * N + i]};
    report_numeric(status, slerp_site(a64, c64, w, out));
  } else {
    float a[3], c[3];
    load3<float>(A, N, i, a);
    load3<float>(Cn, N, i, c);
    report_numeric(status, slerp_site_f(a64, a, c, w, out));
  }
  double *Yn = Y + 3 * N * (long long)n;
  Yn[i] = out[0];
  Yn[N + i] = out[1];
  Yn[2 * N + i] = out[2];
}

// geodesic distance squared between two fields, per-block partials (FP64)
__global__ void __launch_bounds__(kPT) k_geo_pair(const double *__restrict__ A, const double *__restrict__ B,
                                                  long long N, double *__restrict__ partial) {
  __shared__ double sm[kPT];
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * kPT + threadIdx.x; i < N; i += (long long)gridDim.x * kPT) {
    const double s[3] = {A[i], A[N + i], A[2 * N + i]};
    const double d[3] = {B[i] - s[0], B[N + i] - s[1], B[2 * N + i] - s[2]};
    const double th = site_angle<double>(s, d);
    acc += th * th;
  }
  acc = block_sum(acc, sm);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kPT) k_geo_final(const double *__restrict__ partial, int nb,
                                                   double *__restrict__ out) {
  __shared__ double sm[kPT];
  double acc = 0.0;
  for (int j = threadIdx.x; j < nb; j += kPT) acc += partial[j];
  acc = block_sum(acc, sm);
  if (threadIdx.x == 0) out[0] = sqrt(acc);
}

int reduce_grid(long long N) {
  const long long per = (long long)kPT * 4;
  return (int)std::max(1LL, std::min(2048LL, (N + per - 1) / per));
}

struct PathLayout {
  double *W, *partial, *sums, *coef, *E, *L, *eend;
  double *Fp, *vp_partial, *cvp;  // velocity projection: previous force, block sums, coefficient (v = c F_prev)
  float *coeff;
  unsigned long long *fmax;
  size_t bytes;
};

PathLayout layout(double *base, long long N, int nimg, int nb) {
  PathLayout l;
  size_t off = 0;
  auto take = [&](size_t n) {
    double *p = base ? base + off : nullptr;
    off += (n + 31) & ~(size_t)31;  // 256-byte aligned slices
    return p;
  };
  l.W = take(3 * (size_t)N * nimg);
  l.partial = take((size_t)(nimg - 1) * nb * kNS);
  l.sums = take((size_t)nimg * kNS);
  l.coef = take(4 * (size_t)nimg);
  l.coeff = (float *)take(2 * (size_t)nimg);
  l.E = take((size_t)nimg);
  l.L = take((size_t)nimg);
  l.eend = take(2 * kNS);
  l.fmax = (unsigned long long *)take(1);
  l.Fp = take(3 * (size_t)N * nimg);
  l.vp_partial = take(2 * (size_t)((N + kPT - 1) / kPT) * (nimg > 2 ? nimg - 2 : 1));
  l.cvp = take(2);
  l.bytes = off * sizeof(double);
  return l;
}

template <typename R>
cudaError_t run_path(sx_ctx *c, double *img, int M, const sx_path_params *p, int *iters_out, double *E_host,
                     double *fmax_host, cudaStream_t st, FieldBatchFn field) {
  const long long N = c->geo.nsite, stride = 3 * N;
  const int nb = reduce_grid(N);
  const unsigned nbu = (unsigned)((N + kPT - 1) / kPT);
  PathLayout l = layout(nullptr, N, M, nb);
  cudaError_t e;
  if (c->path_bytes < l.bytes) {
    cudaFree(c->d_path);
    c->d_path = nullptr;
    c->path_bytes = 0;
    c->path_vp_nimg = 0;
    if ((e = cudaMalloc(&c->d_path, l.bytes)) != cudaSuccess) return e;
    c->path_bytes = l.bytes;
  }
  const bool vp = p->optimizer == SX_PATH_VP && p->method != SX_PATH_STRING;
  int vp_first = !(vp && p->keep_velocity && c->path_vp_nimg == M);
  c->path_vp_nimg = 0;
  l = layout(c->d_path, N, M, nb);
  const size_t ibytes = (size_t)stride * sizeof(double);
  ZeeR<R> zr;
  for (int a = 0; a < SX_MAX_SUB; ++a)
    for (int k = 0; k < 3; ++k) zr.z[a][k] = (R)c->onsite.zee[a][k];
  const int nsub = c->lat.nsub;
  // endpoint energies (fixed for the whole call), with the same arithmetic as
  // the interior images: fields of images 0 and M-1 into slots 0 and M-1 of W
  if ((e = field(c, img, l.W, 2, stride * (M - 1), true, st)) != cudaSuccess) return e;
  k_path_reduce<R, MODE_ENERGY><<<dim3((unsigned)nb, 2), kPT, 0, st>>>(img, l.W, N, c->geo.ncell, nsub, zr, 0, M - 1,
                                                                        l.partial);
  k_path_sum<<<2, kPT, 0, st>>>(l.partial, nb, 0, l.eend);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // then the endpoint spins into the library chain
  if ((e = cudaMemcpyAsync(l.W, img, ibytes, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(l.W + stride * (M - 1), img + stride * (M - 1), ibytes, cudaMemcpyDeviceToDevice,
                           st)) != cudaSuccess)
    return e;
  const bool string = p->method == SX_PATH_STRING;
  const R dt = (R)p->dt;
  const R *coefR = sizeof(R) == 8 ? (const R *)l.coef : (const R *)l.coeff;
  double *X = img, *Y = l.W;
  const dim3 gred((unsigned)nb, (unsigned)(M - 1)), gupd(nbu, (unsigned)(M - 2));
  int it = 0;
  double fmax = -1.0;
  while (it < p->max_iter) {
    const bool measure = (it + 1) % p->check_every == 0 || it + 1 == p->max_iter;
    unsigned long long *slot = measure ? l.fmax : nullptr;
    if (measure && (e = cudaMemsetAsync(l.fmax, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
    if ((e = field(c, X + stride, Y + stride, M - 2, stride, true, st)) != cudaSuccess) return e;
    if (string) {
      k_string_step<R><<<gupd, kPT, 0, st>>>(X, Y, N, dt, slot, c->d_status);
      k_path_reduce<R, MODE_GEO><<<gred, kPT, 0, st>>>(X, Y, N, c->geo.ncell, nsub, zr, 0, 1, l.partial);
      k_path_sum<<<M - 1, kPT, 0, st>>>(l.partial, nb, 1, l.sums);
      k_path_coef<<<1, kPT, 0, st>>>(l.sums, l.eend, M, p->method, p->k_spring, l.coef, l.coeff, l.E, l.L);
      k_string_redistribute<R><<<gupd, kPT, 0, st>>>(X, Y, N, coefR, c->d_status);
    } else {
      k_path_reduce<R, MODE_FULL><<<gred, kPT, 0, st>>>(X, Y, N, c->geo.ncell, nsub, zr, 0, 1, l.partial);
      k_path_sum<<<M - 1, kPT, 0, st>>>(l.partial, nb, 0, l.sums);
      k_path_coef<<<1, kPT, 0, st>>>(l.sums, l.eend, M, p->method, p->k_spring, l.coef, l.coeff, l.E, l.L);
      if (vp) {
        R *Fr = reinterpret_cast<R *>(l.Fp);
        k_gneb_vp_force<R><<<gupd, kPT, 0, st>>>(X, Y, N, coefR, dt, l.cvp, Fr, vp_first, l.vp_partial, slot);
        k_gneb_vp_coef<<<1, kPT, 0, st>>>(l.vp_partial, (long long)nbu * (M - 2), l.cvp);
        k_gneb_vp_update<R><<<gupd, kPT, 0, st>>>(X, Y, N, Fr, l.cvp, dt, c->d_status);
        vp_first = 0;
      } else {
        k_gneb_update<R><<<gupd, kPT, 0, st>>>(X, Y, N, coefR, dt, slot, c->d_status);
      }
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::swap(X, Y);
    ++it;
    if (measure) {
      unsigned long long bits = 0;
      if ((e = cudaMemcpyAsync(&bits, l.fmax, sizeof(bits), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
      memcpy(&fmax, &bits, sizeof(fmax));
      if (fmax < p->tol || !(fmax == fmax)) break;
    }
  }
  // energies of the final chain (the tangent sums computed alongside are unused)
  if ((e = field(c, X + stride, Y + stride, M - 2, stride, true, st)) != cudaSuccess) return e;
  k_path_reduce<R, MODE_FULL><<<gred, kPT, 0, st>>>(X, Y, N, c->geo.ncell, nsub, zr, 0, 1, l.partial);
  k_path_sum<<<M - 1, kPT, 0, st>>>(l.partial, nb, 0, l.sums);
  k_path_coef<<<1, kPT, 0, st>>>(l.sums, l.eend, M, SX_PATH_GNEB, 0.0, l.coef, l.coeff, l.E, l.L);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (X != img &&
      (e = cudaMemcpyAsync(img + stride, X + stride, ibytes * (M - 2), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
    return e;
  if (E_host && (e = cudaMemcpyAsync(E_host, l.E, sizeof(double) * M, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  if (vp) c->path_vp_nimg = M;
  if (iters_out) *iters_out = it;
  if (fmax_host) *fmax_host = fmax;
  return cudaSuccess;
}

}  // namespace

int path_max_images() { return kMaxImg; }

cudaError_t path_run(sx_ctx *c, double *img, int nimg, const sx_path_params *p, int *iters_out, double *E_host,
                     double *fmax_host, cudaStream_t st, FieldBatchFn field) {
  if (c->prec == SX_PREC_FP64) return run_path<double>(c, img, nimg, p, iters_out, E_host, fmax_host, st, field);
  return run_path<float>(c, img, nimg, p, iters_out, E_host, fmax_host, st, field);
}

cudaError_t geodesic(const sx_ctx *c, const double *A, const double *B, double *out_host, cudaStream_t st) {
  const long long N = c->geo.nsite;
  const int nb = (int)std::min<long long>(c->nblock_red, reduce_grid(N));
  double *out = c->d_partial + 3 * c->nblock_red;
  k_geo_pair<<<nb, kPT, 0, st>>>(A, B, N, c->d_partial);
  k_geo_final<<<1, kPT, 0, st>>>(c->d_partial, nb, out);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, out, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

}  // namespace sx
