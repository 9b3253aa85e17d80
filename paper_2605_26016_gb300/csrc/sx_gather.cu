// Gather backend: every thread evaluates the reduced field of one site by
// walking the directed-bond table of its sublattice,
//   b_a^alpha(R) = sum_b sum_delta sum_beta K_ab^{alpha beta}(delta) S_b^beta(R + delta)
// ("Backend representations", multi-channel convolution), plus the Zeeman
// and anisotropy terms ("Spin Hamiltonian and effective fields").  It serves
// any interaction range and any lattice, and is the reference GPU realisation
// the faster backends are checked against.  The Heun step runs as two passes
// (predictor, corrector) with the predictor state in a workspace.
//
// Also here: the FP64 energy and torque reductions and the noise probe.
#include "sx_device.cuh"
#include "sx_internal.h"
#include "sx_noise.cuh"

namespace sx {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void site_of(const Geo &g, int64_t i, int &x, int &y, int &z, int &a) {
  int64_t t = i;
  x = (int)(t % g.nx);
  t /= g.nx;
  y = (int)(t % g.ny);
  t /= g.ny;
  z = (int)(t % g.nz);
  a = (int)(t / g.nz);
}

// wrap coordinate c into [0, n) on a periodic axis; -1 if it left an open axis
__device__ __forceinline__ int wrap(int c, int n, int periodic) {
  if (c >= 0 && c < n) return c;
  if (!periodic) return -1;
  c %= n;
  return c < 0 ? c + n : c;
}

template <typename R>
__device__ __forceinline__ R tapJ(const DevTap &t, int k);
template <>
__device__ __forceinline__ double tapJ<double>(const DevTap &t, int k) {
  return t.J[k];
}
template <>
__device__ __forceinline__ float tapJ<float>(const DevTap &t, int k) {
  return t.Jf[k];
}

template <typename R>
__device__ __forceinline__ void bilinear(const Geo &g, const DevTap *__restrict__ taps, const int *__restrict__ off,
                                         const double *__restrict__ S, int x, int y, int z, int a, R acc[3]) {
  acc[0] = acc[1] = acc[2] = R(0);
  const int t1 = off[a + 1];
  for (int t = off[a]; t < t1; ++t) {
    const DevTap &tp = taps[t];
    const int xx = wrap(x + tp.dx, g.nx, g.px);
    const int yy = wrap(y + tp.dy, g.ny, g.py);
    const int zz = wrap(z + tp.dz, g.nz, g.pz);
    if ((xx | yy | zz) < 0) continue;
    const int64_t j = (((int64_t)tp.b * g.nz + zz) * g.ny + yy) * g.nx + xx;
    const R s0 = cvt<R>(S[j]), s1 = cvt<R>(S[g.nsite + j]), s2 = cvt<R>(S[2 * g.nsite + j]);
    if (tp.iso) {
      const R J = tapJ<R>(tp, 0);
      acc[0] += J * s0;
      acc[1] += J * s1;
      acc[2] += J * s2;
    } else {
      acc[0] += tapJ<R>(tp, 0) * s0 + tapJ<R>(tp, 1) * s1 + tapJ<R>(tp, 2) * s2;
      acc[1] += tapJ<R>(tp, 3) * s0 + tapJ<R>(tp, 4) * s1 + tapJ<R>(tp, 5) * s2;
      acc[2] += tapJ<R>(tp, 6) * s0 + tapJ<R>(tp, 7) * s1 + tapJ<R>(tp, 8) * s2;
    }
  }
}

// Zeeman mu mu_B B and anisotropy 2K (S.n) n, added in precision R
template <typename R>
__device__ __forceinline__ void onsite_add(const OnSiteT<R> &os, int a, const R s[3], R b[3]) {
  const R n0 = os.axis[a][0], n1 = os.axis[a][1], n2 = os.axis[a][2];
  const R p = os.twoK[a] * (s[0] * n0 + s[1] * n1 + s[2] * n2);
  b[0] += os.zee[a][0] + p * n0;
  b[1] += os.zee[a][1] + p * n1;
  b[2] += os.zee[a][2] + p * n2;
}

// LLG right-hand side f = g [S x B + alpha S x (S x B)], g = -gamma/(1+alpha^2)
template <typename R>
__device__ __forceinline__ void llg_rhs(const R s[3], const R B[3], R g, R alpha, R f[3]) {
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

__device__ __forceinline__ void unit(float x[3]) {
  const float n2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  float r = rsqrtf(n2);
  r = r * (1.5f - 0.5f * n2 * r * r);
  x[0] *= r;
  x[1] *= r;
  x[2] *= r;
}
__device__ __forceinline__ void unit(double x[3]) {
  const double r = rsqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  x[0] *= r;
  x[1] *= r;
  x[2] *= r;
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_field(Geo g, const DevTap *__restrict__ taps,
                                                    const int *__restrict__ off, OnSiteT<R> os, int onsite,
                                                    const double *__restrict__ S, double *__restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i >= g.nsite) return;
  int x, y, z, a;
  site_of(g, i, x, y, z, a);
  R acc[3];
  bilinear<R>(g, taps, off, S, x, y, z, a, acc);
  if (onsite) {
    const R s[3] = {cvt<R>(S[i]), cvt<R>(S[g.nsite + i]), cvt<R>(S[2 * g.nsite + i])};
    onsite_add<R>(os, a, s, acc);
  }
  b[i] = cvt<double>(acc[0]);
  b[g.nsite + i] = cvt<double>(acc[1]);
  b[2 * g.nsite + i] = cvt<double>(acc[2]);
}

template <typename R>
__device__ __forceinline__ void thermal(const HeunT<R> &h, int a, int64_t i, uint64_t step, R th[3]) {
  th[0] = th[1] = th[2] = R(0);
  if (h.thermal) {
    float e0, e1, e2;
    normals3(h.seed, h.replica, (uint64_t)i, step, e0, e1, e2);
    const R sg = h.sigma[a];
    th[0] = sg * cvt<R>(e0);
    th[1] = sg * cvt<R>(e1);
    th[2] = sg * cvt<R>(e2);
  }
}

// Predictor: S~ = N[S + dt f(S)], f0 kept for the corrector.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_predict(Geo g, const DevTap *__restrict__ taps,
                                                      const int *__restrict__ off, OnSiteT<R> os, HeunT<R> h,
                                                      uint64_t step, const double *__restrict__ S,
                                                      double *__restrict__ St, double *__restrict__ F0) {
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i >= g.nsite) return;
  int x, y, z, a;
  site_of(g, i, x, y, z, a);
  R b[3];
  bilinear<R>(g, taps, off, S, x, y, z, a, b);
  const R s[3] = {cvt<R>(S[i]), cvt<R>(S[g.nsite + i]), cvt<R>(S[2 * g.nsite + i])};
  onsite_add<R>(os, a, s, b);
  R th[3];
  thermal<R>(h, a, i, step, th);
  const R im = os.inv_mm[a];
  const R B[3] = {b[0] * im + th[0], b[1] * im + th[1], b[2] * im + th[2]};
  R f[3];
  llg_rhs<R>(s, B, h.g, h.alpha, f);
  const R dt = h.dt;
  R xn[3] = {s[0] + dt * f[0], s[1] + dt * f[1], s[2] + dt * f[2]};
  unit(xn);
  for (int k = 0; k < 3; ++k) {
    St[k * g.nsite + i] = cvt<double>(xn[k]);
    F0[k * g.nsite + i] = cvt<double>(f[k]);
  }
}

// Corrector: S' = N[S + dt/2 (f(S) + f(S~))]; the state sum and N[.] in FP64.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_correct(Geo g, const DevTap *__restrict__ taps,
                                                      const int *__restrict__ off, OnSiteT<R> os, HeunT<R> h,
                                                      uint64_t step, const double *__restrict__ S,
                                                      const double *__restrict__ St, const double *__restrict__ F0,
                                                      double *__restrict__ Snew, int *__restrict__ status) {
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i >= g.nsite) return;
  int x, y, z, a;
  site_of(g, i, x, y, z, a);
  R b[3];
  bilinear<R>(g, taps, off, St, x, y, z, a, b);
  const R s[3] = {cvt<R>(St[i]), cvt<R>(St[g.nsite + i]), cvt<R>(St[2 * g.nsite + i])};
  onsite_add<R>(os, a, s, b);
  R th[3];
  thermal<R>(h, a, i, step, th);
  const R im = os.inv_mm[a];
  const R B[3] = {b[0] * im + th[0], b[1] * im + th[1], b[2] * im + th[2]};
  R f[3];
  llg_rhs<R>(s, B, h.g, h.alpha, f);
  const R hdt = h.hdt;
  R d[3];
  double s64[3], xn[3];
  for (int k = 0; k < 3; ++k) {
    d[k] = hdt * (cvt<R>(F0[k * g.nsite + i]) + f[k]);
    s64[k] = S[k * g.nsite + i];
  }
  if constexpr (sizeof(R) == 4) {
    report_numeric(status, renormalise64(s64, d, xn));
  } else {
    for (int k = 0; k < 3; ++k) xn[k] = s64[k] + d[k];
    report_numeric(status, unit64_checked(xn));
  }
  for (int k = 0; k < 3; ++k) Snew[k * g.nsite + i] = xn[k];
}

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ double block_sum(double v, double *sm) {
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sm[0];
  __syncthreads();
  return r;
}

// per-block partial energies: [bilinear, Zeeman, anisotropy]
__global__ void __launch_bounds__(kThreads) k_energy_partial(Geo g, OnSite os, const double *__restrict__ S,
                                                             const double *__restrict__ bb,
                                                             double *__restrict__ partial) {
  __shared__ double sm[kThreads];
  double eb = 0.0, ez = 0.0, ea = 0.0;
  const int64_t N = g.nsite;
  const int64_t per = g.nx * (int64_t)g.ny * g.nz;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < N; i += (int64_t)gridDim.x * kThreads) {
    const int a = (int)(i / per);
    const double s0 = S[i], s1 = S[N + i], s2 = S[2 * N + i];
    eb += -0.5 * (s0 * bb[i] + s1 * bb[N + i] + s2 * bb[2 * N + i]);
    ez += -(os.zee[a][0] * s0 + os.zee[a][1] * s1 + os.zee[a][2] * s2);
    const double p = s0 * os.axis[a][0] + s1 * os.axis[a][1] + s2 * os.axis[a][2];
    ea += -0.5 * os.twoK[a] * p * p;
  }
  eb = block_sum(eb, sm);
  ez = block_sum(ez, sm);
  ea = block_sum(ea, sm);
  if (threadIdx.x == 0) {
    partial[3 * blockIdx.x + 0] = eb;
    partial[3 * blockIdx.x + 1] = ez;
    partial[3 * blockIdx.x + 2] = ea;
  }
}

// out = [total, bilinear, Zeeman, anisotropy, dipolar(0)]
__global__ void __launch_bounds__(kThreads) k_energy_final(const double *__restrict__ partial, int64_t nb,
                                                           double *__restrict__ out) {
  __shared__ double sm[kThreads];
  double v[3];
  for (int k = 0; k < 3; ++k) {
    double acc = 0.0;
    for (int64_t j = threadIdx.x; j < nb; j += kThreads) acc += partial[3 * j + k];
    v[k] = block_sum(acc, sm);
  }
  if (threadIdx.x == 0) {
    out[1] = v[0];
    out[2] = v[1];
    out[3] = v[2];
    out[4] = 0.0;
    out[0] = v[0] + v[1] + v[2];
  }
}

__global__ void __launch_bounds__(kThreads) k_torque_partial(Geo g, const double *__restrict__ S,
                                                             const double *__restrict__ b,
                                                             double *__restrict__ partial) {
  __shared__ double sm[kThreads];
  const double best = block_torque_max<kThreads>(S, b, g.nsite, sm);
  if (threadIdx.x == 0) partial[blockIdx.x] = best;
}

__global__ void __launch_bounds__(kThreads) k_torque_final(const double *__restrict__ partial, int64_t nb,
                                                           double *__restrict__ out) {
  __shared__ double sm[kThreads];
  double best = 0.0;
  for (int64_t j = threadIdx.x; j < nb; j += kThreads) best = max_nan(best, partial[j]);
  best = block_max_nan<kThreads>(best, sm);
  if (threadIdx.x == 0) out[0] = best;
}

__global__ void k_normals(uint64_t seed, uint32_t replica, uint64_t site0, int64_t n, uint64_t step,
                          float *__restrict__ eta) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  float e0, e1, e2;
  normals3(seed, replica, site0 + (uint64_t)k, step, e0, e1, e2);
  eta[3 * k] = e0;
  eta[3 * k + 1] = e1;
  eta[3 * k + 2] = e2;
}

inline unsigned grid_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// out[i] = (float)in[i], round to nearest (IEEE conversion)
__global__ void __launch_bounds__(kThreads) k_to_f32(const double *__restrict__ in, float *__restrict__ out,
                                                     int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    out[i] = __double2float_rn(in[i]);
}

}  // namespace

int64_t reduce_blocks(int64_t nsite) {
  int64_t nb = (nsite + kThreads - 1) / kThreads;
  return nb < 152 * 8 ? nb : 152 * 8;
}

cudaError_t gather_field(const sx_ctx *c, const double *S, double *b, bool onsite, cudaStream_t st) {
  const Geo &g = c->geo;
  if (c->prec == SX_PREC_FP64)
    k_field<double><<<grid_for(g.nsite), kThreads, 0, st>>>(g, c->d_taps, c->d_tap_off, onsite_cast<double>(c->onsite),
                                                            onsite, S, b);
  else
    k_field<float><<<grid_for(g.nsite), kThreads, 0, st>>>(g, c->d_taps, c->d_tap_off, onsite_cast<float>(c->onsite),
                                                           onsite, S, b);
  return cudaGetLastError();
}

cudaError_t gather_heun_step(const sx_ctx *c, const double *src, double *dst, const HeunConst &h, uint64_t step,
                             cudaStream_t st) {
  const Geo &g = c->geo;
  double *St = c->d_work;
  double *F0 = c->d_work + 3 * g.nsite;
  if (c->prec == SX_PREC_FP64) {
    k_predict<double><<<grid_for(g.nsite), kThreads, 0, st>>>(g, c->d_taps, c->d_tap_off, onsite_cast<double>(c->onsite),
                                                              heun_cast<double>(h), step, src,
                                                              St, F0);
    k_correct<double><<<grid_for(g.nsite), kThreads, 0, st>>>(g, c->d_taps, c->d_tap_off, onsite_cast<double>(c->onsite),
                                                              heun_cast<double>(h), step, src,
                                                              St, F0, dst, c->d_status);
  } else {
    k_predict<float><<<grid_for(g.nsite), kThreads, 0, st>>>(g, c->d_taps, c->d_tap_off, onsite_cast<float>(c->onsite),
                                                              heun_cast<float>(h), step, src,
                                                             St, F0);
    k_correct<float><<<grid_for(g.nsite), kThreads, 0, st>>>(g, c->d_taps, c->d_tap_off, onsite_cast<float>(c->onsite),
                                                              heun_cast<float>(h), step, src,
                                                             St, F0, dst, c->d_status);
  }
  return cudaGetLastError();
}

cudaError_t reduce_energy(const sx_ctx *c, const double *S, const double *bbil, double *partial, int64_t nblock,
                          double *out_dev, cudaStream_t st) {
  k_energy_partial<<<(unsigned)nblock, kThreads, 0, st>>>(c->geo, c->onsite, S, bbil, partial);
  k_energy_final<<<1, kThreads, 0, st>>>(partial, nblock, out_dev);
  return cudaGetLastError();
}

cudaError_t reduce_torque(const sx_ctx *c, const double *S, const double *b, double *partial, int64_t nblock,
                          double *out_dev, cudaStream_t st) {
  k_torque_partial<<<(unsigned)nblock, kThreads, 0, st>>>(c->geo, S, b, partial);
  k_torque_final<<<1, kThreads, 0, st>>>(partial, nblock, out_dev);
  return cudaGetLastError();
}

cudaError_t to_f32(const double *in, float *out, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t nb = std::min<int64_t>(grid_for(n), 152 * 16);
  k_to_f32<<<(unsigned)nb, kThreads, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t thermal_normals(uint64_t seed, uint32_t replica, uint64_t site0, int64_t n, uint64_t step, float *eta,
                            cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_normals<<<grid_for(n), kThreads, 0, st>>>(seed, replica, site0, n, step, eta);
  return cudaGetLastError();
}

}  // namespace sx
