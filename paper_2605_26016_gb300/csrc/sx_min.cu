// Static minimisation on the product of unit spheres ("Static optimization and
// minimum-energy paths"): the tangent gradient G_i = grad_i H - (grad_i H . S_i) S_i,
// i.e. the tangent force f_i = b_i - (b_i . S_i) S_i, and the exponential-map
// retraction R(S, u) = cos|u| S + sin|u| u/|u|.
//
// Velocity projection (VP): per iteration
//   v <- v + dt/2 (f_prev + f)          (v = 0 on the first iteration)
//   v <- max(v.f, 0) / (f.f) f          (dot products over the whole system)
//   S <- R_exp(S, dt v + dt^2/2 f)
// The two global sums are reduced on the device and the step coefficient stays
// on the device, so an iteration needs no host synchronisation.  FP64 plans do
// every step in FP64; FP32-field plans keep v and f in FP32, reduce in FP32
// per warp and FP64 per block, and apply the retraction in FP32 with the state
// sum and renormalisation in FP64.
// Damped LLG: normalised Heun steps at T = 0 with the given damping.
// Convergence: max_i |S_i x b_i| below tol, checked every check_every iterations.
#include <math.h>
#include <string.h>

#include <cmath>

#include "sx_device.cuh"
#include "sx_internal.h"

namespace sx {

namespace {

constexpr int kMinThreads = 256;

__device__ __forceinline__ double block_sum_d(double v, double *sm) {
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int s = kMinThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sm[0];
  __syncthreads();
  return r;
}

// Sum of two per-thread values of type R over the block: shuffle trees in R,
// warp sums widened and added in FP64 by thread 0 (written to out[0], out[1]).
template <typename R>
__device__ __forceinline__ void block_sum2(R a, R b, double *out) {
  __shared__ double red[2][kMinThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = cvt<double>(a);
    red[1][threadIdx.x >> 5] = cvt<double>(b);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int w = 0; w < kMinThreads / 32; ++w) {
      x += red[0][w];
      y += red[1][w];
    }
    out[0] = x;
    out[1] = y;
  }
}

// tangent force, velocity half-update and per-block partial sums of v.f and f.f.
// R: arithmetic and storage type of v and f (FP64 plans: double; FP32-field plans: float).
template <typename R>
__global__ void __launch_bounds__(kMinThreads) k_vp_force(const double *__restrict__ S, const double *__restrict__ b,
                                                          R *__restrict__ v, R *__restrict__ fprev, int first, R hdt,
                                                          long long N, double *__restrict__ partial) {
  R p = 0, F2 = 0;
  for (long long i = (long long)blockIdx.x * kMinThreads + threadIdx.x; i < N;
       i += (long long)gridDim.x * kMinThreads) {
    const R s0 = cvt<R>(S[i]), s1 = cvt<R>(S[N + i]), s2 = cvt<R>(S[2 * N + i]);
    const R b0 = cvt<R>(b[i]), b1 = cvt<R>(b[N + i]), b2 = cvt<R>(b[2 * N + i]);
    const R d = b0 * s0 + b1 * s1 + b2 * s2;
    const R f[3] = {b0 - d * s0, b1 - d * s1, b2 - d * s2};
    // loads of all three components before the stores through the same pointers
    R vo[3] = {0, 0, 0}, fo[3] = {0, 0, 0};
    if (!first)
      for (int k = 0; k < 3; ++k) {
        vo[k] = v[k * N + i];
        fo[k] = fprev[k * N + i];
      }
    for (int k = 0; k < 3; ++k) {
      const R vk = first ? (R)0 : vo[k] + hdt * (fo[k] + f[k]);
      v[k * N + i] = vk;
      fprev[k * N + i] = f[k];
      p += vk * f[k];
      F2 += f[k] * f[k];
    }
  }
  block_sum2<R>(p, F2, partial + 2 * blockIdx.x);
}

__global__ void __launch_bounds__(kMinThreads) k_vp_coef(const double *__restrict__ partial, int nb,
                                                         double *__restrict__ coef) {
  __shared__ double sm[kMinThreads];
  double p = 0.0, F2 = 0.0;
  for (int j = threadIdx.x; j < nb; j += kMinThreads) {
    p += partial[2 * j];
    F2 += partial[2 * j + 1];
  }
  p = block_sum_d(p, sm);
  F2 = block_sum_d(F2, sm);
  if (threadIdx.x == 0) {
    const double c = (p > 0.0 && F2 > 0.0) ? p / F2 : 0.0;
    coef[0] = c;
    reinterpret_cast<float *>(coef + 1)[0] = (float)c;  // the same coefficient for FP32 plans
  }
}

// S <- R_exp(S, u), u tangent: FP64 plans in FP64 (libm cos, sin).  Returns true
// when the result is not finite or has zero length (a numeric error).
__device__ __forceinline__ bool vp_retract(double s[3], const double u[3]) {
  const double a = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  if (a > 0.0) {
    const double cs = cos(a), sn = sin(a) / a;
    for (int k = 0; k < 3; ++k) s[k] = cs * s[k] + sn * u[k];
    return unit64_checked(s);
  }
  return !(a == 0.0);  // NaN step
}

// FP32 arithmetic, FP64 state: d = (cos a - 1) s + (sin a / a) u with cos a - 1 = -2 sin^2(a/2),
// S' = N[S + d] in FP64
__device__ __forceinline__ bool vp_retract(double s[3], const float u[3]) {
  const float a = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  if (a > 0.0f) {
    const float sf[3] = {f64_to_f32(s[0]), f64_to_f32(s[1]), f64_to_f32(s[2])};
    const float h = sinf(0.5f * a);
    const float c1 = -2.0f * h * h, sc = sinf(a) / a;
    const float d[3] = {c1 * sf[0] + sc * u[0], c1 * sf[1] + sc * u[1], c1 * sf[2] + sc * u[2]};
    const double s0[3] = {s[0], s[1], s[2]};
    return renormalise64(s0, d, s);
  }
  return !(a == 0.0f);  // NaN step
}

template <typename R>
__global__ void __launch_bounds__(kMinThreads) k_vp_update(double *__restrict__ S, R *__restrict__ v,
                                                           const R *__restrict__ f, const double *__restrict__ coef,
                                                           R dt, long long N, int *__restrict__ status) {
  const long long i = (long long)blockIdx.x * kMinThreads + threadIdx.x;
  if (i >= N) return;
  R c;
  if constexpr (sizeof(R) == 8)
    c = coef[0];
  else
    c = reinterpret_cast<const float *>(coef + 1)[0];
  const R hdt2 = (R)0.5 * dt * dt;
  R u[3];
  double s[3] = {S[i], S[N + i], S[2 * N + i]};
  for (int k = 0; k < 3; ++k) {
    const R fk = f[k * N + i];
    v[k * N + i] = c * fk;
    u[k] = dt * c * fk + hdt2 * fk;
  }
  report_numeric(status, vp_retract(s, u));
  for (int k = 0; k < 3; ++k) S[k * N + i] = s[k];
}

template <typename R>
cudaError_t vp_iteration(const sx_ctx *c, double *S, double *ws, int first, double dt, int nb, cudaStream_t st) {
  const long long N = c->geo.nsite;
  R *v = reinterpret_cast<R *>(ws), *fp = v + 3 * N;
  double *part = ws + 6 * N, *coef = part + 2 * nb;
  k_vp_force<R><<<nb, kMinThreads, 0, st>>>(S, c->d_field, v, fp, first, (R)(0.5 * dt), N, part);
  k_vp_coef<<<1, kMinThreads, 0, st>>>(part, nb, coef);
  k_vp_update<R><<<(unsigned)((N + kMinThreads - 1) / kMinThreads), kMinThreads, 0, st>>>(S, v, fp, coef, (R)dt, N,
                                                                                              c->d_status);
  return cudaGetLastError();
}

}  // namespace

int minimise(sx_ctx *c, double *S, double *S_scratch, const sx_min_params *p, int *iters_out, double *torque_out,
             cudaStream_t st, cudaError_t (*field)(const sx_ctx *, const double *, double *, bool, cudaStream_t),
             cudaError_t (*step)(const sx_ctx *, const double *, double *, const HeunConst &, uint64_t,
                                 cudaStream_t)) {
  const long long N = c->geo.nsite;
  const int nb = (int)reduce_blocks(N);
  double *out_dev = c->d_partial + 3 * c->nblock_red;
  cudaError_t e = cudaSuccess;
  if (p->method == SX_MIN_VP && !c->d_min) {
    e = cudaMalloc(&c->d_min, (6 * (size_t)N + 2 * (size_t)nb + 8) * sizeof(double));
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc minimiser workspace");
  }
  HeunConst h;
  memset(&h, 0, sizeof(h));
  h.dt = p->dt;
  h.alpha = p->alpha;
  h.g = -kGamma / (1.0 + p->alpha * p->alpha);
  double torque = -1.0;
  int it = 0;
  double *cur = S, *other = S_scratch;
  while (it < p->max_iter) {
    if (p->method == SX_MIN_VP) {
      e = field(c, cur, c->d_field, true, st);
      if (e != cudaSuccess) break;
      e = c->prec == SX_PREC_FP64 ? vp_iteration<double>(c, cur, c->d_min, it == 0 ? 1 : 0, p->dt, nb, st)
                                  : vp_iteration<float>(c, cur, c->d_min, it == 0 ? 1 : 0, p->dt, nb, st);
    } else {
      e = step(c, cur, other, h, (uint64_t)it, st);
      double *t = cur;
      cur = other;
      other = t;
    }
    if (e != cudaSuccess) break;
    ++it;
    if (it % p->check_every == 0 || it == p->max_iter) {
      e = field(c, cur, c->d_field, true, st);
      if (e == cudaSuccess) e = reduce_torque(c, cur, c->d_field, c->d_partial, c->nblock_red, out_dev, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&torque, out_dev, sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess || torque < p->tol || !(torque == torque)) break;
    }
  }
  if (e == cudaSuccess && cur != S)
    e = cudaMemcpyAsync(S, cur, 3 * (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "minimise");
  if (iters_out) *iters_out = it;
  if (torque_out) *torque_out = torque;
  const int rc = take_status(c, st);
  if (rc != SX_OK) return rc;
  if (!std::isfinite(torque) && torque != -1.0)
    return set_error(SX_ERR_NUMERIC, "the torque maximum is not finite: the spin state holds a non-finite value");
  return SX_OK;
}

}  // namespace sx
