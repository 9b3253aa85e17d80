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
// on the device, so an iteration needs no host synchronisation.
// Damped LLG: normalised Heun steps at T = 0 with the given damping.
// Convergence: max_i |S_i x b_i| below tol, checked every check_every iterations.
#include <math.h>
#include <string.h>

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

// tangent force, velocity half-update and per-block partial sums of v.f and f.f
__global__ void __launch_bounds__(kMinThreads) k_vp_force(const double *__restrict__ S, const double *__restrict__ b,
                                                          double *__restrict__ v, double *__restrict__ fprev,
                                                          int first, double dt, long long N,
                                                          double *__restrict__ partial) {
  __shared__ double sm[kMinThreads];
  double p = 0.0, F2 = 0.0;
  for (long long i = (long long)blockIdx.x * kMinThreads + threadIdx.x; i < N;
       i += (long long)gridDim.x * kMinThreads) {
    const double s0 = S[i], s1 = S[N + i], s2 = S[2 * N + i];
    const double b0 = b[i], b1 = b[N + i], b2 = b[2 * N + i];
    const double d = b0 * s0 + b1 * s1 + b2 * s2;
    const double f[3] = {b0 - d * s0, b1 - d * s1, b2 - d * s2};
    for (int k = 0; k < 3; ++k) {
      const long long j = k * N + i;
      const double vk = first ? 0.0 : v[j] + 0.5 * dt * (fprev[j] + f[k]);
      v[j] = vk;
      fprev[j] = f[k];
      p += vk * f[k];
      F2 += f[k] * f[k];
    }
  }
  p = block_sum_d(p, sm);
  F2 = block_sum_d(F2, sm);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = p;
    partial[2 * blockIdx.x + 1] = F2;
  }
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
  if (threadIdx.x == 0) coef[0] = (p > 0.0 && F2 > 0.0) ? p / F2 : 0.0;
}

__global__ void __launch_bounds__(kMinThreads) k_vp_update(double *__restrict__ S, double *__restrict__ v,
                                                           const double *__restrict__ f,
                                                           const double *__restrict__ coef, double dt,
                                                           long long N) {
  const long long i = (long long)blockIdx.x * kMinThreads + threadIdx.x;
  if (i >= N) return;
  const double c = coef[0];
  double u[3], s[3] = {S[i], S[N + i], S[2 * N + i]};
  for (int k = 0; k < 3; ++k) {
    const double fk = f[k * N + i];
    v[k * N + i] = c * fk;
    u[k] = dt * c * fk + 0.5 * dt * dt * fk;
  }
  const double a = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  if (a > 0.0) {
    const double cs = cos(a), sn = sin(a) / a;
    for (int k = 0; k < 3; ++k) s[k] = cs * s[k] + sn * u[k];
    const double r = rsqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    for (int k = 0; k < 3; ++k) S[k * N + i] = s[k] * r;
  }
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
  double *v = c->d_min, *fp = c->d_min ? c->d_min + 3 * N : nullptr;
  double *part = c->d_min ? c->d_min + 6 * N : nullptr, *coef = part ? part + 2 * nb : nullptr;
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
      k_vp_force<<<nb, kMinThreads, 0, st>>>(cur, c->d_field, v, fp, it == 0 ? 1 : 0, p->dt, N, part);
      k_vp_coef<<<1, kMinThreads, 0, st>>>(part, nb, coef);
      k_vp_update<<<(unsigned)((N + kMinThreads - 1) / kMinThreads), kMinThreads, 0, st>>>(cur, v, fp, coef, p->dt,
                                                                                        N);
      e = cudaGetLastError();
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
      if (e != cudaSuccess || torque < p->tol) break;
    }
  }
  if (e == cudaSuccess && cur != S)
    e = cudaMemcpyAsync(S, cur, 3 * (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "minimise");
  if (iters_out) *iters_out = it;
  if (torque_out) *torque_out = torque;
  return SX_OK;
}

}  // namespace sx
