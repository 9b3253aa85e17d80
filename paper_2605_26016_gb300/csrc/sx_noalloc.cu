// max_i |S_i x b_i| without any device allocation.
//
// Who needs this: a caller that owns every byte of device memory itself.
// Examples are an application that reserves the whole GPU up front through its
// own arena, and a time-step loop that must not pay the implicit device
// synchronisation and latency of cudaMalloc/cudaFree.  Such a caller cannot let
// a library allocate reduction scratch behind its back.  The regular
// sx_torque_max keeps its scratch in a workspace that sx_plan allocates; this
// variant needs no context and no plan.  It keeps its per-block partial maxima
// in a fixed array in device memory that is part of the loaded library image.
//
// The array, g_torque_partials, is kStaticBlocks + 1 doubles (9.7 KB).  Every
// GPU on which the library is loaded holds it until the process exits.  Host
// code may not pass the array's name to a kernel: on the host that name is only
// a stand-in, not a device address.  Every call looks the device address up
// with cudaGetSymbolAddress for the device and context current at the call, so
// an address never outlives the context it belongs to (after cudaDeviceReset,
// or with another context current on the same device, the lookup returns the
// array of the module loaded in the context now current).
//
// The reduction body (per-site torque, NaN-propagating block maximum) is the
// one sx_torque_max uses (sx_device.cuh); only the scratch location differs.
#include <cmath>

#include "sx_device.cuh"
#include "sx_internal.h"

namespace {

constexpr int kStaticThreads = 256;
constexpr int kStaticBlocks = 1216;               // grid cap: 152 SMs x 8 resident blocks
constexpr int64_t kMaxSites = (int64_t)1 << 40;  // the library's lattice limit

// slots 0 .. kStaticBlocks-1: per-block partial maxima; slot kStaticBlocks: the result
static __device__ __align__(256) double g_torque_partials[kStaticBlocks + 1];

__global__ void __launch_bounds__(kStaticThreads) k_torque_partial_static(const double *__restrict__ S,
                                                                          const double *__restrict__ b, int64_t n,
                                                                          double *__restrict__ partial) {
  __shared__ double sm[kStaticThreads];
  const double best = sx::block_torque_max<kStaticThreads>(S, b, n, sm);
  if (threadIdx.x == 0) partial[blockIdx.x] = best;
}

// reads exactly the nb slots the partial kernel of the same call wrote, so no
// slot has to be cleared between calls
__global__ void __launch_bounds__(kStaticThreads) k_torque_final_static(double *__restrict__ partial, int nb) {
  __shared__ double sm[kStaticThreads];
  double best = 0.0;
  for (int j = threadIdx.x; j < nb; j += kStaticThreads) best = sx::max_nan(best, partial[j]);
  best = sx::block_max_nan<kStaticThreads>(best, sm);
  if (threadIdx.x == 0) partial[kStaticBlocks] = best;
}

// device address of the static array in the context current now
int scratch_address(double **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_torque_partials);
  if (e != cudaSuccess) return sx::cuda_error(e, "cudaGetSymbolAddress");
  *out = static_cast<double *>(p);
  return SX_OK;
}

}  // namespace

extern "C" int sx_torque_max_noalloc(const double *S, const double *b, int64_t nsite, double *out_host,
                                     void *stream) {
  if (!S || !b || !out_host) return sx::set_error(SX_ERR_ARG, "null argument");
  if ((((uintptr_t)S) | ((uintptr_t)b)) & 7u) return sx::set_error(SX_ERR_ARG, "S and b must be 8-byte aligned");
  if (nsite < 1 || nsite > kMaxSites)
    return sx::set_error(SX_ERR_ARG, "nsite must be in 1 .. 2^40 for sx_torque_max_noalloc");
  const size_t bytes = 3 * (size_t)nsite * sizeof(double);
  const char *ps = (const char *)S, *pb = (const char *)b;
  if (ps < pb + bytes && pb < ps + bytes) return sx::set_error(SX_ERR_ARG, "S and b overlap");
  double *scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != SX_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t want = (nsite + kStaticThreads - 1) / kStaticThreads;
  const int nb = (int)(want < kStaticBlocks ? want : kStaticBlocks);
  k_torque_partial_static<<<nb, kStaticThreads, 0, st>>>(S, b, nsite, scratch);
  k_torque_final_static<<<1, kStaticThreads, 0, st>>>(scratch, nb);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, scratch + kStaticBlocks, sizeof(double),
                                            cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return sx::cuda_error(e, "sx_torque_max_noalloc");
  if (!std::isfinite(*out_host)) return sx::set_error(SX_ERR_NUMERIC, "non-finite spin or field value");
  return SX_OK;
}
