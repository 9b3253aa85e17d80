// Dense-convolution backend on the 5th-generation tensor cores (tcgen05).
//
// The dense backend of the paper evaluates the field as a convolution with a
// compact regular kernel ("Backend representations": dense convolution).  Here
// that convolution is an implicit GEMM per CTA, for one sublattice with scalar
// (isotropic) taps inside a (2R+1)^3 window, R <= 3:
//
//   b^alpha(x, y, z) = sum_{dy,dz} sum_dx J(dx, dy, dz) S^alpha(x + dx, y + dy, z + dz)
//
// For a fixed kernel plane (dy, dz) the x-sum is a banded Toeplitz matrix
// A_{dy,dz}[m][k] = J(k - R - m, dy, dz) (128 output x positions m, 144 input
// x positions k) applied to the spin rows S^alpha(x0 - R + k, y0 + dy + j, z0 +
// dz + i) of an 8 x 8 (y, z) block: D[128 x 64] += A[128 x 144] B[144 x 64].
// All planes accumulate into the same TMEM accumulator (FP32), one 64-column
// accumulator per spin component.
//
//  * B is one resident shared-memory tile per component: the input window
//    (144 x (8+2R) x (8+2R)) in the canonical no-swizzle K-major layout with
//    8 consecutive y rows per core matrix, so the operand of plane (dy, dz) is
//    the same tile seen from a different start address (16-byte rows).
//  * A of every non-zero plane (planes whose taps are all zero are skipped) is
//    built once per plan in global memory, already in the shared-memory
//    operand layout; the kernel streams the planes into a double buffer with
//    16-byte cp.async copies, the copy of plane p+1 overlapping the MMAs of p.
//  * One elected thread issues tcgen05.mma (kind::f16 for BF16, kind::tf32 for
//    TF32), tcgen05.commit arrives on an mbarrier; waits are bounded and set an
//    error flag instead of hanging.  The epilogue reads TMEM with tcgen05.ld.
//
// Executed MMA work per output component is 144 MACs per non-zero plane,
// against 2R+1 useful taps per plane: the band structure wastes most of each
// MMA, which the measurement reports next to the useful flops.
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "sx_device.cuh"
#include "sx_internal.h"

namespace sx {

// buffer-based Heun stages shared with the FFT backend (sx_fft.cu)
cudaError_t bufheun_predict(const sx_ctx *c, const double *S, const float *Bf, float *St, float *F0, float *Th,
                            const HeunConst &h, uint64_t step, cudaStream_t st);
cudaError_t bufheun_correct(const sx_ctx *c, const double *S, const float *St, const float *F0, const float *Bf,
                            const float *Th, double *Snew, const HeunConst &h, cudaStream_t st);

constexpr int kTcM = 128;      // output x per CTA (MMA M)
constexpr int kTcYB = 8;       // output y per CTA (one core-matrix row group)
constexpr int kTcZB = 8;       // output z per CTA
constexpr int kTcN = kTcYB * kTcZB;  // MMA N per component
constexpr int kTcKP = 144;     // input x window, padded to the MMA K granularity
constexpr int kTcRMax = 3;
constexpr int kTcThreads = 128;

struct TcArgs {
  int nx, ny, nz, px, py, pz;
  long long ncell;
  int R, nplanes;
  int plane_dy[49], plane_dz[49];
  float J[7][7][7];  // J[dz+3][dy+3][dx+3]
  float zee[3], twoK, axis[3];
  int onsite;
  int *err;          // set to 1 if a bounded wait gave up
  const unsigned char *A;  // Toeplitz operands of the planes, built once per plan in the
                           // shared-memory layout (tc_a_stride bytes per plane)
  int nabuf;               // shared-memory A buffers: 2 (copy of plane p+1 overlaps the MMAs of p) or 1
  unsigned smem;           // dynamic shared memory of the launch
};

struct TcPlan {
  int tf32;
  unsigned char *A;     // Toeplitz operands, nplanes x tc_a_stride bytes
  TcArgs base;
  float *St, *F0, *Bf;  // Heun workspaces [3][ncell]
  float *Th;            // thermal field of the step [3][ncell]
  int *err;
};

namespace {

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ uint32_t to_tf32(float f) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
  return r;
}

// TF32: one copy, rounded to nearest.  BF16: split representation v = hi + lo
// (both BF16, lo = RN(v - hi)), written to two copies of the operand.
template <bool TF32>
__device__ __forceinline__ void put_elem(unsigned char *base, size_t copy_stride, size_t off, float v) {
  if (TF32) {
    *reinterpret_cast<uint32_t *>(base + off) = to_tf32(v);
  } else {
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    *reinterpret_cast<__nv_bfloat16 *>(base + off) = hi;
    *reinterpret_cast<__nv_bfloat16 *>(base + copy_stride + off) = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

template <typename T>
__device__ __forceinline__ float as_f32(T v);
template <>
__device__ __forceinline__ float as_f32<double>(double v) {
  return f64_to_f32(v);
}
template <>
__device__ __forceinline__ float as_f32<float>(float v) {
  return v;
}

__device__ __forceinline__ bool wait_parity(uint64_t *mbar, uint32_t parity, int *err) {
  for (long it = 0; it < (1L << 24); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(saddr(mbar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it > 1024) __nanosleep(64);
  }
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit_tc() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all_tc() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// bytes of one plane's A operand (TF32: one copy; BF16: hi and lo copies)
template <bool TF32>
constexpr size_t tc_a_stride() {
  return (TF32 ? 1 : 2) * (size_t)kTcM * kTcKP * (TF32 ? 4 : 2);
}

// bytes of one copy of the resident input window for halo R: K chunks x (8+2R) x (8+2R) rows of 16 bytes
template <bool TF32>
__host__ __device__ constexpr size_t tc_b_copy(int R) {
  return (size_t)(kTcKP / (16 / (TF32 ? 4 : 2))) * (kTcZB + 2 * R) * (kTcYB + 2 * R) * 16;
}

// dynamic shared memory of a launch with nabuf A buffers
template <bool TF32>
constexpr size_t tc_smem_bytes(int R, int nabuf) {
  return (TF32 ? 1 : 2) * tc_b_copy<TF32>(R) + (size_t)nabuf * tc_a_stride<TF32>() + 64;
}

// Toeplitz A[m][k] = J(k - R - m, dy, dz) of plane blockIdx.x, in the canonical K-major
// no-swizzle layout the kernel hands to tcgen05.mma (plan time)
template <bool TF32>
__global__ void k_build_a(const TcArgs p, unsigned char *__restrict__ A) {
  constexpr int ESZ = TF32 ? 4 : 2;
  constexpr int EPC = 16 / ESZ;
  constexpr size_t A_COPY = (size_t)kTcM * kTcKP * ESZ;
  const int pl = blockIdx.x, dy = p.plane_dy[pl], dz = p.plane_dz[pl];
  unsigned char *dst = A + (size_t)pl * tc_a_stride<TF32>();
  for (int e = threadIdx.x; e < kTcM * kTcKP; e += blockDim.x) {
    const int k = e % kTcKP, m = e / kTcKP;
    const int dx = k - p.R - m;
    const float v = (dx >= -p.R && dx <= p.R) ? p.J[dz + 3][dy + 3][dx + 3] : 0.0f;
    put_elem<TF32>(dst, A_COPY, ((size_t)(k / EPC) * (kTcM / 8) + m / 8) * 128 + (size_t)(m % 8) * 16 + (size_t)(k % EPC) * ESZ,
                   v);
  }
}

// Field of one spin field (FP64 spins or FP32 predictor state) into out (FP64 or FP32),
// optional on-site terms.  Grid: (ceil(nx/128), ceil(ny/8), ceil(nz/8)), 128 threads.
template <bool TF32, typename Tin, typename Tout>
__global__ void __launch_bounds__(kTcThreads) k_field_tc(const TcArgs p, const Tin *__restrict__ S,
                                                         Tout *__restrict__ out) {
  constexpr int ESZ = TF32 ? 4 : 2;
  constexpr int EPC = 16 / ESZ;            // elements per 16-byte core-matrix row
  constexpr int KSTEP = TF32 ? 8 : 16;     // K per MMA instruction
  constexpr int CHUNKS = kTcKP / EPC;      // K chunks of the window
  extern __shared__ __align__(1024) unsigned char smem[];
  const int R = p.R;
  const int YR = kTcYB + 2 * R, ZR = kTcZB + 2 * R;
  const uint32_t SBO_B = (uint32_t)YR * 16u, LBO_B = (uint32_t)(ZR * YR) * 16u;
  const uint32_t LBO_A = (kTcM / 8) * 128u, SBO_A = 128u;
  // operand copies: TF32 one, BF16 two (hi, lo); each B copy spans CHUNKS * ZR * YR * 16 bytes
  constexpr int NCOPY = TF32 ? 1 : 2;
  const size_t B_COPY = tc_b_copy<TF32>(R);
  constexpr size_t A_COPY = (size_t)kTcM * kTcKP * ESZ;
  constexpr size_t A_STRIDE = tc_a_stride<TF32>();
  unsigned char *sB = smem;
  unsigned char *sAbuf = smem + NCOPY * B_COPY;  // nabuf plane buffers of A_STRIDE bytes
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sAbuf + p.nabuf * A_STRIDE);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * kTcM, y0 = blockIdx.y * kTcYB, z0 = blockIdx.z * kTcZB;

  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(mbar)));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(saddr(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  constexpr uint32_t fmt = TF32 ? 2u : 1u;
  constexpr uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                             ((uint32_t)(kTcM >> 4) << 24);
  uint32_t phase = 0;
  bool alive = true;

  for (int al = 0; al < 3 && alive; ++al) {
    // resident input window of component al: element (k, zg, yrow)
    const int nB = kTcKP * ZR * YR;
    for (int e = tid; e < nB; e += kTcThreads) {
      const int k = e % kTcKP;
      const int r = e / kTcKP;
      const int yrow = r % YR, zg = r / YR;
      float v = 0.0f;
      if (k < kTcM + 2 * R) {
        bool ok = true;
        const int gx = wrap_axis(x0 - R + k, p.nx, p.px, ok);
        const int gy = wrap_axis(y0 - R + yrow, p.ny, p.py, ok);
        const int gz = wrap_axis(z0 - R + zg, p.nz, p.pz, ok);
        if (ok) v = as_f32<Tin>(S[(long long)al * p.ncell + ((long long)gz * p.ny + gy) * p.nx + gx]);
      }
      put_elem<TF32>(sB, B_COPY, ((size_t)(k / EPC) * ZR + zg) * YR * 16 + (size_t)yrow * 16 + (size_t)(k % EPC) * ESZ,
                     v);
    }
    // A of plane pl into buffer pl % nabuf (16-byte copies from the L2-resident plan operands)
    auto copy_a = [&](int pl) {
      const unsigned char *src = p.A + (size_t)pl * A_STRIDE;
      unsigned char *dst = sAbuf + (size_t)(pl % p.nabuf) * A_STRIDE;
      for (int e = tid; e < (int)(A_STRIDE / 16); e += kTcThreads) cp_async16(saddr(dst + 16 * e), src + 16 * e);
      cp_commit_tc();
    };
    if (p.nplanes > 0) copy_a(0);
    for (int pl = 0; pl < p.nplanes && alive; ++pl) {
      const int dy = p.plane_dy[pl], dz = p.plane_dz[pl];
      unsigned char *sA = sAbuf + (size_t)(pl % p.nabuf) * A_STRIDE;
      cp_wait_all_tc();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t bstart = saddr(sB) + (uint32_t)(dz + R) * SBO_B + (uint32_t)(dy + R) * 16u;
        for (int ks = 0; ks < kTcKP / KSTEP; ++ks) {
          const uint32_t kc = (uint32_t)(ks * (KSTEP / EPC));
          const uint32_t d = tmem + (uint32_t)(al * kTcN);
          if (TF32) {
            const uint64_t ad = smem_desc(saddr(sA) + kc * LBO_A, LBO_A, SBO_A);
            const uint64_t bd = smem_desc(bstart + kc * LBO_B, LBO_B, SBO_B);
            const uint32_t acc = (pl > 0 || ks > 0) ? 1u : 0u;
            asm volatile(
                "{\n.reg .pred q;\nsetp.ne.u32 q, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n}\n" ::"r"(d),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          } else {
            // J S = Jh Sh + Jh Sl + Jl Sh (the Jl Sl term is below FP32 resolution of the sum)
            for (int t = 0; t < 3; ++t) {
              const uint32_t ac = (uint32_t)(t == 2 ? A_COPY : 0), bc = (uint32_t)(t == 1 ? B_COPY : 0);
              const uint64_t ad = smem_desc(saddr(sA) + ac + kc * LBO_A, LBO_A, SBO_A);
              const uint64_t bd = smem_desc(bstart + bc + kc * LBO_B, LBO_B, SBO_B);
              const uint32_t acc = (pl > 0 || ks > 0 || t > 0) ? 1u : 0u;
              asm volatile(
                  "{\n.reg .pred q;\nsetp.ne.u32 q, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(d),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(mbar))
                     : "memory");
      }
      // with two buffers the other one was read by the MMAs of plane pl - 1, which have completed
      if (p.nabuf == 2 && pl + 1 < p.nplanes) copy_a(pl + 1);
      // every thread waits for this plane's MMAs before its A buffer (and, after the last plane, B) is rewritten
      alive = wait_parity(mbar, phase, p.err);
      phase ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      __syncthreads();
      if (p.nabuf == 1 && pl + 1 < p.nplanes && alive) copy_a(pl + 1);
    }
  }

  if (alive && p.nplanes > 0) {
    // epilogue: row m = 32*warp + lane is output x = x0 + m; column n is (y0 + n%8, z0 + n/8)
    const int x = x0 + warp * 32 + lane;
    for (int c0 = 0; c0 < kTcN; c0 += 16) {
      float v[3][16];
#pragma unroll
      for (int al = 0; al < 3; ++al) {
        uint32_t r[16];
        const uint32_t a = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(al * kTcN + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(a));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) v[al][j] = __uint_as_float(r[j]);
      }
      if (x < p.nx) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = c0 + j;
          const int y = y0 + (n % kTcYB), z = z0 + (n / kTcYB);
          if (y >= p.ny || z >= p.nz) continue;
          const long long i = ((long long)z * p.ny + y) * p.nx + x;
          float b0 = v[0][j], b1 = v[1][j], b2 = v[2][j];
          if (p.onsite) {
            const float s0 = as_f32<Tin>(S[i]), s1 = as_f32<Tin>(S[p.ncell + i]), s2 = as_f32<Tin>(S[2 * p.ncell + i]);
            const float q = p.twoK * (s0 * p.axis[0] + s1 * p.axis[1] + s2 * p.axis[2]);
            b0 += p.zee[0] + q * p.axis[0];
            b1 += p.zee[1] + q * p.axis[1];
            b2 += p.zee[2] + q * p.axis[2];
          }
          out[i] = (Tout)b0;
          out[p.ncell + i] = (Tout)b1;
          out[2 * p.ncell + i] = (Tout)b2;
        }
      }
    }
  } else if (p.nplanes == 0) {
    // no bilinear taps: only the on-site terms
    for (int e = tid; e < kTcM * kTcN; e += kTcThreads) {
      const int x = x0 + e % kTcM, n = e / kTcM;
      const int y = y0 + (n % kTcYB), z = z0 + (n / kTcYB);
      if (x >= p.nx || y >= p.ny || z >= p.nz) continue;
      const long long i = ((long long)z * p.ny + y) * p.nx + x;
      float b[3] = {0.f, 0.f, 0.f};
      if (p.onsite) {
        const float s0 = as_f32<Tin>(S[i]), s1 = as_f32<Tin>(S[p.ncell + i]), s2 = as_f32<Tin>(S[2 * p.ncell + i]);
        const float q = p.twoK * (s0 * p.axis[0] + s1 * p.axis[1] + s2 * p.axis[2]);
        for (int k = 0; k < 3; ++k) b[k] = p.zee[k] + q * p.axis[k];
      }
      for (int k = 0; k < 3; ++k) out[k * p.ncell + i] = (Tout)b[k];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

constexpr size_t kTcSmemMax = 227 * 1024;

template <bool TF32, typename Tin, typename Tout>
cudaError_t launch_tc(const sx_ctx *c, const TcArgs &a, const Tin *S, Tout *out, cudaStream_t st) {
  const dim3 grid((c->geo.nx + kTcM - 1) / kTcM, (c->geo.ny + kTcYB - 1) / kTcYB, (c->geo.nz + kTcZB - 1) / kTcZB);
  k_field_tc<TF32, Tin, Tout><<<grid, kTcThreads, a.smem, st>>>(a, S, out);
  return cudaGetLastError();
}

template <bool TF32>
cudaError_t set_tc_smem() {
  const int s = (int)kTcSmemMax;
  cudaError_t e = cudaFuncSetAttribute(k_field_tc<TF32, double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_field_tc<TF32, double, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_field_tc<TF32, float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  return e;
}

}  // namespace

int tc_plan(sx_ctx *c) {
  if (c->prec != SX_PREC_BF16 && c->prec != SX_PREC_TF32)
    return set_error(SX_ERR_UNSUPPORTED, "the tensor-core backend computes the field in BF16 or TF32");
  if (c->lat.nsub != 1) return set_error(SX_ERR_UNSUPPORTED, "the tensor-core backend supports one sublattice");
  TcPlan *tp = new (std::nothrow) TcPlan();
  if (!tp) return set_error(SX_ERR_OOM, "host allocation failed");
  memset(tp, 0, sizeof(*tp));
  TcArgs &a = tp->base;
  a.nx = c->geo.nx;
  a.ny = c->geo.ny;
  a.nz = c->geo.nz;
  a.px = c->geo.px;
  a.py = c->geo.py;
  a.pz = c->geo.pz;
  a.ncell = c->geo.ncell;
  int R = 0;
  for (const Tap &t : c->taps[0]) {
    const bool iso = t.J[1] == 0.0 && t.J[2] == 0.0 && t.J[3] == 0.0 && t.J[5] == 0.0 && t.J[6] == 0.0 &&
                     t.J[7] == 0.0 && t.J[0] == t.J[4] && t.J[4] == t.J[8];
    if (!iso) {
      delete tp;
      return set_error(SX_ERR_UNSUPPORTED, "the tensor-core backend takes scalar (isotropic) taps only");
    }
    for (int k = 0; k < 3; ++k) {
      if (abs(t.d[k]) > kTcRMax) {
        delete tp;
        return set_error(SX_ERR_UNSUPPORTED, "the tensor-core backend takes taps within a 7x7x7 window");
      }
      R = std::max(R, abs(t.d[k]));
    }
    a.J[t.d[2] + 3][t.d[1] + 3][t.d[0] + 3] = (float)t.J[0];
  }
  a.R = R;
  for (int dz = -R; dz <= R; ++dz)
    for (int dy = -R; dy <= R; ++dy) {
      bool any = false;
      for (int dx = -R; dx <= R; ++dx) any = any || a.J[dz + 3][dy + 3][dx + 3] != 0.0f;
      if (any) {
        a.plane_dy[a.nplanes] = dy;
        a.plane_dz[a.nplanes] = dz;
        ++a.nplanes;
      }
    }
  for (int k = 0; k < 3; ++k) {
    a.zee[k] = (float)c->onsite.zee[0][k];
    a.axis[k] = (float)c->onsite.axis[0][k];
  }
  a.twoK = (float)c->onsite.twoK[0];
  tp->tf32 = c->prec == SX_PREC_TF32;
  const size_t n3 = 3 * (size_t)c->geo.ncell;
  cudaError_t e = cudaMalloc(&tp->St, n3 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&tp->F0, n3 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&tp->Bf, n3 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&tp->Th, n3 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&tp->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(tp->err, 0, sizeof(int));
  if (e == cudaSuccess) e = tp->tf32 ? set_tc_smem<true>() : set_tc_smem<false>();
  const size_t astride = tp->tf32 ? tc_a_stride<true>() : tc_a_stride<false>();
  const size_t sm2 = tp->tf32 ? tc_smem_bytes<true>(R, 2) : tc_smem_bytes<false>(R, 2);
  a.nabuf = sm2 <= kTcSmemMax ? 2 : 1;
  a.smem = (unsigned)(tp->tf32 ? tc_smem_bytes<true>(R, a.nabuf) : tc_smem_bytes<false>(R, a.nabuf));
  if (e == cudaSuccess && a.nplanes > 0) e = cudaMalloc(&tp->A, (size_t)a.nplanes * astride);
  if (e == cudaSuccess && a.nplanes > 0) {
    if (tp->tf32)
      k_build_a<true><<<a.nplanes, 256>>>(a, tp->A);
    else
      k_build_a<false><<<a.nplanes, 256>>>(a, tp->A);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  a.A = tp->A;
  a.err = tp->err;
  c->tc = tp;
  if (e != cudaSuccess) {
    tc_free(c);
    return cuda_error(e, "tensor-core plan");
  }
  c->launches_per_step = 4;
  return SX_OK;
}

void tc_free(sx_ctx *c) {
  TcPlan *tp = c->tc;
  if (!tp) return;
  cudaFree(tp->St);
  cudaFree(tp->F0);
  cudaFree(tp->Bf);
  cudaFree(tp->Th);
  cudaFree(tp->A);
  cudaFree(tp->err);
  delete tp;
  c->tc = nullptr;
}

cudaError_t tc_field(const sx_ctx *c, const double *S, double *b, bool onsite, cudaStream_t st) {
  TcArgs a = c->tc->base;
  a.onsite = onsite ? 1 : 0;
  return c->tc->tf32 ? launch_tc<true, double, double>(c, a, S, b, st) : launch_tc<false, double, double>(c, a, S, b, st);
}

cudaError_t tc_heun_step(const sx_ctx *c, const double *src, double *dst, const HeunConst &h, uint64_t step,
                         cudaStream_t st) {
  const TcPlan &tp = *c->tc;
  TcArgs a = tp.base;
  a.onsite = 0;
  cudaError_t e = tp.tf32 ? launch_tc<true, double, float>(c, a, src, tp.Bf, st)
                          : launch_tc<false, double, float>(c, a, src, tp.Bf, st);
  if (e == cudaSuccess) e = bufheun_predict(c, src, tp.Bf, tp.St, tp.F0, tp.Th, h, step, st);
  if (e == cudaSuccess)
    e = tp.tf32 ? launch_tc<true, float, float>(c, a, tp.St, tp.Bf, st)
                : launch_tc<false, float, float>(c, a, tp.St, tp.Bf, st);
  if (e == cudaSuccess) e = bufheun_correct(c, src, tp.St, tp.F0, tp.Bf, tp.Th, dst, h, st);
  return e;
}

// 1 if a bounded wait of the tensor-core kernel gave up since the last check (clears it)
int tc_check_error(const sx_ctx *c) {
  int h = 0;
  if (!c->tc || cudaMemcpy(&h, c->tc->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return 0;
  if (h) cudaMemset(c->tc->err, 0, sizeof(int));
  return h;
}

}  // namespace sx
