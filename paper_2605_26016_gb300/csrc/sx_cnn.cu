// Convolutional proposer of minimum-energy-path chains, trained and run on the
// 5th-generation tensor cores (tcgen05).
//
// The proposer maps an image of a chain, placed by geodesic interpolation
// between the endpoints ("Static optimization and minimum-energy paths": the
// string and GNEB methods start from such chains), to a better first guess of
// the converged image.  Per site the input has 10 channels (interpolated image
// I, endpoints A and B, path coordinate s); four 3x3x3 convolutions with zero
// padding and bias map 10 -> 16 -> 16 -> 16 -> 3 channels with ReLU after the
// first three; the proposal is P = N[I + Y] and the training loss is
// L = mean over samples and sites of (1 - P . T), T the converged image.
//
// Data layout (device):
//  * activations: channels-last BF16, [sample][site][16] (32 bytes per site,
//    channels above a layer's width are zero); the packed input X has the
//    channels I(0..2), A(3..5), B(6..8), s(9), zeros(10..15);
//  * gradients of activations: channels-last FP32, [sample][site][16];
//  * parameters: FP32, per layer the weights [out][in][dz][dy][dx] then the
//    biases, layers in order (19,491 values); Adam moments alike;
//  * tensor-core operands of the weights, rebuilt from the FP32 parameters on
//    every update: per layer and tap a 16 x 16 BF16 matrix in the canonical
//    no-swizzle K-major core-matrix layout, one copy for the forward
//    convolution (rows = output channel, K = input channel) and one for the
//    input gradient (taps mirrored, rows = input channel, K = output channel).
//
// Convolutions (forward and input gradient) are implicit GEMMs.  A CTA owns a
// 16 x 16 x BZ block of output sites of one sample and stages the input
// window (18 x 18 x (BZ+2) sites, zero outside the lattice) in shared memory
// as two 16-byte channel planes.  An M = 128 tile is 8 consecutive x sites by
// 16 y rows of one z plane: core-matrix rows are consecutive sites (16 bytes
// apart) and row groups are window rows (288 bytes apart), so the A operand of
// tap (dz, dy, dx) is the same window seen from a start address shifted by
// (dz, dy, dx) sites.  Each tile accumulates 27 MMAs of 128 x 16 x 16 (one per
// tap; two for the input gradient, whose FP32 operand is split into BF16
// hi + lo parts) in 16 TMEM columns.  One elected thread issues tcgen05.mma
// (kind::f16) and tcgen05.commit; every wait is bounded and sets an error flag
// instead of hanging.  Epilogues read TMEM with tcgen05.ld and fuse bias and
// ReLU (forward), the normalisation, loss and loss gradient (last layer), or
// the ReLU mask (input gradient).  The head forms the proposal in FP64 and the
// training loss and dL/dZ in FP32.
//
// Weight gradients sum g_out[s][o] x act[s + tap][c] over all sites: an
// im2col GEMM on the tensor cores with the sites as K, per-CTA partial sums
// reduced over CTAs in FP64 in a fixed order (deterministic).
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <new>

#include "sx_device.cuh"
#include "sx_internal.h"

struct sx_cnn;

namespace sx {
namespace cnn {

constexpr int kC = 16;     // stored channels per site
constexpr int kTaps = 27;  // 3 x 3 x 3 kernel
constexpr int kLayers = 4;
__host__ __device__ constexpr int cin_of(int l) { return l == 0 ? 10 : 16; }
__host__ __device__ constexpr int cout_of(int l) { return l == 3 ? 3 : 16; }
__host__ __device__ constexpr int nparam_of(int l) { return cout_of(l) * cin_of(l) * kTaps + cout_of(l); }
__host__ __device__ constexpr int wofs(int l) {
  int o = 0;
  for (int k = 0; k < l; ++k) o += nparam_of(k);
  return o;
}
constexpr int kNParam = wofs(kLayers);
static_assert(kNParam == 19491, "parameter count");

constexpr int kBX = 16, kBY = 16;  // output block per CTA in x and y
constexpr int kWX = kBX + 2, kWY = kBY + 2;
constexpr int kThreads = 128;
constexpr int kWBytes = kTaps * 512;  // operand of one layer: 27 taps x 16 x 16 BF16
constexpr int kBZF = 4;               // output z planes per CTA, forward
constexpr int kBZD = 2;               // output z planes per CTA, input gradient (4 planes at one CTA per SM measured 1.5x slower)
constexpr int kZW = 8;                // z planes per weight-gradient CTA (two at a time)
constexpr int kPart = kTaps * 256 + 16;  // one partial: gw[tap][o][c] then gb[o]

enum Mode { FWD = 0, HEAD = 1, DGRAD = 2 };

// byte offset of element (tap, row n, column k) in a layer operand
__host__ __device__ __forceinline__ int op_off(int t, int n, int k) {
  return t * 512 + (k >> 3) * 256 + n * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
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

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
  return (uint32_t)__bfloat16_as_ushort(ha) | ((uint32_t)__bfloat16_as_ushort(hb) << 16);
}

// hi = RN_bf16(v), lo = RN_bf16(v - hi), packed pairwise
__device__ __forceinline__ void split_bf16(float a, float b, uint32_t &hi, uint32_t &lo) {
  const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
  hi = (uint32_t)__bfloat16_as_ushort(ha) | ((uint32_t)__bfloat16_as_ushort(hb) << 16);
  lo = pack_bf16(a - __bfloat162float(ha), b - __bfloat162float(hb));
}

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

struct ConvArgs {
  int nx, ny, nz, tiles_x;
  long long ncell;
  const uint16_t *act_in;     // FWD, HEAD: layer input, [nb][ncell][16] BF16
  const float *g_in;          // DGRAD: gradient of the layer output, [nb][ncell][16]
  const unsigned char *wop;   // operand of the layer (kWBytes)
  const float *bias;          // FWD, HEAD: biases of the layer
  int cout;
  uint16_t *act_out;          // FWD: ReLU output, [nb][ncell][16] BF16
  const uint16_t *mask;       // DGRAD: the layer's input activation (ReLU mask)
  float *g_out;               // DGRAD: masked input gradient; HEAD: dL/dZ (channels 0..2)
  const double *I;            // HEAD: interpolated images [nb][3][ncell]
  const double *T;            // HEAD: targets [nb][3][ncell] or null
  double *P;                  // HEAD: proposals [nb][3][ncell] or null (may equal I)
  float inv_mf;               // HEAD: 1 / (nb ncell)
  double *loss_part;          // HEAD: per-CTA sums of (1 - P.T)
  int *err;
};

template <int BZ, int NCOPY>
__host__ __device__ constexpr int conv_nrow() {
  return kWX * kWY * (BZ + 2);
}
template <int BZ, int NCOPY>
__host__ __device__ constexpr size_t conv_smem() {
  return (size_t)kWBytes + (size_t)NCOPY * 2 * conv_nrow<BZ, NCOPY>() * 16 + 64 + 16 * 8;
}

template <int MODE, int BZ>
__global__ void __launch_bounds__(kThreads) k_conv(const ConvArgs p) {
  constexpr int NCOPY = MODE == DGRAD ? 2 : 1;
  constexpr int NROW = conv_nrow<BZ, NCOPY>();
  constexpr uint32_t PLANE = (uint32_t)NROW * 16u;  // one 8-channel plane of the window
  constexpr uint32_t COPY = 2u * PLANE;
  constexpr int NTILE = 2 * BZ;
  constexpr uint32_t TCOLS = NTILE * 16 <= 32 ? 32u : NTILE * 16 <= 64 ? 64u : NTILE * 16 <= 128 ? 128u : 256u;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *sW = smem;
  unsigned char *sWin = smem + kWBytes;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sWin + NCOPY * COPY);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
  double *red = reinterpret_cast<double *>(mbar + 2);  // kThreads / 32 partial sums
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bxy = blockIdx.x;
  const int x0 = (bxy % p.tiles_x) * kBX, y0 = (bxy / p.tiles_x) * kBY, z0 = blockIdx.y * BZ;
  const long long sbase = (long long)blockIdx.z * p.ncell;

  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(mbar)));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)), "n"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // weights
  for (int e = tid; e < kWBytes / 16; e += kThreads) cp_async16(saddr(sW + 16 * e), p.wop + 16 * e);
  // input window: row r = (zw * kWY + yw) * kWX + xw, channel plane ch (channels 8 ch .. 8 ch + 7)
  for (int e = tid; e < NROW * 2; e += kThreads) {
    const int ch = e & 1, r = e >> 1;
    const int xw = r % kWX, q = r / kWX, yw = q % kWY, zw = q / kWY;
    const int gx = x0 - 1 + xw, gy = y0 - 1 + yw, gz = z0 - 1 + zw;
    const bool ok = gx >= 0 && gx < p.nx && gy >= 0 && gy < p.ny && gz >= 0 && gz < p.nz;
    const long long site = sbase + ((long long)gz * p.ny + gy) * p.nx + gx;
    unsigned char *dst = sWin + ch * PLANE + (uint32_t)r * 16u;
    if (MODE != DGRAD) {
      if (ok)
        cp_async16(saddr(dst), p.act_in + site * kC + ch * 8);
      else
        *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
    } else {
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
      if (ok) {
        const float4 *src = reinterpret_cast<const float4 *>(p.g_in + site * kC + ch * 8);
        a = __ldg(src);
        b = __ldg(src + 1);
      }
      uint4 hi, lo;
      split_bf16(a.x, a.y, hi.x, lo.x);
      split_bf16(a.z, a.w, hi.y, lo.y);
      split_bf16(b.x, b.y, hi.z, lo.z);
      split_bf16(b.z, b.w, hi.w, lo.w);
      *reinterpret_cast<uint4 *>(dst) = hi;
      *reinterpret_cast<uint4 *>(dst + COPY) = lo;
    }
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  // kind::f16: D FP32, A and B BF16, both K-major, N = 16, M = 128
  constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(16 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  if (tid == 0) {
    const uint32_t wa = saddr(sW), xa = saddr(sWin);
    for (int tt = 0; tt < NTILE; ++tt) {
      const int zl = tt >> 1, xg = tt & 1;
      const uint32_t d = tmem + (uint32_t)(tt * 16);
      for (int t = 0; t < kTaps; ++t) {
        const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
        const int row = ((zl + 1 + dz) * kWY + (1 + dy)) * kWX + (8 * xg + 1 + dx);
        const uint64_t bd = smem_desc(wa + (uint32_t)t * 512u, 256u, 128u);
#pragma unroll
        for (int cp = 0; cp < NCOPY; ++cp) {
          const uint64_t ad = smem_desc(xa + (uint32_t)cp * COPY + (uint32_t)row * 16u, PLANE, (uint32_t)kWX * 16u);
          const uint32_t acc = (t > 0 || cp > 0) ? 1u : 0u;
          asm volatile(
              "{\n.reg .pred q;\nsetp.ne.u32 q, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(d),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(mbar))
                 : "memory");
  }
  // every thread waits (bounded); the epilogue runs only if all of them saw the MMAs complete
  const bool alive = __syncthreads_and(wait_parity(mbar, 0u, p.err) ? 1 : 0) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  double lsum = 0.0;
  if (alive) {
    // row m = 32 warp + lane of every tile: y = y0 + m / 8, x = x0 + 8 xg + m % 8
    const int m = warp * 32 + lane;
    const int y = y0 + (m >> 3);
    float bias[16];
    if (MODE != DGRAD) {
#pragma unroll
      for (int c = 0; c < 16; ++c) bias[c] = c < p.cout ? __ldg(p.bias + c) : 0.0f;
    }
    for (int tt = 0; tt < NTILE; ++tt) {
      const int zl = tt >> 1, xg = tt & 1;
      uint32_t r[16];
      const uint32_t a = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(tt * 16);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(a));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int x = x0 + 8 * xg + (m & 7), z = z0 + zl;
      if (x >= p.nx || y >= p.ny || z >= p.nz) continue;
      const long long cell = ((long long)z * p.ny + y) * p.nx + x;
      const long long site = sbase + cell;
      if (MODE == FWD) {
        uint32_t w[8];
#pragma unroll
        for (int c = 0; c < 8; ++c)
          w[c] = pack_bf16(fmaxf(__uint_as_float(r[2 * c]) + bias[2 * c], 0.0f),
                           fmaxf(__uint_as_float(r[2 * c + 1]) + bias[2 * c + 1], 0.0f));
        uint4 *dst = reinterpret_cast<uint4 *>(p.act_out + site * kC);
        dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
        dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
      } else if (MODE == HEAD) {
        const long long i0 = (long long)blockIdx.z * 3 * p.ncell + cell;
        float Y[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) Y[k] = __uint_as_float(r[k]) + bias[k];
        if (p.P) {
          // P = Z / |Z| in FP64: 1/|Z| from an FP32 estimate and two Newton steps (FP64 division and square
          // root run on the FP64 pipe, 1/70 of the FP32 rate on this part)
          double Z[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) Z[k] = p.I[i0 + k * p.ncell] + f32_to_f64(Y[k]);
          const double z2 = Z[0] * Z[0] + Z[1] * Z[1] + Z[2] * Z[2];
          double rn = f32_to_f64(rsqrtf(f64_to_f32(z2)));
          rn = rn * (1.5 - 0.5 * z2 * rn * rn);
          rn = rn * (1.5 - 0.5 * z2 * rn * rn);
          p.P[i0] = Z[0] * rn;
          p.P[i0 + p.ncell] = Z[1] * rn;
          p.P[i0 + 2 * p.ncell] = Z[2] * rn;
        }
        if (p.T) {
          // loss term and dL/dZ in FP32 (dL/dZ is stored in FP32): P = Z / |Z|, 1 - P.T = |P - T|^2 / 2 for
          // unit P and T, dL/dP = -T / m, dL/dZ = (dL/dP - (dL/dP . P) P) / |Z|
          float Zf[3], Tf[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            Zf[k] = f64_to_f32(p.I[i0 + k * p.ncell]) + Y[k];
            Tf[k] = f64_to_f32(p.T[i0 + k * p.ncell]);
          }
          const float z2 = Zf[0] * Zf[0] + Zf[1] * Zf[1] + Zf[2] * Zf[2];
          float rn = rsqrtf(z2);
          rn = rn * (1.5f - 0.5f * z2 * rn * rn);
          const float P0 = Zf[0] * rn, P1 = Zf[1] * rn, P2 = Zf[2] * rn;
          const float d0 = P0 - Tf[0], d1 = P1 - Tf[1], d2 = P2 - Tf[2];
          lsum += (double)(0.5f * (d0 * d0 + d1 * d1 + d2 * d2));
          const float im = p.inv_mf;
          const float g0 = -Tf[0] * im, g1 = -Tf[1] * im, g2 = -Tf[2] * im;
          const float gp = g0 * P0 + g1 * P1 + g2 * P2;
          float4 *dst = reinterpret_cast<float4 *>(p.g_out + site * kC);
          dst[0] = make_float4((g0 - gp * P0) * rn, (g1 - gp * P1) * rn, (g2 - gp * P2) * rn, 0.0f);
          const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
          dst[1] = zero;
          dst[2] = zero;
          dst[3] = zero;
        }
      } else {
        const uint4 *mk = reinterpret_cast<const uint4 *>(p.mask + site * kC);
        const uint4 m0 = __ldg(mk), m1 = __ldg(mk + 1);
        const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
        float o[16];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          o[2 * c] = bf16_lo(mw[c]) > 0.0f ? __uint_as_float(r[2 * c]) : 0.0f;
          o[2 * c + 1] = bf16_hi(mw[c]) > 0.0f ? __uint_as_float(r[2 * c + 1]) : 0.0f;
        }
        float4 *dst = reinterpret_cast<float4 *>(p.g_out + site * kC);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
      }
    }
  }
  if (MODE == HEAD && p.T) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_down_sync(0xFFFFFFFFu, lsum, off);
    if (lane == 0) red[warp] = lsum;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (MODE == HEAD && p.T && tid == 0) {
    const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    p.loss_part[blk] = (red[0] + red[1]) + (red[2] + red[3]);
  }
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TCOLS));
}

// Weight and bias gradients of one layer on the tensor cores.  gw[tap][o][c] = sum_s act[s + tap][c] g[s][o]
// is a GEMM with the sites as K: D[(tap, c)][o] += A[(tap, c)][s] B[s][o].  A CTA owns a 16 x 16 x kZW block of
// sites of one sample and walks it in K blocks of 64 sites (4 y rows x 16 x of one z plane):
//  * the channels-last input window of a z pair (18 x 18 x 4 sites, zero outside the lattice) is staged in
//    shared memory;
//  * per K block the im2col operand A is gathered from the window: rows (tap, c) in four M = 128 groups of
//    eight taps (taps 27..31 of the last group are never written and their rows of D are not read), eight
//    consecutive x sites per 16-byte core-matrix row;
//  * B holds g of the 64 sites split into BF16 hi and lo parts as N = 32 columns (o hi, o lo), so one
//    128 x 32 x 16 MMA per group and K step accumulates both parts, summed in the epilogue;
//  * one thread issues the 16 MMAs of a K block and commits; all threads wait (bounded) before the operands
//    are rebuilt.
// Each CTA writes one partial gw[tap][o][c], gb[o]; gb is summed on the CUDA cores from the same g values.
struct WgradArgs {
  int nx, ny, nz, tiles_x;
  long long ncell;
  const float *g;          // gradient of the layer output [nb][ncell][16]
  const uint16_t *act;     // layer input [nb][ncell][16] BF16
  float *part;             // [nblocks][kPart]
  int *err;
};

constexpr int kWgThreads = 256;
constexpr int kWgRows = kWX * kWY * 4;              // window of a z pair: 18 x 18 x 4 sites
constexpr uint32_t kWgAGroup = 128 * 64 * 2;        // one M group of A: 128 rows x 64 sites BF16
constexpr uint32_t kWgA = 4 * kWgAGroup;
constexpr uint32_t kWgB = 32 * 64 * 2;
constexpr size_t kWgSmem = (size_t)kWgRows * 32 + kWgA + kWgB + 128 * 4 + 64;

__global__ void __launch_bounds__(kWgThreads) k_wgrad(const WgradArgs p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint16_t *sWin = reinterpret_cast<uint16_t *>(smem);  // [row][16] BF16
  unsigned char *sA = smem + (size_t)kWgRows * 32;
  unsigned char *sB = sA + kWgA;
  float *sGb = reinterpret_cast<float *>(sB + kWgB);  // [8][16] bias partials
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sGb + 128);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bxy = blockIdx.x;
  const int x0 = (bxy % p.tiles_x) * kBX, y0 = (bxy / p.tiles_x) * kBY, zb = blockIdx.y * kZW;
  const long long sbase = (long long)blockIdx.z * p.ncell;

  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(mbar)));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(saddr(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  // kind::f16: D FP32, A and B BF16, both K-major, N = 32, M = 128
  constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(32 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  float gbacc = 0.0f;
  uint32_t phase = 0;
  bool alive = true;
  int kblk = 0;
  // g of one K block for this thread's B task (kc = tid / 16, o = tid % 16), loaded one block ahead so that
  // the loads overlap the previous block's MMAs
  float vn[8];
  auto load_g = [&](int gz, int yq) {
    const int kc = tid >> 4, o = tid & 15;
    const int gy = y0 + 4 * yq + (kc >> 1), gx0 = x0 + 8 * (kc & 1);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gx = gx0 + j;
      vn[j] = (gx < p.nx && gy < p.ny && gz < p.nz)
                  ? __ldg(p.g + (sbase + ((long long)gz * p.ny + gy) * p.nx + gx) * kC + o)
                  : 0.0f;
    }
  };
  if (tid < 128) load_g(zb, 0);
  for (int z0 = zb; z0 < zb + kZW && z0 < p.nz && alive; z0 += 2) {
    // window rows (zw, yw, xw) of z planes z0 - 1 .. z0 + 2 (the previous K block's MMAs have completed)
    for (int e = tid; e < kWgRows * 2; e += kWgThreads) {
      const int ch = e & 1, r = e >> 1;
      const int xw = r % kWX, q = r / kWX, yw = q % kWY, zw = q / kWY;
      const int gx = x0 - 1 + xw, gy = y0 - 1 + yw, gz = z0 - 1 + zw;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (gx >= 0 && gx < p.nx && gy >= 0 && gy < p.ny && gz >= 0 && gz < p.nz)
        v = __ldg(reinterpret_cast<const uint4 *>(p.act + (sbase + ((long long)gz * p.ny + gy) * p.nx + gx) * kC) + ch);
      reinterpret_cast<uint4 *>(sWin)[2 * r + ch] = v;
    }
    for (int zl = 0; zl < 2 && alive; ++zl) {
      for (int yq = 0; yq < 4 && alive; ++yq) {
        __syncthreads();  // window staged; previous operands consumed
        if (tid < 128) {
          // B: sites k = 8 kc + j (y = 4 yq + kc / 2, x = 8 (kc % 2) + j), column o (hi) and 16 + o (lo)
          const int kc = tid >> 4, o = tid & 15;
          float v[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            v[j] = vn[j];
            gbacc += v[j];
          }
          uint4 hi, lo;
          split_bf16(v[0], v[1], hi.x, lo.x);
          split_bf16(v[2], v[3], hi.y, lo.y);
          split_bf16(v[4], v[5], hi.z, lo.z);
          split_bf16(v[6], v[7], hi.w, lo.w);
          *reinterpret_cast<uint4 *>(sB + kc * 512 + (o >> 3) * 128 + (o & 7) * 16) = hi;
          *reinterpret_cast<uint4 *>(sB + kc * 512 + ((16 + o) >> 3) * 128 + (o & 7) * 16) = lo;
        }
        // A: row m = 16 (tap % 8) + c of group tap / 8, 16-byte chunk of sites 8 kc .. 8 kc + 7.  A task takes
        // the channel pair (2 cp, 2 cp + 1) of one tap and chunk: eight 4-byte reads of the window give both
        // rows.  Groups of eight lanes take neighbouring taps (window rows one site apart).
        for (int e = tid; e < kTaps * 8 * 8; e += kWgThreads) {
          const int cp = e & 7, tk = e >> 3, t = tk % kTaps, kc = tk / kTaps;
          const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
          const int row = ((zl + 1 + dz) * kWY + (4 * yq + (kc >> 1) + 1 + dy)) * kWX + 8 * (kc & 1) + 1 + dx;
          const uint32_t *src = reinterpret_cast<const uint32_t *>(sWin + row * kC) + cp;
          uint32_t v[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) v[j] = src[j * (kC / 2)];
          uint4 we, wo;
          we.x = __byte_perm(v[0], v[1], 0x5410);
          wo.x = __byte_perm(v[0], v[1], 0x7632);
          we.y = __byte_perm(v[2], v[3], 0x5410);
          wo.y = __byte_perm(v[2], v[3], 0x7632);
          we.z = __byte_perm(v[4], v[5], 0x5410);
          wo.z = __byte_perm(v[4], v[5], 0x7632);
          we.w = __byte_perm(v[6], v[7], 0x5410);
          wo.w = __byte_perm(v[6], v[7], 0x7632);
          const int m = 16 * (t & 7) + 2 * cp;
          unsigned char *dst = sA + (t >> 3) * kWgAGroup + kc * 2048 + (m >> 3) * 128 + (m & 7) * 16;
          *reinterpret_cast<uint4 *>(dst) = we;
          *reinterpret_cast<uint4 *>(dst + 16) = wo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          for (int G = 0; G < 4; ++G) {
            for (int ks = 0; ks < 4; ++ks) {
              const uint64_t ad = smem_desc(saddr(sA) + G * kWgAGroup + ks * 2 * 2048, 2048u, 128u);
              const uint64_t bd = smem_desc(saddr(sB) + ks * 2 * 512, 512u, 128u);
              const uint32_t acc = (kblk > 0 || ks > 0) ? 1u : 0u;
              asm volatile(
                  "{\n.reg .pred q;\nsetp.ne.u32 q, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(
                      tmem + (uint32_t)(G * 32)),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(mbar))
                       : "memory");
        }
        if (tid < 128) {
          // the next K block: the next row group, the next plane of the pair, or the first of the next pair
          if (yq < 3)
            load_g(z0 + zl, yq + 1);
          else if (zl == 0)
            load_g(z0 + 1, 0);
          else if (z0 + 2 < zb + kZW && z0 + 2 < p.nz)
            load_g(z0 + 2, 0);
        }
        alive = __syncthreads_and(wait_parity(mbar, phase, p.err) ? 1 : 0) != 0;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        ++kblk;
      }
    }
    __syncthreads();
  }
  if (tid < 128) sGb[tid] = gbacc;
  __syncthreads();
  const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  float *out = p.part + (size_t)blk * kPart;
  if (tid < 16) {
    float sgb = 0.0f;
    for (int k = 0; k < 8; ++k) sgb += sGb[k * 16 + tid];
    out[kTaps * 256 + tid] = sgb;
  }
  if (alive && kblk > 0) {
    // row m = 32 (warp % 4) + lane of groups warp / 4 and warp / 4 + 2: tap 8 G + m / 16, channel m % 16
    const int q = warp & 3;
    for (int G = warp >> 2; G < 4; G += 2) {
      uint32_t r[32];
      const uint32_t a = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(G * 32);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
          "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(a));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int m = q * 32 + lane, t = 8 * G + (m >> 4), c = m & 15;
      if (t < kTaps) {
#pragma unroll
        for (int o = 0; o < 16; ++o) out[t * 256 + o * 16 + c] = __uint_as_float(r[o]) + __uint_as_float(r[16 + o]);
      }
    }
  } else {
    // no K block ran (or a wait gave up): zero weight partials
    for (int e = tid; e < kTaps * 256; e += kWgThreads) out[e] = 0.0f;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

// grad for every parameter: the FP64 sum over the partials of its layer.  Block (x, l) with 32 x 8 threads
// reduces partial entries q = 32 x + lane of layer l: warp w sums slots w, w + 8, ... (coalesced across lanes),
// the eight warp sums combine in a fixed tree, and the entry is scattered to its parameter.  Row l = kLayers
// reduces the loss partials the same way.  The order depends only on the sizes (deterministic).
struct ReduceArgs {
  const float *part[kLayers];
  long long nslot;       // partials per layer
  float *grad;
  const double *loss_part;
  long long nloss;
  double inv_m;
  double *loss;          // device scalar
};

__global__ void __launch_bounds__(256) k_grad_reduce(const ReduceArgs p) {
  __shared__ double red[8][33];
  const int lane = threadIdx.x, w = threadIdx.y, l = blockIdx.y;
  const int q = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (l == kLayers) {
    if (blockIdx.x == 0)
      for (long long k = w * 32 + lane; k < p.nloss; k += 256) s += p.loss_part[k];
  } else if (q < kPart) {
    const float *src = p.part[l] + q;
    for (long long k = w; k < p.nslot; k += 8) s += (double)src[(size_t)k * kPart];
  }
  red[w][lane] = s;
  __syncthreads();
  if (w != 0) return;
  const double t = ((red[0][lane] + red[1][lane]) + (red[2][lane] + red[3][lane])) +
                   ((red[4][lane] + red[5][lane]) + (red[6][lane] + red[7][lane]));
  if (l == kLayers) {
    if (blockIdx.x != 0) return;
    double v = t;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, off);
    if (lane == 0 && p.loss) *p.loss = v * p.inv_m;
    return;
  }
  if (q >= kPart) return;
  const int ci = cin_of(l), co = cout_of(l);
  int j = -1;
  if (q < kTaps * 256) {
    const int tap = q >> 8, o = (q >> 4) & 15, c = q & 15;
    if (o < co && c < ci) j = (o * ci + c) * kTaps + tap;
  } else if (q - kTaps * 256 < co) {
    j = co * ci * kTaps + (q - kTaps * 256);
  }
  if (j >= 0) p.grad[wofs(l) + j] = (float)t;
}

// Writes the BF16 operands of parameter i (a weight) into the forward and input-gradient operands of its layer.
__device__ __forceinline__ void put_operands(int i, float w, unsigned char *wop) {
  int l = 0;
  while (l + 1 < kLayers && i >= wofs(l + 1)) ++l;
  const int j = i - wofs(l);
  const int ci = cin_of(l), co = cout_of(l);
  if (j >= co * ci * kTaps) return;
  const int o = j / (ci * kTaps), c = (j / kTaps) % ci, t = j % kTaps;
  const uint16_t h = __bfloat16_as_ushort(__float2bfloat16_rn(w));
  unsigned char *f = wop + (size_t)(2 * l) * kWBytes, *d = wop + (size_t)(2 * l + 1) * kWBytes;
  *reinterpret_cast<uint16_t *>(f + op_off(t, o, c)) = h;
  *reinterpret_cast<uint16_t *>(d + op_off(kTaps - 1 - t, c, o)) = h;
}

__global__ void k_build_ops(const float *w, unsigned char *wop) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kNParam) put_operands(i, w[i], wop);
}

// Adam (Kingma and Ba, Algorithm 1) on the FP32 parameters; c1 = 1/(1 - beta1^t), c2 = 1/(1 - beta2^t).
__global__ void k_adam(float *w, float *m, float *v, const float *g, float lr, float b1, float b2, float eps, float c1,
                       float c2, unsigned char *wop) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNParam) return;
  const float gi = g[i];
  const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
  const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  w[i] = wi;
  put_operands(i, wi, wop);
}

// Packed BF16 input X[b][site][16] = (I, A, B, s, 0...) rounded through FP32.
__global__ void k_pack(const double *I, long long is, const double *A, const double *B, long long abs_, const double *s,
                       long long ncell, int nb, uint16_t *X) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ncell * nb) return;
  const long long b = idx / ncell, cell = idx % ncell;
  const double *Ib = I + b * is, *Ab = A + b * abs_, *Bb = B + b * abs_;
  float v[16];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    v[k] = __double2float_rn(Ib[k * ncell + cell]);
    v[3 + k] = __double2float_rn(Ab[k * ncell + cell]);
    v[6 + k] = __double2float_rn(Bb[k * ncell + cell]);
  }
  v[9] = __double2float_rn(s[b]);
#pragma unroll
  for (int k = 10; k < 16; ++k) v[k] = 0.0f;
  uint4 *dst = reinterpret_cast<uint4 *>(X + idx * kC);
  dst[0] = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
  dst[1] = make_uint4(pack_bf16(v[8], v[9]), 0u, 0u, 0u);
}

// Geodesic interpolation of the interior images k = 1 .. nimg-2 of a chain at s_k = k / (nimg - 1), site by site
// on the shorter great-circle arc; parallel pairs blend linearly, antiparallel pairs turn through the unit part
// of x-hat (y-hat where |A_x| >= 0.9) orthogonal to A.  Also writes s_k to s_out[k - 1].
__global__ void k_interp(double *chain, int nimg, long long ncell, double *s_out) {
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y + 1;
  const double s = (double)k / (double)(nimg - 1);
  if (cell == 0) s_out[k - 1] = s;
  if (cell >= ncell) return;
  const double *A = chain, *B = chain + (size_t)(nimg - 1) * 3 * ncell;
  double a[3], b[3];
  for (int q = 0; q < 3; ++q) {
    a[q] = A[q * ncell + cell];
    b[q] = B[q * ncell + cell];
  }
  const double c = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
  const double w0 = a[1] * b[2] - a[2] * b[1], w1 = a[2] * b[0] - a[0] * b[2], w2 = a[0] * b[1] - a[1] * b[0];
  const double sn = sqrt(w0 * w0 + w1 * w1 + w2 * w2);
  double out[3];
  if (sn >= 1e-6) {
    const double th = atan2(sn, c), st = sin(th);
    const double fa = sin((1.0 - s) * th) / st, fb = sin(s * th) / st;
    for (int q = 0; q < 3; ++q) out[q] = fa * a[q] + fb * b[q];
  } else if (c > 0.0) {
    double nn = 0.0;
    for (int q = 0; q < 3; ++q) {
      out[q] = (1.0 - s) * a[q] + s * b[q];
      nn += out[q] * out[q];
    }
    nn = sqrt(nn);
    for (int q = 0; q < 3; ++q) out[q] /= nn;
  } else {
    double e[3] = {1.0, 0.0, 0.0};
    if (fabs(a[0]) >= 0.9) {
      e[0] = 0.0;
      e[1] = 1.0;
    }
    const double ae = a[0] * e[0] + a[1] * e[1] + a[2] * e[2];
    double u[3], nu = 0.0;
    for (int q = 0; q < 3; ++q) {
      u[q] = e[q] - ae * a[q];
      nu += u[q] * u[q];
    }
    nu = sqrt(nu);
    const double cs = cos(M_PI * s), sn2 = sin(M_PI * s);
    for (int q = 0; q < 3; ++q) out[q] = cs * a[q] + sn2 * (u[q] / nu);
  }
  double *dst = chain + (size_t)k * 3 * ncell;
  for (int q = 0; q < 3; ++q) dst[q * ncell + cell] = out[q];
}

}  // namespace cnn
}  // namespace sx

using namespace sx;
using namespace sx::cnn;

struct sx_cnn {
  int n[3];
  long long ncell;
  int max_batch;
  int tiles_x, tiles_y;
  float *w, *m, *v, *grad;      // parameters, Adam moments, gradient scratch (kNParam each)
  unsigned char *wop;           // 2 kLayers operands
  uint16_t *act[3];             // activations of layers 1..3
  uint16_t *X;                  // packed input for proposals
  float *g[2];                  // activation gradients (ping-pong)
  float *part[kLayers];         // weight-gradient partials per layer
  long long nslot;              // partials per layer at max_batch
  double *loss_part, *loss, *s_dev;
  long long nloss;
  int *err;
  long long adam_t;
};

namespace {

template <typename T>
cudaError_t dalloc(T **p, size_t count) {
  return cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }
bool aligned8(const void *p) { return ((uintptr_t)p & 7u) == 0; }

int check_err(sx_cnn *h, cudaStream_t st) {
  int e = 0;
  cudaError_t ce = cudaMemcpyAsync(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return cuda_error(ce, "proposer kernels");
  if (e) {
    cudaMemsetAsync(h->err, 0, sizeof(int), st);
    return set_error(SX_ERR_TIMEOUT, "a bounded tensor-core wait gave up in a proposer convolution");
  }
  return SX_OK;
}

template <int MODE, int BZ>
cudaError_t launch_conv(const sx_cnn *h, int nb, ConvArgs a, cudaStream_t st) {
  constexpr size_t smem = conv_smem<BZ, MODE == DGRAD ? 2 : 1>();
  static_assert(smem <= 227 * 1024, "shared memory");
  cudaError_t e = cudaFuncSetAttribute(k_conv<MODE, BZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  a.nx = h->n[0];
  a.ny = h->n[1];
  a.nz = h->n[2];
  a.tiles_x = h->tiles_x;
  a.ncell = h->ncell;
  a.err = h->err;
  const dim3 grid((unsigned)(h->tiles_x * h->tiles_y), (unsigned)((h->n[2] + BZ - 1) / BZ), (unsigned)nb);
  k_conv<MODE, BZ><<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_wgrad(const sx_cnn *h, int nb, const float *g, const uint16_t *act, float *part, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmem);
  if (e != cudaSuccess) return e;
  WgradArgs a;
  a.nx = h->n[0];
  a.ny = h->n[1];
  a.nz = h->n[2];
  a.tiles_x = h->tiles_x;
  a.ncell = h->ncell;
  a.g = g;
  a.act = act;
  a.part = part;
  a.err = h->err;
  const dim3 grid((unsigned)(h->tiles_x * h->tiles_y), (unsigned)((h->n[2] + kZW - 1) / kZW), (unsigned)nb);
  k_wgrad<<<grid, kWgThreads, kWgSmem, st>>>(a);
  return cudaGetLastError();
}

long long wgrad_slots(const sx_cnn *h, int nb) {
  return 1LL * h->tiles_x * h->tiles_y * ((h->n[2] + kZW - 1) / kZW) * nb;
}
long long head_blocks(const sx_cnn *h, int nb) {
  return (long long)h->tiles_x * h->tiles_y * ((h->n[2] + kBZF - 1) / kBZF) * nb;
}

// forward through the four layers; the last writes P (may be null) and, with T, the loss partials and dL/dZ
cudaError_t forward(sx_cnn *h, const uint16_t *X, const double *I, const double *T, int nb, double *P,
                    cudaStream_t st) {
  const uint16_t *in = X;
  for (int l = 0; l < 3; ++l) {
    ConvArgs a{};
    a.act_in = in;
    a.wop = h->wop + (size_t)(2 * l) * kWBytes;
    a.bias = h->w + wofs(l) + cout_of(l) * cin_of(l) * kTaps;
    a.cout = cout_of(l);
    a.act_out = h->act[l];
    cudaError_t e = launch_conv<FWD, kBZF>(h, nb, a, st);
    if (e != cudaSuccess) return e;
    in = h->act[l];
  }
  ConvArgs a{};
  a.act_in = in;
  a.wop = h->wop + (size_t)6 * kWBytes;
  a.bias = h->w + wofs(3) + cout_of(3) * cin_of(3) * kTaps;
  a.cout = 3;
  a.I = I;
  a.T = T;
  a.P = P;
  a.inv_mf = (float)(1.0 / ((double)nb * (double)h->ncell));
  a.g_out = h->g[0];
  a.loss_part = h->loss_part;
  return launch_conv<HEAD, kBZF>(h, nb, a, st);
}

int check_batch(const sx_cnn *h, int nb) {
  if (!h) return set_error(SX_ERR_ARG, "null proposer");
  if (nb < 1 || nb > h->max_batch) return set_error(SX_ERR_ARG, "batch size outside 1..max_batch");
  return SX_OK;
}

}  // namespace

extern "C" {

int64_t sx_cnn_num_params(void) { return kNParam; }

int sx_cnn_create(sx_cnn **out, const int n[3], int max_batch) {
  if (!out || !n) return set_error(SX_ERR_ARG, "null argument");
  *out = nullptr;
  for (int k = 0; k < 3; ++k)
    if (n[k] < 1 || n[k] > 4096) return set_error(SX_ERR_ARG, "every n[k] must be in 1..4096");
  if (max_batch < 1 || max_batch > 65535) return set_error(SX_ERR_ARG, "max_batch must be in 1..65535");
  const long long ncell = (long long)n[0] * n[1] * n[2];
  if (ncell * max_batch > (1LL << 34)) return set_error(SX_ERR_ARG, "max_batch x sites too large");
  sx_cnn *h = new (std::nothrow) sx_cnn();
  if (!h) return set_error(SX_ERR_OOM, "host allocation failed");
  for (int k = 0; k < 3; ++k) h->n[k] = n[k];
  h->ncell = ncell;
  h->max_batch = max_batch;
  h->tiles_x = (n[0] + kBX - 1) / kBX;
  h->tiles_y = (n[1] + kBY - 1) / kBY;
  h->nslot = wgrad_slots(h, max_batch);
  h->nloss = head_blocks(h, max_batch);
  const size_t sites = (size_t)ncell * max_batch;
  cudaError_t e = cudaSuccess;
  auto step = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  step(dalloc(&h->w, kNParam));
  step(dalloc(&h->m, kNParam));
  step(dalloc(&h->v, kNParam));
  step(dalloc(&h->grad, kNParam));
  step(dalloc(&h->wop, (size_t)2 * kLayers * kWBytes));
  for (int k = 0; k < 3; ++k) step(dalloc(&h->act[k], sites * kC));
  step(dalloc(&h->X, sites * kC));
  for (int k = 0; k < 2; ++k) step(dalloc(&h->g[k], sites * kC));
  for (int l = 0; l < kLayers; ++l) step(dalloc(&h->part[l], (size_t)h->nslot * kPart));
  step(dalloc(&h->loss_part, (size_t)h->nloss));
  step(dalloc(&h->loss, 1));
  step(dalloc(&h->s_dev, (size_t)max_batch));
  step(dalloc(&h->err, 1));
  if (e == cudaSuccess) e = cudaMemset(h->w, 0, kNParam * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(h->m, 0, kNParam * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(h->v, 0, kNParam * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(h->wop, 0, (size_t)2 * kLayers * kWBytes);
  if (e == cudaSuccess) e = cudaMemset(h->err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    sx_cnn_destroy(h);
    return cuda_error(e, "sx_cnn_create");
  }
  *out = h;
  return SX_OK;
}

void sx_cnn_destroy(sx_cnn *h) {
  if (!h) return;
  void *ptrs[] = {h->w,  h->m,    h->v,    h->grad,    h->wop,     h->act[0], h->act[1], h->act[2],
                  h->X,  h->g[0], h->g[1], h->part[0], h->part[1], h->part[2], h->part[3], h->loss_part,
                  h->loss, h->s_dev, h->err};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  delete h;
}

int sx_cnn_set_params(sx_cnn *h, const float *params_host) {
  if (!h || !params_host) return set_error(SX_ERR_ARG, "null argument");
  cudaError_t e = cudaMemcpy(h->w, params_host, kNParam * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(h->m, 0, kNParam * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(h->v, 0, kNParam * sizeof(float));
  if (e != cudaSuccess) return cuda_error(e, "sx_cnn_set_params");
  h->adam_t = 0;
  k_build_ops<<<(kNParam + 255) / 256, 256>>>(h->w, h->wop);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e == cudaSuccess ? SX_OK : cuda_error(e, "sx_cnn_set_params");
}

int sx_cnn_get_params(sx_cnn *h, float *params_host) {
  if (!h || !params_host) return set_error(SX_ERR_ARG, "null argument");
  cudaError_t e = cudaMemcpy(params_host, h->w, kNParam * sizeof(float), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SX_OK : cuda_error(e, "sx_cnn_get_params");
}

int sx_cnn_pack(sx_cnn *h, const double *I, int64_t i_stride, const double *A, const double *B, int64_t ab_stride,
                const double *s, int nb, uint16_t *X, void *stream) {
  int rc = check_batch(h, nb);
  if (rc) return rc;
  if (!I || !A || !B || !s || !X) return set_error(SX_ERR_ARG, "null pointer");
  if (!aligned8(I) || !aligned8(A) || !aligned8(B) || !aligned8(s) || !aligned16(X))
    return set_error(SX_ERR_ARG, "misaligned pointer (doubles 8 bytes, X 16 bytes)");
  if (i_stride < 3 * h->ncell || ab_stride < 0) return set_error(SX_ERR_ARG, "bad sample stride");
  cudaStream_t st = (cudaStream_t)stream;
  const long long total = h->ncell * nb;
  k_pack<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(I, i_stride, A, B, ab_stride, s, h->ncell, nb, X);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SX_OK : cuda_error(e, "sx_cnn_pack");
}

int sx_cnn_forward(sx_cnn *h, const uint16_t *X, const double *I, int nb, double *P, void *stream) {
  int rc = check_batch(h, nb);
  if (rc) return rc;
  if (!X || !I || !P) return set_error(SX_ERR_ARG, "null pointer");
  if (!aligned16(X) || !aligned8(I) || !aligned8(P)) return set_error(SX_ERR_ARG, "misaligned pointer");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = forward(h, X, I, nullptr, nb, P, st);
  if (e != cudaSuccess) return cuda_error(e, "sx_cnn_forward");
  return check_err(h, st);
}

int sx_cnn_loss_grad(sx_cnn *h, const uint16_t *X, const double *I, const double *T, int nb, float *grad,
                     double *loss_host, void *stream) {
  int rc = check_batch(h, nb);
  if (rc) return rc;
  if (!X || !I || !T) return set_error(SX_ERR_ARG, "null pointer");
  if (!aligned16(X) || !aligned8(I) || !aligned8(T) || (grad && ((uintptr_t)grad & 3u)))
    return set_error(SX_ERR_ARG, "misaligned pointer");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = forward(h, X, I, T, nb, nullptr, st);
  // backward: layer l's weight gradient from (g_out, act_in); input gradient masked by act_in > 0
  const uint16_t *ins[kLayers] = {X, h->act[0], h->act[1], h->act[2]};
  float *gcur = h->g[0], *gnext = h->g[1];
  for (int l = kLayers - 1; l >= 0 && e == cudaSuccess; --l) {
    e = launch_wgrad(h, nb, gcur, ins[l], h->part[l], st);
    if (l > 0 && e == cudaSuccess) {
      ConvArgs a{};
      a.g_in = gcur;
      a.wop = h->wop + (size_t)(2 * l + 1) * kWBytes;
      a.mask = ins[l];
      a.g_out = gnext;
      e = launch_conv<DGRAD, kBZD>(h, nb, a, st);
      float *t = gcur;
      gcur = gnext;
      gnext = t;
    }
  }
  if (e == cudaSuccess) {
    ReduceArgs r;
    for (int l = 0; l < kLayers; ++l) r.part[l] = h->part[l];
    r.nslot = wgrad_slots(h, nb);
    r.grad = grad ? grad : h->grad;
    r.loss_part = h->loss_part;
    r.nloss = head_blocks(h, nb);
    r.inv_m = 1.0 / ((double)nb * (double)h->ncell);
    r.loss = h->loss;
    k_grad_reduce<<<dim3((kPart + 31) / 32, kLayers + 1), dim3(32, 8), 0, st>>>(r);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_error(e, "sx_cnn_loss_grad");
  if (loss_host) {
    e = cudaMemcpyAsync(loss_host, h->loss, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_error(e, "sx_cnn_loss_grad");
  }
  return check_err(h, st);
}

int sx_cnn_adam_step(sx_cnn *h, const float *grad, const sx_adam_params *p, void *stream) {
  if (!h || !p) return set_error(SX_ERR_ARG, "null argument");
  if (!(p->lr > 0.0) || !(p->beta1 >= 0.0 && p->beta1 < 1.0) || !(p->beta2 >= 0.0 && p->beta2 < 1.0) ||
      !(p->eps > 0.0))
    return set_error(SX_ERR_ARG, "Adam needs lr > 0, 0 <= beta < 1, eps > 0");
  if (grad && ((uintptr_t)grad & 3u)) return set_error(SX_ERR_ARG, "misaligned gradient");
  h->adam_t += 1;
  const double c1 = 1.0 / (1.0 - pow(p->beta1, (double)h->adam_t));
  const double c2 = 1.0 / (1.0 - pow(p->beta2, (double)h->adam_t));
  k_adam<<<(kNParam + 255) / 256, 256, 0, (cudaStream_t)stream>>>(h->w, h->m, h->v, grad ? grad : h->grad,
                                                                    (float)p->lr, (float)p->beta1, (float)p->beta2,
                                                                    (float)p->eps, (float)c1, (float)c2, h->wop);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SX_OK : cuda_error(e, "sx_cnn_adam_step");
}

int sx_cnn_interpolate(sx_cnn *h, double *chain, int nimg, void *stream) {
  if (!h || !chain) return set_error(SX_ERR_ARG, "null argument");
  if (nimg < 3 || nimg - 2 > 65535) return set_error(SX_ERR_ARG, "nimg must be in 3..65537");
  if (!aligned8(chain)) return set_error(SX_ERR_ARG, "misaligned chain");
  if (nimg - 2 > h->max_batch) return set_error(SX_ERR_ARG, "nimg - 2 exceeds max_batch");
  const dim3 grid((unsigned)((h->ncell + 255) / 256), (unsigned)(nimg - 2));
  k_interp<<<grid, 256, 0, (cudaStream_t)stream>>>(chain, nimg, h->ncell, h->s_dev);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SX_OK : cuda_error(e, "sx_cnn_interpolate");
}

int sx_cnn_propose(sx_cnn *h, double *chain, int nimg, void *stream) {
  int rc = sx_cnn_interpolate(h, chain, nimg, stream);
  if (rc) return rc;
  const int nb = nimg - 2;
  double *I = chain + (size_t)3 * h->ncell;
  rc = sx_cnn_pack(h, I, 3 * h->ncell, chain, chain + (size_t)(nimg - 1) * 3 * h->ncell, 0, h->s_dev, nb, h->X,
                   stream);
  if (rc) return rc;
  return sx_cnn_forward(h, h->X, I, nb, I, stream);
}

}  // extern "C"
