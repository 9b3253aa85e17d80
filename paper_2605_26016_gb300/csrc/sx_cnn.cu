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
// the ReLU mask (input gradient).
//
// Weight gradients sum g_out[s][o] x act[s + tap][c] over all sites: CUDA-core
// FMAs on a shared-memory window, per-CTA partial sums in FP32 reduced over
// CTAs in FP64 in a fixed order (deterministic).
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <new>

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
constexpr int kBZD = 2;               // output z planes per CTA, input gradient
constexpr int kZW = 8;                // z planes per weight-gradient CTA (two at a time)
constexpr int kPart = kTaps * 256 + 16;  // one partial: gw[tap][o][c] then gb[o]
constexpr int kWgThreads = 216;          // 2 halves x 27 taps x 4 input-channel quads

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
  double inv_m;               // HEAD: 1 / (nb ncell)
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
        double Z[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) Z[k] = p.I[i0 + k * p.ncell] + (double)(__uint_as_float(r[k]) + bias[k]);
        const double rn = 1.0 / sqrt(Z[0] * Z[0] + Z[1] * Z[1] + Z[2] * Z[2]);
        const double P0 = Z[0] * rn, P1 = Z[1] * rn, P2 = Z[2] * rn;
        if (p.P) {
          p.P[i0] = P0;
          p.P[i0 + p.ncell] = P1;
          p.P[i0 + 2 * p.ncell] = P2;
        }
        if (p.T) {
          const double T0 = p.T[i0], T1 = p.T[i0 + p.ncell], T2 = p.T[i0 + 2 * p.ncell];
          const double dot = P0 * T0 + P1 * T1 + P2 * T2;
          lsum += 1.0 - dot;
          // dL/dP = -T / m; dL/dZ = (dL/dP - (dL/dP . P) P) / |Z|
          const double g0 = -T0 * p.inv_m, g1 = -T1 * p.inv_m, g2 = -T2 * p.inv_m;
          const double gp = g0 * P0 + g1 * P1 + g2 * P2;
          float4 *dst = reinterpret_cast<float4 *>(p.g_out + site * kC);
          dst[0] = make_float4((float)((g0 - gp * P0) * rn), (float)((g1 - gp * P1) * rn),
                               (float)((g2 - gp * P2) * rn), 0.0f);
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

// Weight and bias gradients of one layer: per CTA a 16 x 16 x kZW block of sites of one sample, processed two
// z planes at a time.  Thread (half, tap, quad) accumulates gw[tap][o][4 quad .. 4 quad + 3] for all 16 o over
// the sites of z plane `half` of each pair; threads with (tap, quad) index < 16 also sum gb[o].  Each half writes
// its own partial (2 per CTA).
struct WgradArgs {
  int nx, ny, nz, tiles_x;
  long long ncell;
  const float *g;          // gradient of the layer output [nb][ncell][16]
  const uint16_t *act;     // layer input [nb][ncell][16] BF16
  float *part;             // [2 * nblocks][kPart]
};

constexpr int kWgRows = kWX * kWY * 4;  // window of a z pair: 18 x 18 x 4 sites
constexpr size_t kWgSmem = (size_t)kWgRows * 32 + (size_t)2 * kBX * kBY * kC * 4;

__global__ void __launch_bounds__(kWgThreads) k_wgrad(const WgradArgs p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint16_t *sA = reinterpret_cast<uint16_t *>(smem);                   // [row][16] BF16
  float *sG = reinterpret_cast<float *>(smem + (size_t)kWgRows * 32);  // [zl][y][x][16]
  const int tid = threadIdx.x;
  const int half = tid / 108, task = tid % 108;
  const int tap = task >> 2, quad = task & 3;
  const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
  const int bxy = blockIdx.x;
  const int x0 = (bxy % p.tiles_x) * kBX, y0 = (bxy / p.tiles_x) * kBY, zb = blockIdx.y * kZW;
  const long long sbase = (long long)blockIdx.z * p.ncell;
  float acc[16][4];
#pragma unroll
  for (int o = 0; o < 16; ++o)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[o][c] = 0.0f;
  float gb = 0.0f;
  for (int z0 = zb; z0 < zb + kZW && z0 < p.nz; z0 += 2) {
    __syncthreads();
    for (int e = tid; e < kWgRows * 2; e += kWgThreads) {
      const int ch = e & 1, r = e >> 1;
      const int xw = r % kWX, q = r / kWX, yw = q % kWY, zw = q / kWY;
      const int gx = x0 - 1 + xw, gy = y0 - 1 + yw, gz = z0 - 1 + zw;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (gx >= 0 && gx < p.nx && gy >= 0 && gy < p.ny && gz >= 0 && gz < p.nz)
        v = __ldg(reinterpret_cast<const uint4 *>(p.act + (sbase + ((long long)gz * p.ny + gy) * p.nx + gx) * kC) + ch);
      reinterpret_cast<uint4 *>(sA)[2 * r + ch] = v;
    }
    for (int e = tid; e < 2 * kBX * kBY * 4; e += kWgThreads) {
      const int q4 = e & 3, s = e >> 2;
      const int xl = s % kBX, yl = (s / kBX) % kBY, zl = s / (kBX * kBY);
      const int gx = x0 + xl, gy = y0 + yl, gz = z0 + zl;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gx < p.nx && gy < p.ny && gz < p.nz)
        v = __ldg(reinterpret_cast<const float4 *>(p.g + (sbase + ((long long)gz * p.ny + gy) * p.nx + gx) * kC) + q4);
      reinterpret_cast<float4 *>(sG)[4 * s + q4] = v;
    }
    __syncthreads();
    const float4 *gp = reinterpret_cast<const float4 *>(sG) + (size_t)half * kBX * kBY * 4;
    for (int yl = 0; yl < kBY; ++yl) {
      const int rowb = ((half + 1 + dz) * kWY + (yl + 1 + dy)) * kWX + 1 + dx;
#pragma unroll 2
      for (int xl = 0; xl < kBX; ++xl) {
        const uint2 av = *reinterpret_cast<const uint2 *>(sA + (rowb + xl) * kC + 4 * quad);
        const float a0 = bf16_lo(av.x), a1 = bf16_hi(av.x), a2 = bf16_lo(av.y), a3 = bf16_hi(av.y);
        const float4 *gs = gp + (yl * kBX + xl) * 4;
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          const float4 g = gs[q4];
          const float gv[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[4 * q4 + j][0] = fmaf(gv[j], a0, acc[4 * q4 + j][0]);
            acc[4 * q4 + j][1] = fmaf(gv[j], a1, acc[4 * q4 + j][1]);
            acc[4 * q4 + j][2] = fmaf(gv[j], a2, acc[4 * q4 + j][2]);
            acc[4 * q4 + j][3] = fmaf(gv[j], a3, acc[4 * q4 + j][3]);
          }
        }
      }
    }
    if (task < 16) {
      const float *gsum = sG + (size_t)half * kBX * kBY * kC + task;
      for (int s = 0; s < kBX * kBY; ++s) gb += gsum[(size_t)s * kC];
    }
  }
  const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  float *out = p.part + (size_t)(2 * blk + half) * kPart;
#pragma unroll
  for (int o = 0; o < 16; ++o)
    *reinterpret_cast<float4 *>(out + tap * 256 + o * 16 + 4 * quad) =
        make_float4(acc[o][0], acc[o][1], acc[o][2], acc[o][3]);
  if (task < 16) out[kTaps * 256 + task] = gb;
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
  const dim3 grid((unsigned)(h->tiles_x * h->tiles_y), (unsigned)((h->n[2] + kZW - 1) / kZW), (unsigned)nb);
  k_wgrad<<<grid, kWgThreads, kWgSmem, st>>>(a);
  return cudaGetLastError();
}

long long wgrad_slots(const sx_cnn *h, int nb) {
  return 2LL * h->tiles_x * h->tiles_y * ((h->n[2] + kZW - 1) / kZW) * nb;
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
  a.inv_m = 1.0 / ((double)nb * (double)h->ncell);
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
  if (max_batch < 1) return set_error(SX_ERR_ARG, "max_batch must be >= 1");
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
