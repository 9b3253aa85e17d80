// Dense multi-channel convolution backend on the 5th-generation tensor cores (tcgen05).
//
// The dense backend of the paper evaluates the field as a convolution of the
// sublattice spin channels with a compact regular kernel ("Backend
// representations": dense sublattice convolution, kernel table K_ab^{alpha beta}(delta)).
// With channels c = alpha nsub + a (component alpha, sublattice a; C = 3 nsub)
//
//   b_c(x, y, z) = sum_{dy,dz} sum_{dx} sum_{c'} K_{c c'}(dx, dy, dz) S_{c'}(x + dx, y + dy, z + dz),
//
// and every 3x3 tensor tap (exchange, DMI, anisotropic exchange) and every
// sublattice pair is one block of the channel matrix K_{c c'}.
//
// Implicit GEMM per CTA.  A tile is XO output x positions (XO = floor(64 / C))
// times an 8 (y) x 16 (z) block of rows.  For one kernel plane (dy, dz):
//
//   D[m][n] += sum_k A_{dy,dz}[m][k] B_{dy,dz}[k][n],   m = (y, z) row (M = 128),
//   k = (x_in, c') (K = (XO + 2 rx) C, padded), n = (x_out, c) (N = 64),
//   A[m][k] = S_{c'}(x0 - rx + x_in, y + dy, z + dz),
//   B[k][n] = K_{c c'}(x_in - rx - x_out, dy, dz)   (zero outside |dx| <= rx).
//
// B is a channel-blocked Toeplitz band along x; its density is
// (2 rx + 1) / (XO + 2 rx) of the channel-dense product (7/27 for one
// sublattice with rx = 3), where a Toeplitz matrix over 128 x positions of a
// single channel would be 7/134.
//
//  * A: a pack kernel writes each tile column's input window (x window times
//    channels along K, with periodic wrap and zero open faces applied) as
//    16-byte K chunks in the canonical no-swizzle K-major operand layout; the
//    tile kernel stages its whole window with one 4-D TMA tile load
//    (cp.async.bulk.tensor) onto an mbarrier.  Row (y, z) of the window sits at
//    16 (y + yr z) bytes inside a chunk, so the operand of plane (dy, dz) is the
//    same window seen from a start address shifted by 16 (dy + yr dz) bytes.
//  * B: built in shared memory from the plane's K_{c c'}(dx) values, double
//    buffered: the band of plane p+1 is written while the MMAs of plane p run
//    (the zero pattern outside the band is written once).
//  * One thread issues tcgen05.mma (kind::tf32, or kind::f16 with BF16 hi+lo
//    operands and three MMAs per K step) into a 64-column FP32 TMEM
//    accumulator; tcgen05.commit arrives on the buffer's mbarrier.  Every wait
//    is bounded and sets an error flag instead of hanging.
//  * Epilogue: tcgen05.ld of the accumulator, on-site terms, FP32 or FP64 store.
#include <cuda.h>
#include <cudaTypedefs.h>
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

constexpr int kTcTY = 8;        // output y per tile (one core-matrix row group)
constexpr int kTcTZ = 16;       // output z per tile
constexpr int kTcN = 64;        // MMA N: output x positions x channels, padded
constexpr int kTcRMax = 3;      // taps within |d| <= 3 on every axis
constexpr int kTcMaxSub = 4;
constexpr int kTcIssuers = 2;                      // warps 0-1 issue the MMAs (planes alternate between them)
constexpr int kTcThreads = 32 * (kTcIssuers + 3);  // warps 2-4 build the B bands
constexpr int kTcMaxPlanes = (2 * kTcRMax + 1) * (2 * kTcRMax + 1);
constexpr int kTcPackRows = 32;  // window rows per pack block
constexpr int kTcPackThreads = 256;
constexpr int kTcBuilders = 96;  // threads of the three builder warps
constexpr int kTcMaxRing = 4;    // B buffers of the plane ring
constexpr int kTcMaxK = 144;     // largest K of a tile, (XO + 2 kTcRMax) C rounded up
constexpr size_t kTcSmemMax = 227 * 1024;

template <int NSUB>
struct TcShape {
  static constexpr int C = 3 * NSUB;
  static constexpr int XO = kTcN / C;  // 21, 10, 7, 5
  static constexpr int NE_MAX = XO * C * C * (2 * kTcRMax + 1);
  static constexpr int EPT_MAX = NSUB == 1 ? 16 : NSUB == 2 ? 30 : 44;  // band entries per builder thread
  static constexpr int XP = XO | 1;  // odd x pitch of the epilogue staging
  static constexpr int STAGE_BYTES = C * 128 * XP * 4;
};

// Tile geometry of a plan.
struct TcGeo {
  int nsub, C, xo;
  int rx, ry, rz;
  int kb;          // K of a tile: (xo + 2 rx) C rounded up to the MMA K step
  int nch;         // 16-byte K chunks per operand copy
  int yr, zr;      // window rows: 8 + 2 ry, 16 + 2 rz
  int nbx, nby, nbz;
  int yp, zp;      // rows of the packed array: 8 nby + 2 ry, 16 nbz + 2 rz
};

struct TcArgs {
  TcGeo t;
  int nx, ny, nz, px, py, pz;
  long long ncell;
  int nplanes;
  int plane_dy[kTcMaxPlanes], plane_dz[kTcMaxPlanes];
  const float *Jp;       // [nplanes][C][C][2 rx + 1]: K_{c c'}(dx) of each plane
  const uint32_t *ent;   // [ept][96] band entries: B byte offset | index into a plane's values << 18
  int ept;               // band entries per builder thread
  int jp_smem;           // 1: the plane values are staged in shared memory
  int nbuf;              // B buffers of the plane ring (2..4)
  OnSiteT<float> os;
  int onsite;
  int *err;              // set to 1 if a bounded wait gave up
  unsigned win_bytes;    // window bytes (all operand copies)
  unsigned b_bytes;      // one B buffer (all operand copies)
  unsigned bar_off;      // offset of the barrier block in shared memory
  unsigned smem;         // dynamic shared memory of the tile kernel
  int grid;              // persistent CTAs
};

struct TcPlan {
  int tf32;
  int nsm;
  int ctas;          // CTAs per SM the layout is sized for (1 or 2)
  size_t jp_bytes;   // plane values (bytes)
  TcArgs base;
  CUtensorMap tmap;     // 4-D view of Wp: (4 yp words, zp, nch, ncopy nbx)
  uint4 *Wp;            // packed input windows
  float *Jp;
  uint32_t *ent;
  float *St, *F0, *Bf;  // Heun workspaces [3 nsub][ncell]
  float *Th;            // thermal field of the step
  int *err;
};

namespace {

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, no swizzle: lbo = byte distance of K-adjacent core matrices,
// sbo = byte distance of core matrices 8 rows apart
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ uint32_t to_tf32(float f) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
  return r;
}

// BF16 split v = hi + lo, lo = RN(v - hi)
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

template <typename T>
__device__ __forceinline__ float as_f32(T v) {
  return cvt<float>(v);
}

// FP32 -> output type by integer bit operations (the FP64 conversion pipe runs at ~1/70 of the FP32
// rate), keeping NaN and infinity non-finite so that a non-finite field stays visible
template <typename T>
__device__ __forceinline__ T from_f32(float f);
template <>
__device__ __forceinline__ float from_f32<float>(float f) {
  return f;
}
template <>
__device__ __forceinline__ double from_f32<double>(float f) {
  const unsigned b = __float_as_uint(f), a = b & 0x7FFFFFFFu;
  if (a >= 0x7F800000u) return __hiloint2double((int)((b & 0x80000000u) | 0x7FF00000u | ((a & 0x7FFFFFu) >> 3)), (int)(b << 29));
  return f32_to_f64(f);
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

__device__ __forceinline__ int wrap_or_neg(int c, int n, int periodic) {
  if (c >= 0 && c < n) return c;
  if (!periodic) return -1;
  c %= n;
  return c < 0 ? c + n : c;
}

// Packs the input windows of the tile columns: element k = (x_in, c') of K chunk q = k / EPC,
// window row (ye, ze), tile column bx, operand copy cp (TF32: one; BF16: hi, lo) goes to the
// 16-byte unit ((((bx ncopy + cp) nch + q) zp + ze) yp + ye).  Grid (nbx, zp, ceil(yp / 32)),
// 256 threads: lane l of a warp reads window position x_in = l (XO + 2 rx <= 32) of every
// channel of a row, so the loads of a warp are x-contiguous and independent.
template <int NSUB, bool TF32, typename Tin>
__global__ void __launch_bounds__(kTcPackThreads) k_tc_pack(const TcArgs a, const Tin *__restrict__ S,
                                                            uint4 *__restrict__ Wp) {
  constexpr int C = TcShape<NSUB>::C, XO = TcShape<NSUB>::XO;
  constexpr int NCOPY = TF32 ? 1 : 2;
  constexpr int NW = kTcPackThreads / 32;
  __shared__ float st[kTcPackRows][kTcMaxK + 1];
  const TcGeo &t = a.t;
  const int bx = blockIdx.x, ze = blockIdx.y, ye0 = blockIdx.z * kTcPackRows;
  const int XW = XO + 2 * t.rx;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int z = wrap_or_neg(ze - t.rz, a.nz, a.pz);
  const int x = lane < XW ? wrap_or_neg(bx * XO - t.rx + lane, a.nx, a.px) : -1;
#pragma unroll
  for (int rr = 0; rr < kTcPackRows / NW; ++rr) {
    const int r = warp + rr * NW, ye = ye0 + r;
    const int y = ye < t.yp ? wrap_or_neg(ye - t.ry, a.ny, a.py) : -1;
    const bool ok = (x | y | z) >= 0;
    const long long cell = ok ? ((long long)z * a.ny + y) * a.nx + x : 0;
    float v[C];
#pragma unroll
    for (int ch = 0; ch < C; ++ch) v[ch] = ok ? as_f32(S[(long long)ch * a.ncell + cell]) : 0.0f;
    if (lane < XW) {
#pragma unroll
      for (int ch = 0; ch < C; ++ch) st[r][lane * C + ch] = v[ch];
    }
  }
  __syncthreads();
  const int kval = XW * C;
  for (int idx = threadIdx.x; idx < NCOPY * t.nch * kTcPackRows; idx += kTcPackThreads) {
    const int r = idx % kTcPackRows, q = (idx / kTcPackRows) % t.nch, cp = idx / (kTcPackRows * t.nch);
    const int ye = ye0 + r;
    if (ye >= t.yp) continue;
    uint32_t w[4];
    if (TF32) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = q * 4 + u;
        w[u] = to_tf32(k < kval ? st[r][k] : 0.0f);
      }
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        uint16_t h[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int k = q * 8 + 2 * u + s;
          __nv_bfloat16 hi, lo;
          split_bf16(k < kval ? st[r][k] : 0.0f, hi, lo);
          h[s] = __bfloat16_as_ushort(cp == 0 ? hi : lo);
        }
        w[u] = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
      }
    }
    Wp[((((size_t)bx * NCOPY + cp) * t.nch + q) * t.zp + ze) * t.yp + ye] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

__device__ __forceinline__ float lds_f32(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint16_t lds_u16(uint32_t a) {
  uint16_t v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts_b32(uint32_t a, uint32_t v) {
  asm volatile("st.shared.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void sts_b16(uint32_t a, uint16_t v) {
  asm volatile("st.shared.b16 [%0], %1;" ::"r"(a), "h"(v) : "memory");
}
// tcgen05.commit of the calling warp's MMAs by one elected lane (warp converged)
__device__ __forceinline__ void commit_elected(uint64_t *mbar) {
  asm volatile(
      "{\n.reg .pred e;\nelect.sync _|e, 0xffffffff;\n"
      "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(saddr(mbar))
      : "memory");
}

// mbarriers and shared words of the tile kernel
struct TcBars {
  uint64_t win;                 // the tile's window landed (TMA transaction bytes)
  uint64_t full[kTcMaxRing];    // B buffer built (one arrival per builder thread)
  uint64_t empty[kTcMaxRing];   // B buffer consumed by its MMAs (tcgen05.commit)
  uint64_t acc;                 // every MMA of the tile complete (tcgen05.commit)
  uint32_t tmem;                // accumulator address from tcgen05.alloc
  int abort;                    // set by any thread whose bounded wait gave up
};

// bounded wait that also gives up once another thread of the CTA gave up
__device__ __forceinline__ bool wait_bar(uint64_t *mbar, uint32_t parity, TcBars *bar, int *err) {
  for (long it = 0; it < (1L << 24); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(saddr(mbar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (*(volatile int *)&bar->abort) return false;
    if (it > 1024) __nanosleep(64);
  }
  *(volatile int *)&bar->abort = 1;
  atomicExch(err, 1);
  return false;
}

// Field of the tiles of a persistent CTA: tile = blockIdx.x + k gridDim.x, each XO x positions
// times 8 y times 16 z, every channel.  Warp 0: lane 0 loads windows (TMA) and issues the MMAs;
// warps 1-3 build the B bands of the planes into a ring of nbuf buffers (full / empty
// mbarriers); all four warps run the epilogue of each tile.
template <int NSUB, bool TF32, typename Tin, typename Tout>
__global__ void __maxnreg__(200)
    k_tc_field(const __grid_constant__ CUtensorMap tmap, const TcArgs a, const Tin *__restrict__ S,
               Tout *__restrict__ out) {
  using Sh = TcShape<NSUB>;
  constexpr int C = Sh::C, XO = Sh::XO;
  constexpr int ESZ = TF32 ? 4 : 2, EPC = 16 / ESZ, KSTEP = TF32 ? 8 : 16, NCOPY = TF32 ? 1 : 2;
  extern __shared__ __align__(1024) unsigned char smem[];
  const TcGeo &t = a.t;
  unsigned char *win = smem;
  unsigned char *ring = smem + a.win_bytes;
  float *jsm = reinterpret_cast<float *>(ring + (size_t)a.nbuf * a.b_bytes);
  TcBars *bar = reinterpret_cast<TcBars *>(smem + a.bar_off);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int W = 2 * t.rx + 1, CCW = C * C * W;
  const int ntiles = t.nbx * t.nby * t.nbz;
  const uint32_t LBO_A = (uint32_t)(t.yr * t.zr * 16), SBO_A = (uint32_t)(t.yr * 16);
  const uint32_t LBO_B = kTcN * 16, SBO_B = 128;
  const uint32_t A_COPY = (uint32_t)t.nch * LBO_A;         // bytes of one window copy
  const uint32_t B_COPY = (uint32_t)(t.kb / EPC) * LBO_B;  // bytes of one B copy

  if (tid == 0) {
    bar->abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar->win)));
    // one tcgen05.commit per issuing warp that has planes
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&bar->acc)),
                 "r"(a.nplanes < kTcIssuers ? (a.nplanes > 0 ? a.nplanes : 1) : kTcIssuers));
    for (int b = 0; b < kTcMaxRing; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&bar->full[b])), "r"(kTcBuilders));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar->empty[b])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    static_assert(kTcN * kTcIssuers == 128, "the TMEM allocation below is 128 columns");
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(saddr(&bar->tmem)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // the zero pattern of the B buffers (only band entries are rewritten per plane), the band
  // entry table and, when it fits, the plane values
  for (uint32_t o = tid * 16u; o < (uint32_t)a.nbuf * a.b_bytes; o += kTcThreads * 16u)
    *reinterpret_cast<uint4 *>(ring + o) = make_uint4(0u, 0u, 0u, 0u);
  if (a.jp_smem)
    for (int i = tid; i < a.nplanes * CCW; i += kTcThreads) jsm[i] = a.Jp[i];
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = bar->tmem;
  // builder threads keep their band entries in registers for the whole kernel
  uint32_t my_ent[Sh::EPT_MAX];
#pragma unroll
  for (int i = 0; i < Sh::EPT_MAX; ++i)
    my_ent[i] = (warp >= kTcIssuers && i < a.ept) ? a.ent[i * kTcBuilders + tid - 32 * kTcIssuers] : 0xFFFFFFFFu;

  auto load_window = [&](int tile) {
    const int bx = tile % t.nbx, r = tile / t.nbx, by = r % t.nby, bz = r / t.nby;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(&bar->win)), "r"(a.win_bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(saddr(win)),
        "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(4 * by * kTcTY), "r"(bz * kTcTZ), "r"(0), "r"(bx * NCOPY),
        "r"(saddr(&bar->win))
        : "memory");
  };
  constexpr uint32_t fmt = TF32 ? 2u : 1u;
  constexpr uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);
  // descriptors advance by adding byte offsets / 16 to the start-address field (< 2^14 units)
  const uint64_t adesc0 = smem_desc(saddr(win), LBO_A, SBO_A);
  const uint64_t bdesc0 = smem_desc(saddr(ring), LBO_B, SBO_B);
  const uint32_t kc_step = KSTEP / EPC;

  bool live = true;  // this thread has not given up
  int win_wait = -1;  // lane 0 of warp 0: parity of a window load not yet waited for, else -1
  int acc_wait = -1;  // lane 0 of warp 0: parity of an accumulator commit not yet waited for, else -1
  if (tid == 0 && (int)blockIdx.x < ntiles) {
    load_window(blockIdx.x);
    win_wait = 0;
  }
  uint32_t P = 0;  // planes of the earlier tiles of this CTA (ring position)
  int k = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
    live = *(volatile int *)&bar->abort == 0;
    if (warp < kTcIssuers) {
      // each issuing warp runs its loop with warp-uniform descriptors (one elected lane issues) over
      // the planes p = warp, warp + kTcIssuers, ... into its own accumulator
      live = __all_sync(0xFFFFFFFFu, wait_bar(&bar->win, (uint32_t)k & 1u, bar, a.err));
      if (live) win_wait = -1;
      const uint32_t dacc = tmem + (uint32_t)(warp * kTcN);
      int issued = 0;
      for (int p = warp; p < a.nplanes && live; p += kTcIssuers) {
        const uint32_t Pp = P + (uint32_t)p, b = Pp % (uint32_t)a.nbuf;
        live = __all_sync(0xFFFFFFFFu, wait_bar(&bar->full[b], (Pp / (uint32_t)a.nbuf) & 1u, bar, a.err));
        if (!live) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t ad =
            adesc0 + (((uint32_t)(a.plane_dz[p] + t.rz) * SBO_A + (uint32_t)(a.plane_dy[p] + t.ry) * 16u) >> 4);
        const uint64_t bd = bdesc0 + ((b * a.b_bytes) >> 4);
        for (int ks = 0; ks < t.kb / KSTEP; ++ks) {
          const uint64_t ak = ad + ((ks * kc_step * LBO_A) >> 4), bk = bd + ((ks * kc_step * LBO_B) >> 4);
#pragma unroll
          for (int term = 0; term < (TF32 ? 1 : 3); ++term) {
            // BF16: K S = Kh Sh + Kl Sh + Kh Sl (the Kl Sl term is below FP32 resolution of the sum)
            const uint64_t at = ak + (term == 2 ? (A_COPY >> 4) : 0u), bt = bk + (term == 1 ? (B_COPY >> 4) : 0u);
            const uint32_t acc = (p > warp || ks > 0 || term > 0) ? 1u : 0u;
            if (TF32)
              asm volatile(
                  "{\n.reg .pred e, q;\nelect.sync _|e, 0xffffffff;\nsetp.ne.u32 q, %4, 0;\n"
                  "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n}\n" ::"r"(dacc),
                  "l"(at), "l"(bt), "r"(idesc), "r"(acc));
            else
              asm volatile(
                  "{\n.reg .pred e, q;\nelect.sync _|e, 0xffffffff;\nsetp.ne.u32 q, %4, 0;\n"
                  "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(dacc),
                  "l"(at), "l"(bt), "r"(idesc), "r"(acc));
          }
        }
        commit_elected(&bar->empty[b]);
        ++issued;
      }
      if (issued > 0) {  // also after a failed wait, so that the MMAs in flight can be waited for
        commit_elected(&bar->acc);
        acc_wait = k & 1;
      }
      // the next window may land once every MMA of this tile has read the current one
      if (live && a.nplanes > 0) {
        live = __all_sync(0xFFFFFFFFu, wait_bar(&bar->acc, (uint32_t)k & 1u, bar, a.err));
        if (live) acc_wait = -1;
      }
      __syncwarp();
    } else {
      const uint32_t ring_sa = saddr(ring), jsa = saddr(jsm);
      for (int p = 0; p < a.nplanes && live; ++p) {
        const uint32_t Pp = P + (uint32_t)p, b = Pp % (uint32_t)a.nbuf;
        if (Pp >= (uint32_t)a.nbuf && !(live = wait_bar(&bar->empty[b], (Pp / (uint32_t)a.nbuf - 1u) & 1u, bar, a.err)))
          break;
        const uint32_t Bsa = ring_sa + b * a.b_bytes;
        // in chunks of 16 entries: the chunk's loads before its stores
#pragma unroll
        for (int i0 = 0; i0 < Sh::EPT_MAX; i0 += 16) {
          constexpr int CH = 16;
          float v[CH];
          if (a.jp_smem) {
            const uint32_t jp = jsa + (uint32_t)(p * CCW) * 4u;
#pragma unroll
            for (int i = 0; i < CH; ++i)
              if (i0 + i < Sh::EPT_MAX)
                v[i] = my_ent[i0 + i] != 0xFFFFFFFFu ? lds_f32(jp + (my_ent[i0 + i] >> 18) * 4u) : 0.0f;
          } else {
            const float *Jpl = a.Jp + (size_t)p * CCW;
#pragma unroll
            for (int i = 0; i < CH; ++i)
              if (i0 + i < Sh::EPT_MAX)
                v[i] = my_ent[i0 + i] != 0xFFFFFFFFu ? __ldg(Jpl + (my_ent[i0 + i] >> 18)) : 0.0f;
          }
#pragma unroll
          for (int i = 0; i < CH; ++i) {
            if (i0 + i >= Sh::EPT_MAX || my_ent[i0 + i] == 0xFFFFFFFFu) continue;
            const uint32_t off = Bsa + (my_ent[i0 + i] & 0x3FFFFu);
            if (TF32) {
              sts_b32(off, to_tf32(v[i]));
            } else {
              __nv_bfloat16 hi, lo;
              split_bf16(v[i], hi, lo);
              sts_b16(off, __bfloat16_as_ushort(hi));
              sts_b16(off + B_COPY, __bfloat16_as_ushort(lo));
            }
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&bar->full[b])) : "memory");
      }
    }
    P += (uint32_t)a.nplanes;
    // epilogue: accumulator -> staging in the (now idle) B ring -> x-contiguous global stores
    if (live && a.nplanes > 0) live = wait_bar(&bar->acc, (uint32_t)k & 1u, bar, a.err);
    __syncthreads();
    if (*(volatile int *)&bar->abort) break;  // uniform: read after the barrier
    float *stage = reinterpret_cast<float *>(ring);  // [c][128 rows][XP]: the tile's field, x fastest
    const int bx = tile % t.nbx, rr = tile / t.nbx, by = rr % t.nby, bz = rr / t.nby;
    {
      // thread m < 128 owns accumulator row m = (y, z) = (m % 8, m / 8): all x positions and channels
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int m = warp * 32 + lane;
      float v[kTcN];
      if (warp < 4) {
#pragma unroll
        for (int i = 0; i < kTcN; ++i) v[i] = 0.0f;
        // fixed order: accumulator 0 (planes 0, 2, ...) + accumulator 1 (planes 1, 3, ...)
#pragma unroll
        for (int w = 0; w < kTcIssuers; ++w) {
          if (w >= a.nplanes) break;
#pragma unroll
          for (int c0 = 0; c0 < kTcN; c0 += 16) {
            uint32_t r[16];
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(w * kTcN + c0);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 16; ++q) v[c0 + q] += __uint_as_float(r[q]);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      if (warp < 4 && a.onsite) {
        // Zeeman and anisotropy from the spins at the row's own sites, read from the window (the
        // operand values: TF32-rounded, or BF16 hi + lo)
        const uint32_t rowoff = (uint32_t)((m >> 3) + t.rz) * SBO_A + (uint32_t)((m & 7) + t.ry) * 16u;
#pragma unroll
        for (int j = 0; j < XO; ++j) {
#pragma unroll
          for (int s = 0; s < NSUB; ++s) {
            float sv[3];
#pragma unroll
            for (int al = 0; al < 3; ++al) {
              const uint32_t kk = (uint32_t)((j + t.rx) * C + al * NSUB + s);
              const uint32_t off = (kk / EPC) * LBO_A + rowoff + (kk % EPC) * ESZ;
              if (TF32) {
                sv[al] = lds_f32(saddr(win) + off);
              } else {
                sv[al] = __bfloat162float(__ushort_as_bfloat16(lds_u16(saddr(win) + off))) +
                         __bfloat162float(__ushort_as_bfloat16(lds_u16(saddr(win) + A_COPY + off)));
              }
            }
            const float q = a.os.twoK[s] * (sv[0] * a.os.axis[s][0] + sv[1] * a.os.axis[s][1] + sv[2] * a.os.axis[s][2]);
#pragma unroll
            for (int al = 0; al < 3; ++al) v[j * C + al * NSUB + s] += a.os.zee[s][al] + q * a.os.axis[s][al];
          }
        }
      }
      // column n = j C + c goes to stage[(c * 128 + m) * XP + j] (XP odd: conflict-free for both phases)
      if (warp < 4) {
#pragma unroll
        for (int n = 0; n < XO * C; ++n) stage[((n % C) * 128 + m) * Sh::XP + n / C] = v[n];
      }
    }
    __syncthreads();
    // the window is no longer read: the next tile's window may land while the field is stored
    if (tid == 0 && tile + (int)gridDim.x < ntiles) {
      load_window(tile + (int)gridDim.x);
      win_wait = (k + 1) & 1;
    }
    {
      // row r = c * 128 + m of the stage is a contiguous x-run of the output: one warp per run
      const int xs = bx * XO, nxr = min(XO, a.nx - xs);
      for (int r = warp; r < C * 128; r += kTcThreads / 32) {
        const int c = r >> 7, m = r & 127;
        const int y = by * kTcTY + (m & 7), z = bz * kTcTZ + (m >> 3);
        if (y >= a.ny || z >= a.nz || lane >= nxr) continue;
        out[(long long)c * a.ncell + ((long long)z * a.ny + y) * a.nx + xs + lane] =
            from_f32<Tout>(stage[r * Sh::XP + lane]);
      }
    }
    __syncthreads();
    // the staging area is the B ring of the next tile: restore its zero pattern outside the band
    for (uint32_t o = tid * 16u; o < (uint32_t)Sh::STAGE_BYTES; o += kTcThreads * 16u)
      *reinterpret_cast<uint4 *>(ring + o) = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  }
  // after a wait gave up: let copies and MMAs still in flight finish (bounded) before the CTA's
  // shared memory and TMEM are released
  if (tid == 0) {
    if (win_wait >= 0) wait_parity(&bar->win, (uint32_t)win_wait, a.err);
    if (acc_wait >= 0) wait_parity(&bar->acc, (uint32_t)acc_wait, a.err);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

template <int NSUB, bool TF32, typename Tin>
cudaError_t launch_pack(const TcPlan &tp, const Tin *S, cudaStream_t st) {
  const TcGeo &t = tp.base.t;
  const dim3 grid(t.nbx, t.zp, (t.yp + kTcPackRows - 1) / kTcPackRows);
  k_tc_pack<NSUB, TF32, Tin><<<grid, kTcPackThreads, 0, st>>>(tp.base, S, tp.Wp);
  return cudaGetLastError();
}

template <int NSUB, bool TF32, typename Tin, typename Tout>
cudaError_t launch_tile(const TcPlan &tp, const TcArgs &a, const Tin *S, Tout *out, cudaStream_t st) {
  k_tc_field<NSUB, TF32, Tin, Tout><<<a.grid, kTcThreads, a.smem, st>>>(tp.tmap, a, S, out);
  return cudaGetLastError();
}

template <int NSUB, bool TF32, typename Tin, typename Tout>
cudaError_t field_nt(const TcPlan &tp, const TcArgs &a, const Tin *S, Tout *out, cudaStream_t st) {
  cudaError_t e = launch_pack<NSUB, TF32, Tin>(tp, S, st);
  if (e == cudaSuccess) e = launch_tile<NSUB, TF32, Tin, Tout>(tp, a, S, out, st);
  return e;
}

template <typename Tin, typename Tout>
cudaError_t field_any(const TcPlan &tp, const TcArgs &a, const Tin *S, Tout *out, cudaStream_t st) {
  const bool f = tp.tf32 != 0;
  switch (a.t.nsub) {
    case 1: return f ? field_nt<1, true>(tp, a, S, out, st) : field_nt<1, false>(tp, a, S, out, st);
    case 2: return f ? field_nt<2, true>(tp, a, S, out, st) : field_nt<2, false>(tp, a, S, out, st);
    case 3: return f ? field_nt<3, true>(tp, a, S, out, st) : field_nt<3, false>(tp, a, S, out, st);
    default: return f ? field_nt<4, true>(tp, a, S, out, st) : field_nt<4, false>(tp, a, S, out, st);
  }
}

template <int NSUB, bool TF32>
cudaError_t set_smem_nt(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_tc_field<NSUB, TF32, double, double>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_field<NSUB, TF32, double, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_field<NSUB, TF32, float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
  return e;
}

template <int NSUB, bool TF32>
cudaError_t occupancy_nt(int bytes, int *occ) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_tc_field<NSUB, TF32, double, double>, kTcThreads,
                                                       (size_t)bytes);
}

cudaError_t occupancy(int nsub, bool tf32, int bytes, int *occ) {
  switch (nsub) {
    case 1: return tf32 ? occupancy_nt<1, true>(bytes, occ) : occupancy_nt<1, false>(bytes, occ);
    case 2: return tf32 ? occupancy_nt<2, true>(bytes, occ) : occupancy_nt<2, false>(bytes, occ);
    case 3: return tf32 ? occupancy_nt<3, true>(bytes, occ) : occupancy_nt<3, false>(bytes, occ);
    default: return tf32 ? occupancy_nt<4, true>(bytes, occ) : occupancy_nt<4, false>(bytes, occ);
  }
}

// Band entries of B in bank-balanced groups of 32: entry (x_out j, channel c, tap dxi, channel c')
// writes K_{c c'}(dxi - rx) at row n = j C + c, column k = (j + dxi) C + c'.  Grouping one entry
// of each shared-memory bank per warp store keeps the builders' stores conflict-free.  Returns the
// table [ept][96] (builder thread fastest) and ept.
std::vector<uint32_t> band_entries(const TcGeo &t, bool tf32, int &ept) {
  const int C = t.C, W = 2 * t.rx + 1, epc = tf32 ? 4 : 8, esz = tf32 ? 4 : 2;
  std::vector<std::vector<uint32_t>> bank(32);
  for (int j = 0; j < t.xo; ++j)
    for (int c = 0; c < C; ++c)
      for (int dxi = 0; dxi < W; ++dxi)
        for (int cq = 0; cq < C; ++cq) {
          const int n = j * C + c, k = (j + dxi) * C + cq;
          const uint32_t off = (uint32_t)(k / epc) * (kTcN * 16) + (uint32_t)(n >> 3) * 128u + (uint32_t)(n & 7) * 16u +
                               (uint32_t)(k % epc) * esz;
          bank[(off >> 2) & 31].push_back(off | ((uint32_t)((c * C + cq) * W + dxi) << 18));
        }
  size_t ngroup = 0;
  for (const auto &b : bank) ngroup = std::max(ngroup, b.size());
  ept = (int)((ngroup + 2) / 3);
  std::vector<uint32_t> tab((size_t)ept * kTcBuilders, 0xFFFFFFFFu);
  for (size_t g = 0; g < ngroup; ++g) {
    int lane = 0;
    for (const auto &b : bank)
      if (g < b.size()) tab[(g / 3) * kTcBuilders + (g % 3) * 32 + lane++] = b[g];
  }
  return tab;
}

cudaError_t set_smem(int nsub, bool tf32, int bytes) {
  switch (nsub) {
    case 1: return tf32 ? set_smem_nt<1, true>(bytes) : set_smem_nt<1, false>(bytes);
    case 2: return tf32 ? set_smem_nt<2, true>(bytes) : set_smem_nt<2, false>(bytes);
    case 3: return tf32 ? set_smem_nt<3, true>(bytes) : set_smem_nt<3, false>(bytes);
    default: return tf32 ? set_smem_nt<4, true>(bytes) : set_smem_nt<4, false>(bytes);
  }
}

int encode_window_map(TcPlan *tp, int ncopy) {
  const auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encode_fn());
  if (!enc) return set_error(SX_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  // 4-D view (words of the y rows, z, chunk, copy and tile column): the y rows of one chunk and
  // z plane are contiguous, so each box row is 16 (8 + 2 ry) bytes instead of one 16-byte unit
  const TcGeo &t = tp->base.t;
  const cuuint64_t dims[4] = {4ull * t.yp, (cuuint64_t)t.zp, (cuuint64_t)t.nch, (cuuint64_t)ncopy * t.nbx};
  const cuuint64_t strides[3] = {16ull * t.yp, 16ull * t.yp * t.zp, 16ull * t.yp * t.zp * t.nch};
  const cuuint32_t box[4] = {4u * (cuuint32_t)t.yr, (cuuint32_t)t.zr, (cuuint32_t)t.nch, (cuuint32_t)ncopy};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = enc(&tp->tmap, CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, tp->Wp, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(SX_ERR_CUDA, "cuTensorMapEncodeTiled rejected the window layout");
  return SX_OK;
}

// Shared-memory layout of the tile kernel for a ring of nbuf B buffers and `ctas` CTAs per SM:
// window | nbuf B buffers | plane values (when they fit) | barriers.  The ring also stages the
// epilogue (C x 128 rows x (xo | 1) floats).  False when it does not fit.
bool tc_layout(TcPlan &tp, int nbuf, int ctas) {
  TcArgs &a = tp.base;
  const TcGeo &t = a.t;
  const size_t stage_bytes = (size_t)t.C * 128 * (t.xo | 1) * 4;
  if (nbuf < 2 || nbuf > kTcMaxRing || (size_t)nbuf * a.b_bytes < stage_bytes) return false;
  const size_t budget = ctas == 2 ? kTcSmemMax / 2 - 1024 : kTcSmemMax;
  auto size = [&](bool jsm) {
    const size_t off = (size_t)a.win_bytes + (size_t)nbuf * a.b_bytes + (jsm ? tp.jp_bytes : 0);
    return ((off + 15) / 16) * 16 + 128;
  };
  bool jsm = size(true) <= budget;
  if (!jsm && size(false) > budget) return false;
  a.nbuf = nbuf;
  a.jp_smem = jsm ? 1 : 0;
  a.smem = (unsigned)size(jsm);
  a.bar_off = a.smem - 128;
  tp.ctas = ctas;
  return true;
}

// candidate (ring depth, CTAs per SM) pairs, the plan's default first: two CTAs per SM with the
// deepest ring that allows it, else one CTA with the deepest ring
std::vector<TcTiles> tc_tile_candidates_of(TcPlan &tp) {
  const TcArgs keep = tp.base;
  const int keep_ctas = tp.ctas;
  std::vector<TcTiles> out;
  for (int ctas : {2, 1})
    for (int nb = (ctas == 2 ? 3 : kTcMaxRing); nb >= 2; --nb)
      if (tc_layout(tp, nb, ctas)) out.push_back({nb, ctas});
  tp.base = keep;
  tp.ctas = keep_ctas;
  return out;
}

cudaError_t tc_set_grid(TcPlan &tp) {
  int occ = 1;
  const cudaError_t e = occupancy(tp.base.t.nsub, tp.tf32 != 0, (int)tp.base.smem, &occ);
  if (e != cudaSuccess) return e;
  const long long ntiles = (long long)tp.base.t.nbx * tp.base.t.nby * tp.base.t.nbz;
  tp.base.grid = (int)std::max(1LL, std::min(ntiles, (long long)tp.nsm * std::max(1, std::min(occ, tp.ctas))));
  return cudaSuccess;
}

}  // namespace

int tc_plan(sx_ctx *c) {
  if (c->prec != SX_PREC_BF16 && c->prec != SX_PREC_TF32)
    return set_error(SX_ERR_UNSUPPORTED, "the tensor-core backend computes the field in BF16 or TF32");
  const int nsub = c->lat.nsub;
  if (nsub > kTcMaxSub) return set_error(SX_ERR_UNSUPPORTED, "the tensor-core backend supports up to 4 sublattices");
  const bool tf32 = c->prec == SX_PREC_TF32;
  TcGeo t;
  t.nsub = nsub;
  t.C = 3 * nsub;
  t.xo = kTcN / t.C;
  t.rx = t.ry = t.rz = 0;
  for (int a = 0; a < nsub; ++a)
    for (const Tap &tp : c->taps[a]) {
      for (int k = 0; k < 3; ++k)
        if (abs(tp.d[k]) > kTcRMax)
          return set_error(SX_ERR_UNSUPPORTED, "the tensor-core backend takes taps within a 7x7x7 cell window");
      t.rx = std::max(t.rx, abs(tp.d[0]));
      t.ry = std::max(t.ry, abs(tp.d[1]));
      t.rz = std::max(t.rz, abs(tp.d[2]));
    }
  const int kstep = tf32 ? 8 : 16, epc = tf32 ? 4 : 8, ncopy = tf32 ? 1 : 2;
  t.kb = ((t.xo + 2 * t.rx) * t.C + kstep - 1) / kstep * kstep;
  t.nch = t.kb / epc;
  t.yr = kTcTY + 2 * t.ry;
  t.zr = kTcTZ + 2 * t.rz;
  t.nbx = (c->geo.nx + t.xo - 1) / t.xo;
  t.nby = (c->geo.ny + kTcTY - 1) / kTcTY;
  t.nbz = (c->geo.nz + kTcTZ - 1) / kTcTZ;
  t.yp = t.nby * kTcTY + 2 * t.ry;
  t.zp = t.nbz * kTcTZ + 2 * t.rz;

  // K_{c c'}(dx) per plane (dy, dz) with any non-zero entry
  const int W = 2 * t.rx + 1, C = t.C;
  std::vector<float> Jall((size_t)kTcMaxPlanes * C * C * W, 0.0f);
  auto at = [&](int dy, int dz) { return ((dz + kTcRMax) * (2 * kTcRMax + 1) + dy + kTcRMax); };
  std::vector<char> used(kTcMaxPlanes, 0);
  for (int a = 0; a < nsub; ++a)
    for (const Tap &tp : c->taps[a]) {
      const int pl = at(tp.d[1], tp.d[2]);
      for (int al = 0; al < 3; ++al)
        for (int be = 0; be < 3; ++be) {
          const double J = tp.J[al * 3 + be];
          if (J == 0.0) continue;
          used[pl] = 1;
          const int cc = al * nsub + a, cq = be * nsub + tp.b;
          Jall[(((size_t)pl * C + cc) * C + cq) * W + tp.d[0] + t.rx] += (float)J;
        }
    }
  TcPlan *tp = new (std::nothrow) TcPlan();
  if (!tp) return set_error(SX_ERR_OOM, "host allocation failed");
  memset(tp, 0, sizeof(*tp));
  tp->tf32 = tf32 ? 1 : 0;
  TcArgs &a = tp->base;
  a.t = t;
  a.nx = c->geo.nx;
  a.ny = c->geo.ny;
  a.nz = c->geo.nz;
  a.px = c->geo.px;
  a.py = c->geo.py;
  a.pz = c->geo.pz;
  a.ncell = c->geo.ncell;
  a.os = onsite_cast<float>(c->onsite);
  std::vector<float> Jp;
  for (int dz = -t.rz; dz <= t.rz; ++dz)
    for (int dy = -t.ry; dy <= t.ry; ++dy) {
      const int pl = at(dy, dz);
      if (!used[pl]) continue;
      a.plane_dy[a.nplanes] = dy;
      a.plane_dz[a.nplanes] = dz;
      ++a.nplanes;
      Jp.insert(Jp.end(), Jall.begin() + (size_t)pl * C * C * W, Jall.begin() + (size_t)(pl + 1) * C * C * W);
    }
  if (Jp.empty()) Jp.assign(1, 0.0f);
  const int esz = tf32 ? 4 : 2;
  std::vector<uint32_t> ent = band_entries(t, tf32, a.ept);
  const int ept_max = nsub == 1 ? 16 : nsub == 2 ? 30 : 44;
  if (a.ept > ept_max) {
    delete tp;
    return set_error(SX_ERR_UNSUPPORTED, "the tensor-core band table exceeds its register budget");
  }
  a.win_bytes = (unsigned)(ncopy * t.nch * t.yr * t.zr * 16);
  a.b_bytes = (unsigned)(ncopy * kTcN * t.kb * esz);
  tp->jp_bytes = Jp.size() * 4;
  // Prefer two CTAs per SM (the window load and epilogue of one overlap the MMAs of the other), else
  // the deepest ring that fits one CTA; sx_autotune may pick another of tc_tile_candidates.
  std::vector<TcTiles> cand = tc_tile_candidates_of(*tp);
  if (cand.empty()) {
    delete tp;
    return set_error(SX_ERR_UNSUPPORTED, "the tensor-core tile does not fit in shared memory");
  }
  tc_layout(*tp, cand[0].nbuf, cand[0].ctas);
  const size_t n3 = 3 * (size_t)c->geo.nsite;
  const size_t wunits = (size_t)t.nbx * ncopy * t.nch * t.zp * t.yp;
  cudaError_t e = cudaMalloc(&tp->Wp, wunits * sizeof(uint4));
  if (e == cudaSuccess) e = cudaMalloc(&tp->Jp, Jp.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(tp->Jp, Jp.data(), Jp.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&tp->ent, ent.size() * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemcpy(tp->ent, ent.data(), ent.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&tp->St, n3 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&tp->F0, n3 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&tp->Bf, n3 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&tp->Th, n3 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&tp->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(tp->err, 0, sizeof(int));
  // every layout up to the limit may be launched (sx_autotune switches between them)
  if (e == cudaSuccess) e = set_smem(nsub, tf32, (int)kTcSmemMax);
  tp->nsm = 152;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&tp->nsm, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = tc_set_grid(*tp);
  a.Jp = tp->Jp;
  a.ent = tp->ent;
  a.err = tp->err;
  c->tc = tp;
  if (e != cudaSuccess) {
    tc_free(c);
    return cuda_error(e, "tensor-core plan");
  }
  const int rc = encode_window_map(tp, ncopy);
  if (rc != SX_OK) {
    tc_free(c);
    return rc;
  }
  c->launches_per_step = 6;
  return SX_OK;
}

void tc_free(sx_ctx *c) {
  TcPlan *tp = c->tc;
  if (!tp) return;
  cudaFree(tp->Wp);
  cudaFree(tp->Jp);
  cudaFree(tp->ent);
  cudaFree(tp->St);
  cudaFree(tp->F0);
  cudaFree(tp->Bf);
  cudaFree(tp->Th);
  cudaFree(tp->err);
  delete tp;
  c->tc = nullptr;
}

cudaError_t tc_field(const sx_ctx *c, const double *S, double *b, bool onsite, cudaStream_t st) {
  TcArgs a = c->tc->base;
  a.onsite = onsite ? 1 : 0;
  return field_any<double, double>(*c->tc, a, S, b, st);
}

cudaError_t tc_field_f32(const sx_ctx *c, const double *S, float *b, bool onsite, cudaStream_t st) {
  TcArgs a = c->tc->base;
  a.onsite = onsite ? 1 : 0;
  return field_any<double, float>(*c->tc, a, S, b, st);
}

cudaError_t tc_heun_step(const sx_ctx *c, const double *src, double *dst, const HeunConst &h, uint64_t step,
                         cudaStream_t st) {
  const TcPlan &tp = *c->tc;
  TcArgs a = tp.base;
  a.onsite = 0;  // the Heun stages add the on-site terms
  cudaError_t e = field_any<double, float>(tp, a, src, tp.Bf, st);
  if (e == cudaSuccess) e = bufheun_predict(c, src, tp.Bf, tp.St, tp.F0, tp.Th, h, step, st);
  if (e == cudaSuccess) e = field_any<float, float>(tp, a, tp.St, tp.Bf, st);
  if (e == cudaSuccess) e = bufheun_correct(c, src, tp.St, tp.F0, tp.Bf, tp.Th, dst, h, st);
  return e;
}

// 1 if a bounded wait of the tensor-core kernel gave up since the last check (clears it)
// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against the driver library)
void *tensor_map_encode_fn() {
  static void *fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void *f = nullptr;
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q);
    if (e == cudaSuccess && q == cudaDriverEntryPointSuccess) fn = f;
    else cudaGetLastError();
  }
  return fn;
}

int tc_check_error(const sx_ctx *c) {
  int h = 0;
  if (!c->tc || cudaMemcpy(&h, c->tc->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return 0;
  if (h) cudaMemset(c->tc->err, 0, sizeof(int));
  return h;
}

std::vector<TcTiles> tc_tile_candidates(const sx_ctx *c) { return tc_tile_candidates_of(*c->tc); }

int tc_apply_tiles(sx_ctx *c, const TcTiles &t) {
  TcPlan &tp = *c->tc;
  const TcArgs keep = tp.base;
  const int keep_ctas = tp.ctas;
  if (!tc_layout(tp, t.nbuf, t.ctas)) {
    tp.base = keep;
    tp.ctas = keep_ctas;
    return set_error(SX_ERR_ARG, "tile layout does not fit");
  }
  const cudaError_t e = tc_set_grid(tp);
  if (e != cudaSuccess) {
    tp.base = keep;
    tp.ctas = keep_ctas;
    return cuda_error(e, "tensor-core occupancy");
  }
  return SX_OK;
}

TcTiles tc_current_tiles(const sx_ctx *c) { return {c->tc->base.nbuf, c->tc->ctas}; }

void tc_tiles_info(const sx_ctx *c, int64_t out[8]) {
  const TcArgs &a = c->tc->base;
  out[0] = 0;
  out[1] = a.t.xo;
  out[2] = kTcTY;
  out[3] = kTcTZ;
  out[4] = a.grid;
  out[5] = a.nbuf;
}

}  // namespace sx
