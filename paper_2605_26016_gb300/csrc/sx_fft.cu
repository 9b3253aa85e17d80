// FFT backend: the bilinear and dipolar field in reciprocal space,
//   b^_a^alpha(q) = sum_b sum_beta K^_ab^{alpha beta}(q) S^_b^beta(q)
// ("Backend representations": the FFT backend transforms the spin field,
// multiplies by the precomputed kernel spectrum and transforms back; long-range
// dipolar fields use the same reciprocal-space convolution).
//
// Design:
//  * Own radix-2 FFT: each 1D pass stages W lines of length n in shared memory
//    (bit-reversed placement, then log2 n in-place butterfly stages with a
//    host-built twiddle table), lines grouped so that global accesses are
//    coalesced along x.  Power-of-two axes up to 4096, FP32 or FP64 complex.
//  * The 3*nsub real spin channels are packed two per complex field; the
//    k-space multiply treats q and -q together, which recovers every real
//    channel's spectrum from the packed one and writes the packed spectrum of
//    the real field back.
//  * The kernel matrix M(q) = sum_delta K(delta) e^{+i q.delta} over channels
//    (a, alpha) x (b, beta) is Hermitian (reverse bonds carry the transpose,
//    the dipolar tensor is symmetric), so only its diagonal (real) and upper
//    triangle (complex) are stored.  It is built once per plan in FP64 from the
//    directed taps and, when enabled, the periodic point-dipole sum (minimum
//    image; a separation of exactly half a period split into its two images
//    with weight 1/2).
//  * Heun step: field(S^n) -> predictor -> field(S~) -> corrector, the state sum
//    and renormalisation in FP64 as in the stencil backend.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "sx_device.cuh"
#include "sx_internal.h"
#include "sx_noise.cuh"

namespace sx {

template <typename R>
struct CxT;
template <>
struct CxT<float> {
  using T = float2;
};
template <>
struct CxT<double> {
  using T = double2;
};

struct FftPlan {
  int prec;  // SX_PREC_FP32 or SX_PREC_FP64 (arithmetic of transforms and fields)
  int n[3], logn[3];
  int nsub, nch, noff;
  long long N;   // cells
  long long Nh;  // half-spectrum storage per channel: np ny nz, np = nx/2 + 1 rounded up to a multiple of 16
  void *Z;       // [nch][Nh] complex: half spectra of the channels
  void *Md;      // [nch][Nh] real: diagonal of M(q)
  void *Mo;      // [noff][Nh] complex: upper triangle of M(q)
  void *tw[3];   // per axis: n/2 complex twiddles exp(-2 pi i k / n) (full-length transforms)
  void *twm;     // nx/4 twiddles of the nx/2-point transform of the x pass
  void *twr;     // nx/2 + 1 split factors exp(-2 pi i q / nx) of the real-to-complex x pass
  void *St, *F0;  // Heun: predictor state and f0, [nch][N] real each
  void *Th;       // Heun: thermal field of the step, [nch][N] real
  int wx, wy, wz, wc;  // lines per CTA of the x (r2c), y, z (with the kernel multiply) and x (c2r) passes
};

namespace {

constexpr int kFftThreads = 512;   // the full-length complex passes of the plan-time kernel transform
constexpr int kHalfThreads = 256;  // the half-spectrum passes of every field evaluation
constexpr size_t kHalfBudget = 56 * 1024;  // shared memory per CTA of the half-spectrum passes (four CTAs per SM)
constexpr size_t kFftSmem = 200 * 1024;

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

// Shared-memory slot of element i of a staged line: one padding slot after every
// eight elements, so that the strided element patterns of the early fused stages
// and the bit-reversed staging spread over the banks.  The line pitch
// fft_pitch(n) is odd, so equal elements of adjacent lines fall in different banks.
__host__ __device__ __forceinline__ int fft_slot(int i) { return i + (i >> 3); }
__host__ __device__ __forceinline__ int fft_pitch(int n) { return n + (n >> 3) + 1; }

// a <- a + w b, b <- a - w b
template <typename C>
__device__ __forceinline__ void bfly(C &a, C &b, const C &w) {
  const C t = cmul(b, w);
  b.x = a.x - t.x;
  b.y = a.y - t.y;
  a.x += t.x;
  a.y += t.y;
}

// w times -i (forward) or +i (inverse)
template <typename C>
__device__ __forceinline__ C rot_quarter(C w, int inverse) {
  C r;
  if (inverse) {
    r.x = -w.y;
    r.y = w.x;
  } else {
    r.x = w.y;
    r.y = -w.x;
  }
  return r;
}

// w times exp(-i pi/4) (forward) or exp(+i pi/4) (inverse)
template <typename C, typename R>
__device__ __forceinline__ C rot_eighth(C w, int inverse) {
  const R h = (R)0.70710678118654752440;
  C r;
  if (inverse) {
    r.x = h * (w.x - w.y);
    r.y = h * (w.x + w.y);
  } else {
    r.x = h * (w.x + w.y);
    r.y = h * (w.y - w.x);
  }
  return r;
}

// LR consecutive radix-2 decimation-in-time stages s .. s + LR - 1 in registers.  Stage s
// pairs elements h = 2^s apart with twiddle w_{2h}^k; the 2^LR elements i0 + m h
// (i0 = block * 2^LR h + k) only meet each other in these stages, so one thread
// takes them through all LR stages and writes them back in place: stage s+1 uses
// w_{4h}^{k + (m&1) h} = w_{4h}^k (-i)^(m&1), stage s+2 w_{8h}^{k + m h} = w_{8h}^k w_8^m.
template <typename R, int LR>
__device__ __forceinline__ void dit_stages(typename CxT<R>::T *sm, int pitch, int W, int logn, int s,
                                           const typename CxT<R>::T *__restrict__ tw, int inverse) {
  using C = typename CxT<R>::T;
  constexpr int RAD = 1 << LR;
  const int h = 1 << s;
  const int logng = logn - LR;
  const int total = W << logng;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int w = t >> logng, j = t & ((1 << logng) - 1);
    const int k = j & (h - 1);
    C *line = sm + w * pitch;
    const int i0 = ((j >> s) << (s + LR)) + k;
    C v[RAD];
#pragma unroll
    for (int m = 0; m < RAD; ++m) v[m] = line[fft_slot(i0 + m * h)];
    C t1 = tw[k << (logn - 1 - s)];
    if (inverse) t1.y = -t1.y;
#pragma unroll
    for (int m = 0; m < RAD; m += 2) bfly(v[m], v[m + 1], t1);
    if constexpr (LR >= 2) {
      C t2 = tw[k << (logn - 2 - s)];
      if (inverse) t2.y = -t2.y;
      const C t2b = rot_quarter(t2, inverse);
#pragma unroll
      for (int m = 0; m < RAD; m += 4) {
        bfly(v[m], v[m + 2], t2);
        bfly(v[m + 1], v[m + 3], t2b);
      }
    }
    if constexpr (LR >= 3) {
      C t3 = tw[k << (logn - 3 - s)];
      if (inverse) t3.y = -t3.y;
      const C t31 = rot_eighth<C, R>(t3, inverse);
      const C t32 = rot_quarter(t3, inverse);
      const C t33 = rot_eighth<C, R>(t32, inverse);
      bfly(v[0], v[4], t3);
      bfly(v[1], v[5], t31);
      bfly(v[2], v[6], t32);
      bfly(v[3], v[7], t33);
    }
#pragma unroll
    for (int m = 0; m < RAD; ++m) line[fft_slot(i0 + m * h)] = v[m];
  }
}

// One 1D pass over every line of one axis.  Line group g (W lines, adjacent
// along the grouping axis, stride gs), outer line index o (stride os), element
// i along the transform axis (stride is); blockIdx.z selects the field.  The
// lines are staged bit-reversed in shared memory and transformed in place by
// radix-2 DIT stages taken three (then two, then one) at a time in registers.
template <typename R>
__global__ void __launch_bounds__(kFftThreads)
    k_fft_pass(typename CxT<R>::T *__restrict__ data, int n, int logn, int W, int ifast, long long gs, long long os,
               long long is, long long fstride, const typename CxT<R>::T *__restrict__ tw, int inverse) {
  using C = typename CxT<R>::T;
  extern __shared__ __align__(16) unsigned char smraw[];
  C *sm = reinterpret_cast<C *>(smraw);
  const int pitch = fft_pitch(n);
  C *base = data + blockIdx.z * fstride + (long long)blockIdx.x * W * gs + (long long)blockIdx.y * os;
  const int total = W * n;
  const int logw = 31 - __clz(W);  // W and n are powers of two
  for (int e = threadIdx.x; e < total; e += kFftThreads) {
    int w, i;
    if (ifast) {
      w = e >> logn;
      i = e & (n - 1);
    } else {
      i = e >> logw;
      w = e & (W - 1);
    }
    const int r = (int)(__brev((unsigned)i) >> (32 - logn));
    sm[w * pitch + fft_slot(r)] = base[w * gs + i * is];
  }
  __syncthreads();
  for (int s = 0; s < logn;) {
    const int rem = logn - s;
    if (rem >= 3) {
      dit_stages<R, 3>(sm, pitch, W, logn, s, tw, inverse);
      s += 3;
    } else if (rem == 2) {
      dit_stages<R, 2>(sm, pitch, W, logn, s, tw, inverse);
      s += 2;
    } else {
      dit_stages<R, 1>(sm, pitch, W, logn, s, tw, inverse);
      s += 1;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < total; e += kFftThreads) {
    int w, i;
    if (ifast) {
      w = e >> logn;
      i = e & (n - 1);
    } else {
      i = e >> logw;
      w = e & (W - 1);
    }
    base[w * gs + i * is] = sm[w * pitch + fft_slot(i)];
  }
}

// ---------------------------------------------------------------- real-to-complex pipeline
//
// The spin channels and fields are real, so only the half spectrum qx = 0 .. nx/2 (nh = nx/2 + 1
// values) is kept, one complex spectrum per real channel k = c * nsub + a:
//   Zh[k * Nh + zrow(qz, qy) * np + qx],  Nh = np * ny * nz,
// with the row pitch np = nh rounded up to a multiple of 16, so that every row starts on a 128-byte
// boundary and the y and z passes read whole 32-byte sectors (the padding columns are never read back).
// The rows are blocked along z: zrow(qz, qy) = ((qz / ZB) ny + qy) ZB + qz mod ZB with ZB = min(16, nz),
// i.e. the ZB rows of one qy within a block of ZB planes are adjacent.  A z line then spans nz / ZB
// separate regions of memory instead of nz rows one plane (ny np values) apart; at 1024^3 those
// 1024 rows 4.3 MB apart read at 1.6 TB/s against 2.9 TB/s blocked by 16, through the translation
// of that many pages.
// One field evaluation is five passes over it:
//   k_xr2c   x lines of every channel, real to complex: the nx/2-point complex transform of the
//            (even, odd) sample pairs, then its split into the half spectrum;
//   k_hpass  y lines, forward;
//   k_zkz    z lines: forward transform, b^(q) = M(q) s^(q) over the channels, inverse transform,
//            all in shared memory;
//   k_hpass  y lines, inverse;
//   k_xc2r   x lines of every channel, complex to real (times 1/N), followed on the cells of those
//            lines by the field output, the Heun predictor or the Heun corrector.

struct FftGeo {
  int nx, ny, nz, nh, np, m, logm, logx;
  int lzb;  // log2 of the z block ZB
  long long N, Nh;
};

// row of (qz, qy) in a channel's half spectrum (see above)
__host__ __device__ __forceinline__ long long zrow(const FftGeo &g, int qz, int qy) {
  return ((((long long)(qz >> g.lzb) * g.ny + qy)) << g.lzb) + (qz & ((1 << g.lzb) - 1));
}
// offset, in rows, of plane qz along a z line (the line of qy = 0)
__host__ __device__ __forceinline__ long long zline_row(const FftGeo &g, int qz) {
  return (((long long)(qz >> g.lzb) * g.ny) << g.lzb) + (qz & ((1 << g.lzb) - 1));
}

__device__ __forceinline__ int brev_n(int i, int logn) {
  return logn ? (int)(__brev((unsigned)i) >> (32 - logn)) : 0;
}

// asynchronous global -> shared copy of one complex value (8 or 16 bytes), so that a CTA's whole staging
// load is in flight at once
template <typename C>
__device__ __forceinline__ void cp_async_c(C *smem_dst, const C *gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  if constexpr (sizeof(C) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// every radix-2 DIT stage of nlines staged lines of length 2^logn (bit-reversed input, natural output)
template <typename R>
__device__ __forceinline__ void fft_stages(typename CxT<R>::T *sm, int pitch, int nlines, int logn,
                                           const typename CxT<R>::T *__restrict__ tw, int inverse) {
  for (int s = 0; s < logn;) {
    const int rem = logn - s;
    if (rem >= 3) {
      dit_stages<R, 3>(sm, pitch, nlines, logn, s, tw, inverse);
      s += 3;
    } else if (rem == 2) {
      dit_stages<R, 2>(sm, pitch, nlines, logn, s, tw, inverse);
      s += 2;
    } else {
      dit_stages<R, 1>(sm, pitch, nlines, logn, s, tw, inverse);
      s += 1;
    }
    __syncthreads();
  }
}

// x lines y0 .. y0 + W - 1 of plane z, every channel: real samples src[k][cell] -> half spectrum.
// z_j = x_2j + i x_2j+1 (j < m = nx/2), Z = FFT_m(z); X_q = E_q + w^q O_q for q = 0 .. m with
// E_q = (Z_q + conj Z_{m-q}) / 2, O_q = (Z_q - conj Z_{m-q}) / (2i), w = exp(-2 pi i / nx), Z_m = Z_0.
template <typename R, typename Tin>
__device__ __forceinline__ void r2c_lines(const Tin *__restrict__ src, typename CxT<R>::T *Zh, const FftGeo &g,
                                          int nch, int W, int y0, int z, typename CxT<R>::T *sm,
                                          const typename CxT<R>::T *__restrict__ twm,
                                          const typename CxT<R>::T *__restrict__ twr) {
  using C = typename CxT<R>::T;
  const int m = g.m, logm = g.logm, pitch = fft_pitch(m);
  const int nw = min(W, g.ny - y0);
  for (int k = 0; k < nch; ++k) {
    const Tin *in = src + (long long)k * g.N + ((long long)z * g.ny + y0) * g.nx;
    // four sample pairs per thread and round, loaded before any is converted
    constexpr int U = 4;
    for (int e0 = threadIdx.x; e0 < nw * m; e0 += U * kHalfThreads) {
      Tin a[U], b[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * kHalfThreads;
        if (e < nw * m) {
          const Tin *pq = in + (long long)(e >> logm) * g.nx + 2 * (e & (m - 1));
          a[u] = pq[0];
          b[u] = pq[1];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * kHalfThreads;
        if (e < nw * m) {
          C v;
          v.x = cvt<R>(a[u]);
          v.y = cvt<R>(b[u]);
          sm[(e >> logm) * pitch + fft_slot(brev_n(e & (m - 1), logm))] = v;
        }
      }
    }
    __syncthreads();
    fft_stages<R>(sm, pitch, nw, logm, twm, 0);
    C *dst = Zh + (long long)k * g.Nh + zrow(g, z, y0) * g.np;  // row of y0 + w: w ZB rows further
    for (int e = threadIdx.x; e < nw * (m + 1); e += kHalfThreads) {
      // e = w (m + 1) + q, 0 <= q <= m, without a division: e >> logm overshoots w by (w + q) >> logm
      int w = e >> logm;
      int q = e - w * (m + 1);
      while (q < 0) {
        --w;
        q += m + 1;
      }
      const C a = sm[w * pitch + fft_slot(q & (m - 1))];
      const C b = sm[w * pitch + fft_slot((m - q) & (m - 1))];
      const R ex = (R)0.5 * (a.x + b.x), ey = (R)0.5 * (a.y - b.y);
      const R ox = (R)0.5 * (a.y + b.y), oy = (R)-0.5 * (a.x - b.x);
      const C t = twr[q];
      C X;
      X.x = ex + (t.x * ox - t.y * oy);
      X.y = ey + (t.x * oy + t.y * ox);
      dst[((long long)w << g.lzb) * g.np + q] = X;
    }
    __syncthreads();
  }
}

template <typename R, typename Tin>
__global__ void __launch_bounds__(kHalfThreads)
    k_xr2c(const Tin *__restrict__ src, typename CxT<R>::T *__restrict__ Zh, FftGeo g, int nch, int W,
           const typename CxT<R>::T *__restrict__ twm, const typename CxT<R>::T *__restrict__ twr) {
  using C = typename CxT<R>::T;
  extern __shared__ __align__(16) unsigned char smraw[];
  r2c_lines<R, Tin>(src, Zh, g, nch, W, blockIdx.x * W, blockIdx.y, reinterpret_cast<C *>(smraw), twm, twr);
}

// One pass of complex transforms along y on the half spectrum: lines of length 2^logn (element stride
// is = ZB np), W lines adjacent along the contiguous qx axis (ngroup = nh lines in all, the last group
// partial), plane qz = blockIdx.y (row zline_row(qz)), channel blockIdx.z (stride fs).
template <typename R>
__global__ void __launch_bounds__(kHalfThreads)
    k_hpass(typename CxT<R>::T *__restrict__ data, FftGeo g, int logn, int W, int ngroup, long long is,
            long long fs, const typename CxT<R>::T *__restrict__ tw, int inverse) {
  using C = typename CxT<R>::T;
  extern __shared__ __align__(16) unsigned char smraw[];
  C *sm = reinterpret_cast<C *>(smraw);
  const int n = 1 << logn, pitch = fft_pitch(n);
  const int g0 = blockIdx.x * W, nw = min(W, ngroup - g0);
  const int logw = 31 - __clz(W);  // W is a power of two; lines w >= nw of the last group are skipped
  C *base = data + blockIdx.z * fs + g0 + zline_row(g, blockIdx.y) * g.np;
  for (int e = threadIdx.x; e < (n << logw); e += kHalfThreads) {
    const int i = e >> logw, w = e & (W - 1);
    if (w < nw) cp_async_c(&sm[w * pitch + fft_slot(brev_n(i, logn))], &base[w + i * is]);
  }
  cp_async_wait_all();
  __syncthreads();
  fft_stages<R>(sm, pitch, nw, logn, tw, inverse);
  for (int e = threadIdx.x; e < (n << logw); e += kHalfThreads) {
    const int i = e >> logw, w = e & (W - 1);
    if (w < nw) base[w + i * is] = sm[w * pitch + fft_slot(i)];
  }
}

// b = M(q) s at one wave vector (half-spectrum index q): diagonal Md, upper triangle Mo (Hermitian)
template <typename R, int NCH>
__device__ __forceinline__ void kmul_point(const R *__restrict__ Md, const typename CxT<R>::T *__restrict__ Mo,
                                           long long Nh, long long q, const typename CxT<R>::T (&s)[NCH],
                                           typename CxT<R>::T (&b)[NCH]) {
  using C = typename CxT<R>::T;
#pragma unroll
  for (int k = 0; k < NCH; ++k) {
    const R d = Md[k * Nh + q];
    C acc;
    acc.x = d * s[k].x;
    acc.y = d * s[k].y;
#pragma unroll
    for (int l = 0; l < NCH; ++l) {
      if (l == k) continue;
      const int lo = k < l ? k : l, hi = k < l ? l : k;
      const int p = lo * NCH - lo * (lo + 1) / 2 + (hi - lo - 1);
      C mkl = Mo[p * Nh + q];
      if (k > l) mkl.y = -mkl.y;
      const C t = cmul(mkl, s[l]);
      acc.x += t.x;
      acc.y += t.y;
    }
    b[k] = acc;
  }
}

// z lines of qx0 .. qx0 + W - 1 at qy = blockIdx.y, every channel: forward transform, kernel multiply,
// inverse transform.  After the forward DIT the spectrum is in natural order; the multiply writes each
// result to the bit-reversed position of its wave vector (pairs i <-> brev(i) are handled by one
// thread), which is the input order of the inverse DIT.
template <typename R, int NCH>
__global__ void __launch_bounds__(kHalfThreads)
    k_zkz(typename CxT<R>::T *__restrict__ Zh, const R *__restrict__ Md, const typename CxT<R>::T *__restrict__ Mo,
          FftGeo g, int logz, int W, const typename CxT<R>::T *__restrict__ tw) {
  using C = typename CxT<R>::T;
  extern __shared__ __align__(16) unsigned char smraw[];
  C *sm = reinterpret_cast<C *>(smraw);
  const int n = 1 << logz, pitch = fft_pitch(n);
  const int qx0 = blockIdx.x * W, qy = blockIdx.y, nw = min(W, g.nh - qx0);
  C *base = Zh + zrow(g, 0, qy) * g.np + qx0;  // plane i of the line: zline_row(i) rows further
  const int logw = 31 - __clz(W);  // W is a power of two; lines w >= nw of the last group are skipped
  for (int e = threadIdx.x; e < (NCH << (logw + logz)); e += kHalfThreads) {
    const int k = e >> (logw + logz), i = (e >> logw) & (n - 1), w = e & (W - 1);
    if (w < nw)
      cp_async_c(&sm[(k * W + w) * pitch + fft_slot(brev_n(i, logz))], &base[k * g.Nh + zline_row(g, i) * g.np + w]);
  }
  cp_async_wait_all();
  __syncthreads();
  fft_stages<R>(sm, pitch, NCH * W, logz, tw, 0);
  for (int e = threadIdx.x; e < (n << logw); e += kHalfThreads) {
    const int i = e >> logw, w = e & (W - 1), r = brev_n(i, logz);
    if (w >= nw || r < i) continue;
    C si[NCH], bi[NCH];
#pragma unroll
    for (int k = 0; k < NCH; ++k) si[k] = sm[(k * W + w) * pitch + fft_slot(i)];
    const long long q0 = zrow(g, 0, qy) * g.np + qx0 + w;
    kmul_point<R, NCH>(Md, Mo, g.Nh, q0 + zline_row(g, i) * g.np, si, bi);
    if (r == i) {
#pragma unroll
      for (int k = 0; k < NCH; ++k) sm[(k * W + w) * pitch + fft_slot(i)] = bi[k];
    } else {
      C sr[NCH], br[NCH];
#pragma unroll
      for (int k = 0; k < NCH; ++k) sr[k] = sm[(k * W + w) * pitch + fft_slot(r)];
      kmul_point<R, NCH>(Md, Mo, g.Nh, q0 + zline_row(g, r) * g.np, sr, br);
#pragma unroll
      for (int k = 0; k < NCH; ++k) {
        sm[(k * W + w) * pitch + fft_slot(r)] = bi[k];
        sm[(k * W + w) * pitch + fft_slot(i)] = br[k];
      }
    }
  }
  __syncthreads();
  fft_stages<R>(sm, pitch, NCH * W, logz, tw, 1);
  for (int e = threadIdx.x; e < (NCH << (logw + logz)); e += kHalfThreads) {
    const int k = e >> (logw + logz), i = (e >> logw) & (n - 1), w = e & (W - 1);
    if (w < nw) base[k * g.Nh + zline_row(g, i) * g.np + w] = sm[(k * W + w) * pitch + fft_slot(i)];
  }
}

enum XEpilogue { XE_FIELD = 0, XE_PRED = 1, XE_CORR = 2 };

// Arguments of the complex-to-real x pass and its epilogue
template <typename R, typename Tout>
struct XArgs {
  const double *S;  // FIELD: spins of the on-site terms (may be the predictor state, then Sr); PRED, CORR: S^n
  const R *Sr;      // FIELD: spins in R instead of S when set; CORR: S~
  Tout *out;        // FIELD: the field
  R *St, *F0, *Th;  // PRED: written; CORR: F0, Th read
  double *Snew;     // CORR: S^{n+1}
  int *status;
  OnSiteT<R> os;
  HeunT<R> h;
  unsigned long long step;
  int onsite;
};

template <typename R>
__device__ __forceinline__ void onsite_r(const OnSiteT<R> &os, int a, const R s[3], R b[3]) {
  const R p = os.twoK[a] * (s[0] * os.axis[a][0] + s[1] * os.axis[a][1] + s[2] * os.axis[a][2]);
#pragma unroll
  for (int c = 0; c < 3; ++c) b[c] += os.zee[a][c] + p * os.axis[a][c];
}

__device__ __forceinline__ void unit_r(float x[3]) {
  const float n2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  float r = rsqrtf(n2);
  r = r * fmaf(-0.5f * n2, r * r, 1.5f);
  x[0] *= r;
  x[1] *= r;
  x[2] *= r;
}
__device__ __forceinline__ void unit_r(double x[3]) {
  const double r = rsqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  x[0] *= r;
  x[1] *= r;
  x[2] *= r;
}
__device__ __forceinline__ bool correct_r(const double S[3], const float d[3], double o[3]) {
  return renormalise64(S, d, o);
}
__device__ __forceinline__ bool correct_r(const double S[3], const double d[3], double o[3]) {
  o[0] = S[0] + d[0];
  o[1] = S[1] + d[1];
  o[2] = S[2] + d[2];
  return unit64_checked(o);
}

// x lines y0 .. y0 + W - 1 of plane z, every channel: half spectrum -> real samples times 1/N, then the
// epilogue on those cells.  Inverse of k_xr2c: Z'_q = E'_q + i O'_q (q < m) with E'_q = X_q + conj X_{m-q},
// O'_q = (X_q - conj X_{m-q}) conj(w^q); the unnormalised inverse m-point transform of Z' holds
// (x_2j, x_2j+1) times N of the 3D transform.
template <typename R, int MODE, typename Tout, int NSUB>
__global__ void __launch_bounds__(kHalfThreads)
    k_xc2r(typename CxT<R>::T *Zh, FftGeo g, int W, const typename CxT<R>::T *__restrict__ twm,
           const typename CxT<R>::T *__restrict__ twr, XArgs<R, Tout> xa) {
  using C = typename CxT<R>::T;
  extern __shared__ __align__(16) unsigned char smraw[];
  C *sm = reinterpret_cast<C *>(smraw);
  constexpr int nsub = NSUB, nch = 3 * NSUB;
  const int m = g.m, logm = g.logm, pitch = fft_pitch(m);
  const int y0 = blockIdx.x * W, z = blockIdx.y;
  const int nw = min(W, g.ny - y0);
  const int logw = 31 - __clz(W);  // W is a power of two; lines w >= nw of the last group are skipped
  // four elements per thread and round: their eight loads are issued before any is used
  constexpr int U = 4;
  const int total = nch << (logw + logm);
  for (int e0 = threadIdx.x; e0 < total; e0 += U * kHalfThreads) {
    C xs[U], ys[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * kHalfThreads;
      const int k = e >> (logw + logm), w = (e >> logm) & (W - 1), q = e & (m - 1);
      if (e < total && w < nw) {
        const C *row = Zh + (long long)k * g.Nh + zrow(g, z, y0 + w) * g.np;
        xs[u] = row[q];
        ys[u] = row[m - q];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * kHalfThreads;
      const int k = e >> (logw + logm), w = (e >> logm) & (W - 1), q = e & (m - 1);
      if (e < total && w < nw) {
        const C x = xs[u], y = ys[u];
        const R ex = x.x + y.x, ey = x.y - y.y, dx = x.x - y.x, dy = x.y + y.y;
        const C t = twr[q];
        const R ox = dx * t.x + dy * t.y, oy = dy * t.x - dx * t.y;  // (d) conj(t)
        C v;
        v.x = ex - oy;
        v.y = ey + ox;
        sm[(k * W + w) * pitch + fft_slot(brev_n(q, logm))] = v;
      }
    }
  }
  __syncthreads();
  fft_stages<R>(sm, pitch, nch * W, logm, twm, 1);
  const R scale = (R)(1.0 / (double)g.N);
  for (int e = threadIdx.x; e < nw * g.nx; e += kHalfThreads) {
    const int w = e >> g.logx, x = e & (g.nx - 1);
    const long long cell = ((long long)z * g.ny + y0 + w) * g.nx + x;
    R v[nch];
#pragma unroll
    for (int k = 0; k < nch; ++k) {
      const C c = sm[(k * W + w) * pitch + fft_slot(x >> 1)];
      v[k] = ((x & 1) ? c.y : c.x) * scale;
    }
#pragma unroll
    for (int a = 0; a < nsub; ++a) {
      R b[3] = {v[a], v[nsub + a], v[2 * nsub + a]};
      const long long i0 = (long long)a * g.N + cell;  // channel c of sublattice a at (c nsub + a) N + cell
      if constexpr (MODE == XE_FIELD) {
        if (xa.onsite) {
          R s[3];
          for (int c = 0; c < 3; ++c)
            s[c] = xa.Sr ? xa.Sr[(long long)c * nsub * g.N + i0] : cvt<R>(xa.S[(long long)c * nsub * g.N + i0]);
          onsite_r<R>(xa.os, a, s, b);
        }
        for (int c = 0; c < 3; ++c) xa.out[(long long)c * nsub * g.N + i0] = cvt<Tout>(b[c]);
      } else if constexpr (MODE == XE_PRED) {
        R s[3], th[3] = {(R)0, (R)0, (R)0}, f[3];
        for (int c = 0; c < 3; ++c) s[c] = cvt<R>(xa.S[(long long)c * nsub * g.N + i0]);
        onsite_r<R>(xa.os, a, s, b);
        if (xa.h.thermal) {
          float e0, e1, e2;
          normals3(xa.h.seed, xa.h.replica, (uint64_t)i0, xa.step, e0, e1, e2);
          const R sg = xa.h.sigma[a];
          th[0] = sg * cvt<R>(e0);
          th[1] = sg * cvt<R>(e1);
          th[2] = sg * cvt<R>(e2);
          for (int c = 0; c < 3; ++c) xa.Th[(long long)c * nsub * g.N + i0] = th[c];
        }
        const R im = xa.os.inv_mm[a];
        const R B[3] = {b[0] * im + th[0], b[1] * im + th[1], b[2] * im + th[2]};
        llg_rhs_t<R>(s, B, xa.h.g, xa.h.alpha, f);
        R xs[3] = {s[0] + xa.h.dt * f[0], s[1] + xa.h.dt * f[1], s[2] + xa.h.dt * f[2]};
        unit_r(xs);
        for (int c = 0; c < 3; ++c) {
          xa.St[(long long)c * nsub * g.N + i0] = xs[c];
          xa.F0[(long long)c * nsub * g.N + i0] = f[c];
        }
      } else {
        R s[3], th[3] = {(R)0, (R)0, (R)0}, f[3], d[3];
        double s64[3], o[3];
        for (int c = 0; c < 3; ++c) {
          s[c] = xa.Sr[(long long)c * nsub * g.N + i0];
          s64[c] = xa.S[(long long)c * nsub * g.N + i0];
          if (xa.h.thermal) th[c] = xa.Th[(long long)c * nsub * g.N + i0];
        }
        onsite_r<R>(xa.os, a, s, b);
        const R im = xa.os.inv_mm[a];
        const R B[3] = {b[0] * im + th[0], b[1] * im + th[1], b[2] * im + th[2]};
        llg_rhs_t<R>(s, B, xa.h.g, xa.h.alpha, f);
        for (int c = 0; c < 3; ++c) d[c] = xa.h.hdt * (xa.F0[(long long)c * nsub * g.N + i0] + f[c]);
        report_numeric(xa.status, correct_r(s64, d, o));
        for (int c = 0; c < 3; ++c) xa.Snew[(long long)c * nsub * g.N + i0] = o[c];
      }
    }
  }
  if constexpr (MODE == XE_PRED) {
    // the forward transform of S~ along these x lines, for the corrector's field: S~ was just written by
    // this CTA (visible to it after the barrier, L2-resident), and the spectrum rows are this CTA's own
    __syncthreads();
    r2c_lines<R, R>(xa.St, Zh, g, nch, W, y0, z, sm, twm, twr);
  }
}

// kernel spectrum of the half spectrum (z-blocked rows) from the full FP64 spectrum Zb ([qz][qy][qx])
__device__ __forceinline__ long long full_row_of(const FftGeo &g, long long srow) {
  const long long zb = srow / ((long long)g.ny << g.lzb), r = srow - zb * ((long long)g.ny << g.lzb);
  const long long qy = r >> g.lzb, qz = (zb << g.lzb) + (r & ((1 << g.lzb) - 1));
  return qz * g.ny + qy;
}
template <typename R>
__global__ void k_store_diag_h(const double2 *__restrict__ Zb, R *__restrict__ Md, FftGeo g) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.Nh) return;
  const long long srow = i / g.np, qx = i - srow * g.np, row = full_row_of(g, srow);
  Md[i] = qx < g.nh ? (R)Zb[row * g.nx + qx].x : (R)0;
}
template <typename R>
__global__ void k_store_off_h(const double2 *__restrict__ Zb, typename CxT<R>::T *__restrict__ Mo, FftGeo g) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.Nh) return;
  const long long srow = i / g.np, qx = i - srow * g.np, row = full_row_of(g, srow);
  typename CxT<R>::T v;
  v.x = qx < g.nh ? (R)Zb[row * g.nx + qx].x : (R)0;
  v.y = qx < g.nh ? (R)Zb[row * g.nx + qx].y : (R)0;
  Mo[i] = v;
}

// ---------------------------------------------------------------- Heun

template <typename R>
__device__ __forceinline__ void onsite_t(const OnSiteT<R> &os, int a, const R s[3], R b[3]) {
  const R p = os.twoK[a] * (s[0] * os.axis[a][0] + s[1] * os.axis[a][1] + s[2] * os.axis[a][2]);
#pragma unroll
  for (int c = 0; c < 3; ++c) b[c] += os.zee[a][c] + p * os.axis[a][c];
}

__device__ __forceinline__ void unit_t(float x[3]) {
  const float n2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  float r = rsqrtf(n2);
  r = r * fmaf(-0.5f * n2, r * r, 1.5f);
  x[0] *= r;
  x[1] *= r;
  x[2] *= r;
}
__device__ __forceinline__ void unit_t(double x[3]) {
  const double r = rsqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  x[0] *= r;
  x[1] *= r;
  x[2] *= r;
}

template <typename R>
__device__ __forceinline__ void thermal_t(const HeunT<R> &h, int a, long long site, uint64_t step, R th[3]) {
  th[0] = th[1] = th[2] = (R)0;
  if (h.thermal) {
    float e0, e1, e2;
    normals3(h.seed, h.replica, (uint64_t)site, step, e0, e1, e2);
    const R sg = h.sigma[a];
    th[0] = sg * cvt<R>(e0);
    th[1] = sg * cvt<R>(e1);
    th[2] = sg * cvt<R>(e2);
  }
}

// predictor from the bilinear+dipolar field Bf of S (on-site terms added here)
// (a thermal step also stores the thermal field sigma eta in Th for the corrector)
template <typename R>
__global__ void k_fft_predict(const double *__restrict__ S, const R *__restrict__ Bf, R *__restrict__ St,
                              R *__restrict__ F0, R *__restrict__ Th, int nsub, long long N, OnSiteT<R> os,
                              HeunT<R> h, uint64_t step) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int a = 0; a < nsub; ++a) {
    R s[3], b[3], th[3], f[3];
    for (int c = 0; c < 3; ++c) {
      s[c] = cvt<R>(S[(long long)(c * nsub + a) * N + i]);
      b[c] = Bf[(long long)(c * nsub + a) * N + i];
    }
    onsite_t<R>(os, a, s, b);
    thermal_t<R>(h, a, (long long)a * N + i, step, th);
    if (h.thermal)
      for (int c = 0; c < 3; ++c) Th[(long long)(c * nsub + a) * N + i] = th[c];
    const R im = os.inv_mm[a];
    const R B[3] = {b[0] * im + th[0], b[1] * im + th[1], b[2] * im + th[2]};
    llg_rhs_t<R>(s, B, h.g, h.alpha, f);
    R x[3] = {s[0] + h.dt * f[0], s[1] + h.dt * f[1], s[2] + h.dt * f[2]};
    unit_t(x);
    for (int c = 0; c < 3; ++c) {
      St[(long long)(c * nsub + a) * N + i] = x[c];
      F0[(long long)(c * nsub + a) * N + i] = f[c];
    }
  }
}

__device__ __forceinline__ bool correct_state(const double S[3], const float d[3], double o[3]) {
  return renormalise64(S, d, o);
}
__device__ __forceinline__ bool correct_state(const double S[3], const double d[3], double o[3]) {
  o[0] = S[0] + d[0];
  o[1] = S[1] + d[1];
  o[2] = S[2] + d[2];
  return unit64_checked(o);
}

template <typename R>
__global__ void k_fft_correct(const double *__restrict__ S, const R *__restrict__ St, const R *__restrict__ F0,
                              const R *__restrict__ Bf, const R *__restrict__ Th, double *__restrict__ Snew, int nsub,
                              long long N, OnSiteT<R> os, HeunT<R> h, int *__restrict__ status) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int a = 0; a < nsub; ++a) {
    R s[3], b[3], th[3], f[3], d[3];
    double s64[3], o[3];
    for (int c = 0; c < 3; ++c) {
      const long long k = (long long)(c * nsub + a) * N + i;
      s[c] = St[k];
      b[c] = Bf[k];
      s64[c] = S[k];
    }
    onsite_t<R>(os, a, s, b);
    for (int c = 0; c < 3; ++c) th[c] = h.thermal ? Th[(long long)(c * nsub + a) * N + i] : (R)0;
    const R im = os.inv_mm[a];
    const R B[3] = {b[0] * im + th[0], b[1] * im + th[1], b[2] * im + th[2]};
    llg_rhs_t<R>(s, B, h.g, h.alpha, f);
    const R hdt = h.hdt;
    for (int c = 0; c < 3; ++c) d[c] = hdt * (F0[(long long)(c * nsub + a) * N + i] + f[c]);
    report_numeric(status, correct_state(s64, d, o));
    for (int c = 0; c < 3; ++c) Snew[(long long)(c * nsub + a) * N + i] = o[c];
  }
}

// ---------------------------------------------------------------- kernel spectrum (plan time, FP64)

struct DipArgs {
  int nx, ny, nz, nsub;
  double A[3][3];
  double pos[SX_MAX_SUB][3];
  double mu[SX_MAX_SUB];
  double pref, tol;
  int dipolar;
};

// real-space kernel component K_{(a,alpha),(b,beta)}(delta) for every cell delta (imag = 0):
// the periodic point-dipole sum; exchange taps are added afterwards
__global__ void k_fill_dipolar(double2 *__restrict__ Zb, DipArgs d, int a, int al, int b, int be) {
  const long long N = (long long)d.nx * d.ny * d.nz;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N) return;
  double val = 0.0;
  if (d.dipolar) {
    const int cx = (int)(idx % d.nx), cy = (int)((idx / d.nx) % d.ny), cz = (int)(idx / ((long long)d.nx * d.ny));
    const int c[3] = {cx, cy, cz};
    const int L[3] = {d.nx, d.ny, d.nz};
    double img[3][2], wgt[3][2];
    int nim[3];
    for (int k = 0; k < 3; ++k) {
      const double f = c[k] + d.pos[b][k] - d.pos[a][k];
      const double t = f - L[k] * floor(f / L[k] + 0.5);
      if (fabs(fabs(t) - 0.5 * L[k]) < 1e-12) {
        nim[k] = 2;
        img[k][0] = -0.5 * L[k];
        img[k][1] = 0.5 * L[k];
        wgt[k][0] = wgt[k][1] = 0.5;
      } else {
        nim[k] = 1;
        img[k][0] = t;
        wgt[k][0] = 1.0;
      }
    }
    for (int ix = 0; ix < nim[0]; ++ix)
      for (int iy = 0; iy < nim[1]; ++iy)
        for (int iz = 0; iz < nim[2]; ++iz) {
          const double f[3] = {img[0][ix], img[1][iy], img[2][iz]};
          double r[3];
          for (int k = 0; k < 3; ++k) r[k] = f[0] * d.A[0][k] + f[1] * d.A[1][k] + f[2] * d.A[2][k];
          const double len = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
          if (len <= d.tol) continue;
          const double e_al = r[al] / len, e_be = r[be] / len;
          const double w = wgt[0][ix] * wgt[1][iy] * wgt[2][iz];
          val += w * d.pref * d.mu[a] * d.mu[b] * (3.0 * e_al * e_be - (al == be ? 1.0 : 0.0)) / (len * len * len);
        }
  }
  Zb[idx] = make_double2(val, 0.0);
}

// add exchange taps of (target a, source b) to component (alpha, beta); serial, deterministic
__global__ void k_add_taps(double2 *__restrict__ Zb, const DevTap *__restrict__ taps, int t0, int t1, int b, int al,
                           int be, int nx, int ny, int nz) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int t = t0; t < t1; ++t) {
    const DevTap &tp = taps[t];
    if (tp.b != b) continue;
    const double J = tp.iso ? (al == be ? tp.J[0] : 0.0) : tp.J[3 * al + be];
    if (J == 0.0) continue;
    const int x = ((tp.dx % nx) + nx) % nx, y = ((tp.dy % ny) + ny) % ny, z = ((tp.dz % nz) + nz) % nz;
    Zb[x + (long long)nx * (y + (long long)ny * z)].x += J;
  }
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

template <typename R>
int pick_w(int n, int extent) {
  const size_t csz = sizeof(typename CxT<R>::T);
  int w = 16;
  while (w > 1 && ((size_t)w * fft_pitch(n) * csz > kFftSmem || w > extent)) w >>= 1;
  return w;
}

// 3D transform of nfields packed fields in place (x, y, z passes; axes of length 1 skipped)
template <typename R>
cudaError_t fft3d(const FftPlan &fp, typename CxT<R>::T *Z, int nfields, const void *const tw[3], int inverse,
                  cudaStream_t st) {
  using C = typename CxT<R>::T;
  const int nx = fp.n[0], ny = fp.n[1], nz = fp.n[2];
  const long long N = fp.N;
  for (int ax = 0; ax < 3; ++ax) {
    const int n = fp.n[ax];
    if (n < 2) continue;
    int W;
    dim3 grid;
    long long gs, os, is;
    int ifast;
    if (ax == 0) {  // lines along x, grouped along y
      W = pick_w<R>(n, ny);
      grid = dim3(ny / W, nz, nfields);
      gs = nx;
      os = (long long)nx * ny;
      is = 1;
      ifast = 1;
    } else if (ax == 1) {  // lines along y, grouped along x
      W = pick_w<R>(n, nx);
      grid = dim3(nx / W, nz, nfields);
      gs = 1;
      os = (long long)nx * ny;
      is = nx;
      ifast = 0;
    } else {  // lines along z, grouped along x
      W = pick_w<R>(n, nx);
      grid = dim3(nx / W, ny, nfields);
      gs = 1;
      os = nx;
      is = (long long)nx * ny;
      ifast = 0;
    }
    const size_t smem = (size_t)W * fft_pitch(n) * sizeof(C);
    k_fft_pass<R><<<grid, kFftThreads, smem, st>>>(Z, n, fp.logn[ax], W, ifast, gs, os, is, N,
                                                   static_cast<const C *>(tw[ax]), inverse);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

FftGeo fft_geo(const FftPlan &fp) {
  FftGeo g;
  g.nx = fp.n[0];
  g.ny = fp.n[1];
  g.nz = fp.n[2];
  g.m = g.nx / 2;
  g.nh = g.m + 1;
  g.np = (g.nh + 15) & ~15;
  g.logx = fp.logn[0];
  g.logm = fp.logn[0] - 1;
  g.lzb = std::min(fp.logn[2], 4);  // z blocks of min(16, nz) planes
  g.N = fp.N;
  g.Nh = fp.Nh;
  return g;
}

// The half spectrum b^ = M s^ of the real channels `in`, left in fp.Z (x, y forward, z with the
// kernel multiply, y inverse); k_xc2r then brings it back along x.
// in == nullptr: the x pass has been done already (the predictor's pass transforms S~ along x).
template <typename R, typename Tin>
cudaError_t spectrum_field(const FftPlan &fp, const Tin *in, cudaStream_t st) {
  using C = typename CxT<R>::T;
  C *Z = static_cast<C *>(fp.Z);
  const FftGeo g = fft_geo(fp);
  const C *twm = static_cast<const C *>(fp.twm), *twr = static_cast<const C *>(fp.twr);
  const size_t cs = sizeof(C);
  cudaError_t e = cudaSuccess;
  if (in) {
    k_xr2c<R, Tin><<<dim3((g.ny + fp.wx - 1) / fp.wx, g.nz), kHalfThreads, fp.wx * fft_pitch(g.m) * cs, st>>>(
        in, Z, g, fp.nch, fp.wx, twm, twr);
    e = cudaGetLastError();
  }
  const dim3 gy((g.nh + fp.wy - 1) / fp.wy, g.nz, fp.nch);
  const size_t smy = fp.wy * fft_pitch(g.ny) * cs;
  if (e == cudaSuccess && g.ny > 1) {
    k_hpass<R><<<gy, kHalfThreads, smy, st>>>(Z, g, fp.logn[1], fp.wy, g.nh, (long long)g.np << g.lzb, g.Nh,
                                             static_cast<const C *>(fp.tw[1]), 0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const dim3 gz((g.nh + fp.wz - 1) / fp.wz, g.ny);
    const size_t smz = (size_t)fp.nch * fp.wz * fft_pitch(g.nz) * cs;
    const R *Md = static_cast<const R *>(fp.Md);
    const C *Mo = static_cast<const C *>(fp.Mo);
    if (fp.nch == 3)
      k_zkz<R, 3><<<gz, kHalfThreads, smz, st>>>(Z, Md, Mo, g, fp.logn[2], fp.wz, static_cast<const C *>(fp.tw[2]));
    else
      k_zkz<R, 6><<<gz, kHalfThreads, smz, st>>>(Z, Md, Mo, g, fp.logn[2], fp.wz, static_cast<const C *>(fp.tw[2]));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && g.ny > 1) {
    k_hpass<R><<<gy, kHalfThreads, smy, st>>>(Z, g, fp.logn[1], fp.wy, g.nh, (long long)g.np << g.lzb, g.Nh,
                                             static_cast<const C *>(fp.tw[1]), 1);
    e = cudaGetLastError();
  }
  return e;
}

template <typename R, int MODE, typename Tout>
cudaError_t launch_xc2r(const FftPlan &fp, const XArgs<R, Tout> &xa, cudaStream_t st) {
  using C = typename CxT<R>::T;
  const FftGeo g = fft_geo(fp);
  const size_t sm = (size_t)fp.nch * fp.wc * fft_pitch(g.m) * sizeof(C);
  const dim3 grid((g.ny + fp.wc - 1) / fp.wc, g.nz);
  C *Z = static_cast<C *>(fp.Z);
  const C *twm = static_cast<const C *>(fp.twm), *twr = static_cast<const C *>(fp.twr);
  if (fp.nsub == 1)
    k_xc2r<R, MODE, Tout, 1><<<grid, kHalfThreads, sm, st>>>(Z, g, fp.wc, twm, twr, xa);
  else
    k_xc2r<R, MODE, Tout, 2><<<grid, kHalfThreads, sm, st>>>(Z, g, fp.wc, twm, twr, xa);
  return cudaGetLastError();
}

// field of the real channels `in` (FP64 spins or plan-precision predictor state) into `out`
template <typename R, typename Tin, typename Tout>
cudaError_t field_pipeline(const sx_ctx *c, const Tin *in, Tout *out, bool onsite, cudaStream_t st) {
  const FftPlan &fp = *c->fft;
  cudaError_t e = spectrum_field<R, Tin>(fp, in, st);
  if (e != cudaSuccess) return e;
  XArgs<R, Tout> xa;
  memset(&xa, 0, sizeof(xa));
  if constexpr (sizeof(Tin) == sizeof(double))
    xa.S = reinterpret_cast<const double *>(in);
  else
    xa.Sr = reinterpret_cast<const R *>(in);
  xa.out = out;
  xa.os = onsite_cast<R>(c->onsite);
  xa.onsite = onsite ? 1 : 0;
  return launch_xc2r<R, XE_FIELD, Tout>(fp, xa, st);
}

// field(S^n) -> predictor and the x transform of S~ (in one x pass) -> field(S~) -> corrector (in the x pass)
template <typename R>
cudaError_t heun_pipeline(const sx_ctx *c, const double *src, double *dst, const HeunConst &h, uint64_t step,
                          cudaStream_t st) {
  const FftPlan &fp = *c->fft;
  XArgs<R, R> xa;
  memset(&xa, 0, sizeof(xa));
  xa.S = src;
  xa.St = static_cast<R *>(fp.St);
  xa.F0 = static_cast<R *>(fp.F0);
  xa.Th = static_cast<R *>(fp.Th);
  xa.Sr = static_cast<const R *>(fp.St);
  xa.Snew = dst;
  xa.status = c->d_status;
  xa.os = onsite_cast<R>(c->onsite);
  xa.h = heun_cast<R>(h);
  xa.step = step;
  cudaError_t e = spectrum_field<R, double>(fp, src, st);
  if (e == cudaSuccess) e = launch_xc2r<R, XE_PRED, R>(fp, xa, st);
  if (e == cudaSuccess) e = spectrum_field<R, R>(fp, nullptr, st);  // S~ was transformed along x by the predictor
  if (e == cudaSuccess) e = launch_xc2r<R, XE_CORR, R>(fp, xa, st);
  return e;
}

template <typename R>
std::vector<typename CxT<R>::T> twiddles(int n) {
  std::vector<typename CxT<R>::T> t(n / 2 > 0 ? n / 2 : 1);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n / 2; ++k) {
    t[k].x = (R)cos(-2.0 * pi * k / n);
    t[k].y = (R)sin(-2.0 * pi * k / n);
  }
  return t;
}

template <typename R>
cudaError_t alloc_twiddles(const FftPlan &fp, void *tw[3]) {
  for (int ax = 0; ax < 3; ++ax) {
    std::vector<typename CxT<R>::T> t = twiddles<R>(fp.n[ax]);
    cudaError_t e = cudaMalloc(&tw[ax], t.size() * sizeof(t[0]));
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(tw[ax], t.data(), t.size() * sizeof(t[0]), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename R>
cudaError_t set_fft_smem() {
  const int b = (int)kFftSmem;
  cudaError_t e = cudaFuncSetAttribute(k_fft_pass<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xr2c<R, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xr2c<R, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_hpass<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_zkz<R, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_zkz<R, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  for (auto fn : {k_xc2r<R, XE_FIELD, double, 1>, k_xc2r<R, XE_FIELD, double, 2>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  for (auto fn : {k_xc2r<R, XE_PRED, R, 1>, k_xc2r<R, XE_PRED, R, 2>, k_xc2r<R, XE_CORR, R, 1>,
                  k_xc2r<R, XE_CORR, R, 2>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  return e;
}

// lines per CTA: the largest power of two up to 16 whose staging (bytes_per_line each) fits in a quarter of
// the shared memory (four CTAs per SM) and that does not exceed the extent of the grouping axis
inline int pick_lines(size_t bytes_per_line, int extent, size_t budget = kHalfBudget) {
  int w = 16;
  while (w > 1 && ((size_t)w * bytes_per_line > budget || w > extent)) w >>= 1;
  return w;
}

// M(q) in FP64: fill each upper-triangle component in real space, transform
// with e^{+i q.delta}, store in the plan precision
template <typename R>
cudaError_t build_kernel(sx_ctx *c, FftPlan &fp) {
  const long long N = fp.N;
  double2 *Zb = nullptr;
  void *tw64[3] = {nullptr, nullptr, nullptr};
  cudaError_t e = cudaMalloc(&Zb, N * sizeof(double2));
  if (e == cudaSuccess) e = alloc_twiddles<double>(fp, tw64);
  if (e == cudaSuccess) e = set_fft_smem<double>();
  DipArgs d;
  memset(&d, 0, sizeof(d));
  d.nx = fp.n[0];
  d.ny = fp.n[1];
  d.nz = fp.n[2];
  d.nsub = fp.nsub;
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 3; ++j) d.A[k][j] = c->lat.a[k][j];
  for (int s = 0; s < fp.nsub; ++s) {
    for (int k = 0; k < 3; ++k) d.pos[s][k] = c->lat.sub_pos[s][k];
    d.mu[s] = c->lat.mu[s];
  }
  // mu0 mu_B^2 / (4 pi) in meV nm^3: 1e-7 T m/A * (9.2740100783e-24 J/T)^2, J m^3 -> meV nm^3
  d.pref = 1e-7 * 9.2740100783e-24 * 9.2740100783e-24 * 1e27 / 1.602176634e-22;
  d.tol = c->tol;
  d.dipolar = c->dipolar;
  std::vector<int> off(fp.nsub + 1, 0);
  for (int a = 0; a < fp.nsub; ++a) off[a + 1] = off[a] + (int)c->taps[a].size();
  int p = 0;
  for (int ka = 0; ka < fp.nch && e == cudaSuccess; ++ka)
    for (int kb = ka; kb < fp.nch && e == cudaSuccess; ++kb) {
      const int a = ka % fp.nsub, al = ka / fp.nsub, b = kb % fp.nsub, be = kb / fp.nsub;
      k_fill_dipolar<<<blocks_for(N, 256), 256>>>(Zb, d, a, al, b, be);
      k_add_taps<<<1, 1>>>(Zb, c->d_taps, off[a], off[a + 1], b, al, be, fp.n[0], fp.n[1], fp.n[2]);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = fft3d<double>(fp, Zb, 1, tw64, 1, 0);
      if (e != cudaSuccess) break;
      const FftGeo g = fft_geo(fp);
      if (ka == kb) {
        k_store_diag_h<R><<<blocks_for(fp.Nh, 256), 256>>>(Zb, static_cast<R *>(fp.Md) + ka * fp.Nh, g);
      } else {
        k_store_off_h<R><<<blocks_for(fp.Nh, 256), 256>>>(Zb, static_cast<typename CxT<R>::T *>(fp.Mo) + p * fp.Nh,
                                                          g);
        ++p;
      }
      e = cudaGetLastError();
    }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(Zb);
  for (int k = 0; k < 3; ++k) cudaFree(tw64[k]);
  return e;
}

template <typename R>
cudaError_t alloc_plan(FftPlan &fp) {
  using C = typename CxT<R>::T;
  const long long N = fp.N, Nh = fp.Nh;
  cudaError_t e = cudaMalloc(&fp.Z, (size_t)fp.nch * Nh * sizeof(C));
  if (e == cudaSuccess) e = cudaMalloc(&fp.Md, (size_t)fp.nch * Nh * sizeof(R));
  if (e == cudaSuccess && fp.noff) e = cudaMalloc(&fp.Mo, (size_t)fp.noff * Nh * sizeof(C));
  if (e == cudaSuccess) e = cudaMalloc(&fp.St, (size_t)fp.nch * N * sizeof(R));
  if (e == cudaSuccess) e = cudaMalloc(&fp.F0, (size_t)fp.nch * N * sizeof(R));
  if (e == cudaSuccess) e = cudaMalloc(&fp.Th, (size_t)fp.nch * N * sizeof(R));
  if (e == cudaSuccess) e = alloc_twiddles<R>(fp, fp.tw);
  if (e == cudaSuccess) {
    // the nx/2-point transform of the x passes and the split factors of the real-to-complex step
    const int m = fp.n[0] / 2;
    std::vector<C> tm = twiddles<R>(m), tr(m + 1);
    const double pi = 3.14159265358979323846;
    for (int q = 0; q <= m; ++q) {
      tr[q].x = (R)cos(-2.0 * pi * q / fp.n[0]);
      tr[q].y = (R)sin(-2.0 * pi * q / fp.n[0]);
    }
    e = cudaMalloc(&fp.twm, tm.size() * sizeof(C));
    if (e == cudaSuccess) e = cudaMemcpy(fp.twm, tm.data(), tm.size() * sizeof(C), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&fp.twr, tr.size() * sizeof(C));
    if (e == cudaSuccess) e = cudaMemcpy(fp.twr, tr.data(), tr.size() * sizeof(C), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = set_fft_smem<R>();
  const size_t cs = sizeof(C);
  const int nh = fp.n[0] / 2 + 1;
  fp.wx = pick_lines((size_t)fft_pitch(fp.n[0] / 2) * cs, fp.n[1]);
  // the y pass takes up to twice the four-CTA budget: at ny = 1024 eight lines (74 KB, three CTAs per SM,
  // 64-byte row segments) ran the 1024^3 step 3% faster than four
  fp.wy = pick_lines((size_t)fft_pitch(fp.n[1]) * cs, nh, 2 * kHalfBudget);
  // the z pass reads rows of W adjacent qx: at least four (a whole 32-byte sector) even at two CTAs per SM
  fp.wz = pick_lines((size_t)fp.nch * fft_pitch(fp.n[2]) * cs, nh);
  if (fp.wz < 4) fp.wz = std::max(fp.wz, pick_lines((size_t)fp.nch * fft_pitch(fp.n[2]) * cs, std::min(nh, 4),
                                                      2 * kHalfBudget + 1024));
  fp.wc = pick_lines((size_t)fp.nch * fft_pitch(fp.n[0] / 2) * cs, fp.n[1]);
  return e;
}

}  // namespace

void fft_free(sx_ctx *c) {
  FftPlan *fp = c->fft;
  if (!fp) return;
  cudaFree(fp->Z);
  cudaFree(fp->Md);
  cudaFree(fp->Mo);
  cudaFree(fp->St);
  cudaFree(fp->F0);
  cudaFree(fp->Th);
  cudaFree(fp->twm);
  cudaFree(fp->twr);
  for (int k = 0; k < 3; ++k) cudaFree(fp->tw[k]);
  delete fp;
  c->fft = nullptr;
}

int fft_plan(sx_ctx *c) {
  if (c->prec != SX_PREC_FP32 && c->prec != SX_PREC_FP64)
    return set_error(SX_ERR_UNSUPPORTED, "the FFT backend computes in FP32 or FP64");
  if (c->lat.nsub > 2) return set_error(SX_ERR_UNSUPPORTED, "the FFT backend supports up to two sublattices");
  for (int k = 0; k < 3; ++k) {
    const int n = c->lat.n[k];
    if (!c->lat.pbc[k]) return set_error(SX_ERR_UNSUPPORTED, "the FFT backend needs periodic boundaries on every axis");
    if (n & (n - 1)) return set_error(SX_ERR_UNSUPPORTED, "the FFT backend needs power-of-two cell counts");
    if (k == 0 && n < 2) return set_error(SX_ERR_UNSUPPORTED, "the FFT backend needs at least two cells along x");
    if (n > 4096) return set_error(SX_ERR_UNSUPPORTED, "the FFT backend supports up to 4096 cells per axis");
  }
  FftPlan *fp = new (std::nothrow) FftPlan();
  if (!fp) return set_error(SX_ERR_OOM, "host allocation failed");
  memset(fp, 0, sizeof(*fp));
  fp->prec = c->prec;
  for (int k = 0; k < 3; ++k) {
    fp->n[k] = c->lat.n[k];
    fp->logn[k] = ilog2(c->lat.n[k]);
  }
  fp->nsub = c->lat.nsub;
  fp->nch = 3 * fp->nsub;
  fp->noff = fp->nch * (fp->nch - 1) / 2;
  fp->N = c->geo.ncell;
  fp->Nh = (long long)((fp->n[0] / 2 + 1 + 15) & ~15) * fp->n[1] * fp->n[2];
  c->fft = fp;
  cudaError_t e = (fp->prec == SX_PREC_FP32) ? alloc_plan<float>(*fp) : alloc_plan<double>(*fp);
  if (e == cudaSuccess) e = (fp->prec == SX_PREC_FP32) ? build_kernel<float>(c, *fp) : build_kernel<double>(c, *fp);
  if (e != cudaSuccess) {
    fft_free(c);
    return cuda_error(e, "FFT plan");
  }
  c->launches_per_step = 2 * (3 + 2 * (fp->n[1] > 1)) - 1;
  return SX_OK;
}

// Heun stages that take the bilinear field from a buffer (also used by the tensor-core backend)
cudaError_t bufheun_predict(const sx_ctx *c, const double *S, const float *Bf, float *St, float *F0, float *Th,
                            const HeunConst &h, uint64_t step, cudaStream_t st) {
  const long long N = c->geo.ncell;
  k_fft_predict<float><<<blocks_for(N, 256), 256, 0, st>>>(S, Bf, St, F0, Th, c->lat.nsub, N,
                                                           onsite_cast<float>(c->onsite), heun_cast<float>(h), step);
  return cudaGetLastError();
}

cudaError_t bufheun_correct(const sx_ctx *c, const double *S, const float *St, const float *F0, const float *Bf,
                            const float *Th, double *Snew, const HeunConst &h, cudaStream_t st) {
  const long long N = c->geo.ncell;
  k_fft_correct<float><<<blocks_for(N, 256), 256, 0, st>>>(S, St, F0, Bf, Th, Snew, c->lat.nsub, N,
                                                           onsite_cast<float>(c->onsite), heun_cast<float>(h),
                                                           c->d_status);
  return cudaGetLastError();
}

cudaError_t fft_field(const sx_ctx *c, const double *S, double *b, bool onsite, cudaStream_t st) {
  if (c->fft->prec == SX_PREC_FP32) return field_pipeline<float, double, double>(c, S, b, onsite, st);
  return field_pipeline<double, double, double>(c, S, b, onsite, st);
}

cudaError_t fft_heun_step(const sx_ctx *c, const double *src, double *dst, const HeunConst &h, uint64_t step,
                          cudaStream_t st) {
  if (c->fft->prec == SX_PREC_FP32) return heun_pipeline<float>(c, src, dst, h, step, st);
  return heun_pipeline<double>(c, src, dst, h, step, st);
}

}  // namespace sx
