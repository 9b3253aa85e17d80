// Work orders of the stencil backend's multi-unit launches, as plain host C++ (the library builds them
// at plan or launch time; the tests compile this header with a host compiler and check the orders).
//
// Units are (z chunk, tile column) pairs of the two-pass Heun step: a predictor unit writes S~, f0 and
// the normals of its cells; a corrector unit reads S~ on its cells plus a halo of r cells, which lies in
// the 3 x 3 neighbouring columns of the chunks z - 1 .. z + 1 (wrapped on periodic axes, absent beyond
// open faces) as long as edge columns, rows and the last chunk are at least r wide.
#pragma once
#include <stdint.h>

#include <algorithm>
#include <vector>

namespace sx {
namespace sched {

constexpr int kUnitCorr = 1 << 30;  // queue code of a corrector unit: index | kUnitCorr

// index c on an axis of n positions: wrapped when periodic, else ok = false outside 0 .. n - 1
inline int wrap_index(int c, int n, int periodic, bool &ok) {
  if (c >= 0 && c < n) return c;
  if (!periodic) {
    ok = false;
    return 0;
  }
  return ((c % n) + n) % n;
}

// Queue of the overlapped step (one launch, CTAs taking units in queue order).  Unit index = chunk *
// ncol + column, column = cy * ncx + cx.  Predictor units chunk by chunk (on a periodic z axis the last
// chunk first: chunk 0's corrector reads it), columns in order.  Corrector units chunk by chunk, tile
// rows 1 .. ncy - 1 before row 0 (whose periodic y halo is the last row), each queued one-for-one with
// the predictor stream once `lag` more predictor units have been queued after the last predictor unit
// it depends on, so every dependency is queued before the unit itself.
inline std::vector<int> overlap_order(int ncx, int ncy, int nchunk, int px, int py, int pz, long long lag) {
  const int ncol = ncx * ncy;
  const long long P = (long long)nchunk * ncol;
  std::vector<int> pred, corr;
  std::vector<long long> pos(P), need;
  pred.reserve(P);
  corr.reserve(P);
  need.reserve(P);
  std::vector<int> zorder;
  if (pz && nchunk > 1) zorder.push_back(nchunk - 1);
  for (int z = 0; z < nchunk; ++z)
    if (!(pz && nchunk > 1 && z == nchunk - 1)) zorder.push_back(z);
  for (int z : zorder)
    for (int col = 0; col < ncol; ++col) {
      pos[(long long)z * ncol + col] = (long long)pred.size();
      pred.push_back(z * ncol + col);
    }
  for (int z = 0; z < nchunk; ++z)
    for (int r = 0; r < ncy; ++r) {
      const int cy = (r + 1) % ncy;
      for (int cx = 0; cx < ncx; ++cx) {
        long long nd = 0;
        for (int t = 0; t < 27; ++t) {
          bool ok = true;
          const int zz = wrap_index(z + t / 9 - 1, nchunk, pz, ok), yy = wrap_index(cy + (t / 3) % 3 - 1, ncy, py, ok),
                    xx = wrap_index(cx + t % 3 - 1, ncx, px, ok);
          if (ok) nd = std::max(nd, pos[(long long)zz * ncol + yy * ncx + xx]);
        }
        corr.push_back((z * ncol + cy * ncx + cx) | kUnitCorr);
        need.push_back(nd);
      }
    }
  std::vector<int> out;
  out.reserve(2 * P);
  long long pi = 0, ci = 0;
  while (pi < P || ci < P) {
    if (pi < P) out.push_back(pred[pi++]);
    if (ci < P && (pi >= P || need[ci] + lag < pi)) out.push_back(corr[ci++]);
  }
  return out;
}

// The z chunks whose planes chunk z of K reads (itself and its neighbours); returns how many.
inline int chunk_neighbours(int z, int K, bool pz, int out[3]) {
  int n = 0;
  for (int d = -1; d <= 1; ++d) {
    bool ok = true;
    const int q = wrap_index(z + d, K, pz ? 1 : 0, ok);
    if (ok) out[n++] = q;
  }
  return n;
}

// One launch of the pipelined host-array step: the predictor or corrector pass over z chunk z; a
// predictor of the first step first waits until chunks 0 .. wait have been uploaded (-1: no wait).
struct ChunkOp {
  int corr;
  int z;
  int wait;
};

// Launch sequence of one Heun step of the pipelined host-array path over K z chunks.  The uploads run
// in chunk order, so in the first step each predictor waits for the last chunk it reads, and the
// predictors go in the order in which their inputs complete.  In the last step each corrector follows
// as soon as every predictor of its S~ halo precedes it (its download can then start); otherwise the
// correctors follow the predictors in chunk order.
inline std::vector<ChunkOp> host_step_ops(int K, bool pz, bool first, bool last) {
  std::vector<int> order(K), need(K);
  for (int z = 0; z < K; ++z) {
    int nb[3];
    const int n = chunk_neighbours(z, K, pz, nb);
    need[z] = *std::max_element(nb, nb + n);
    order[z] = z;
  }
  if (first) std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return need[x] < need[y]; });
  std::vector<ChunkOp> ops;
  std::vector<char> pred_done(K, 0), corr_done(K, 0);
  for (int i = 0; i < K; ++i) {
    const int z = order[i];
    ops.push_back({0, z, first ? need[z] : -1});
    pred_done[z] = 1;
    for (int y = 0; y < K && last; ++y) {
      if (corr_done[y]) continue;
      int nb[3];
      const int n = chunk_neighbours(y, K, pz, nb);
      bool ready = true;
      for (int j = 0; j < n; ++j) ready = ready && pred_done[nb[j]];
      if (ready) {
        ops.push_back({1, y, -1});
        corr_done[y] = 1;
      }
    }
  }
  for (int y = 0; y < K; ++y)
    if (!corr_done[y]) ops.push_back({1, y, -1});
  return ops;
}

// Balanced schedule of the two-pass passes over `slots` resident CTAs, for lattices with fewer tile
// columns than CTA slots: the column-plane units u = column * nz + z are cut into contiguous ranges
// {first unit, count} (Range is any two-int aggregate: int2 on the device side), one per CTA, so that
// the largest cost (planes + 2R warm-up planes per column segment) is as small as the greedy packing
// under a binary-searched bound allows.  balanced_schedule_multi: the same over several replicas
// whose units follow each other (replica r: ncol[r] columns of nz[r] planes each).
template <class Range>
inline std::vector<Range> balanced_schedule_multi(const std::vector<long long> &ncol, const std::vector<int> &nz,
                                                 int R, long long slots) {
  const int nr = (int)ncol.size();
  std::vector<long long> off(nr + 1, 0);
  for (int r = 0; r < nr; ++r) off[r + 1] = off[r] + ncol[r] * nz[r];
  const long long U = off[nr], w = 2LL * R;
  long long colsum = 0;
  for (int r = 0; r < nr; ++r) colsum += ncol[r];
  auto pack = [&](long long B, std::vector<Range> *out) {
    long long u = 0, n = 0;
    int r = 0;
    while (u < U) {
      const long long u0 = u;
      long long cost = 0;
      while (u < U) {
        while (u >= off[r + 1]) ++r;
        const long long avail = nz[r] - (u - off[r]) % nz[r];
        if (cost + w + 1 > B) break;
        const long long t = std::min(avail, B - cost - w);
        cost += w + t;
        u += t;
        if (t < avail) break;
      }
      if (out) out->push_back(Range{(int)u0, (int)(u - u0)});
      ++n;
    }
    return n;
  };
  long long lo = std::max<long long>(w + 1, (U + slots - 1) / slots + w);
  long long hi = std::max(lo, U + w * colsum);  // one CTA taking everything always fits
  while (lo < hi) {
    const long long mid = (lo + hi) / 2;
    if (pack(mid, nullptr) <= slots)
      hi = mid;
    else
      lo = mid + 1;
  }
  std::vector<Range> out;
  pack(lo, &out);
  return out;
}

template <class Range>
inline std::vector<Range> balanced_schedule(long long ncol, int nz, int R, long long slots) {
  const long long U = ncol * nz, w = 2LL * R;
  auto pack = [&](long long B, std::vector<Range> *out) {
    long long u = 0, n = 0;
    while (u < U) {
      const long long u0 = u;
      long long cost = 0;
      while (u < U) {
        const long long avail = nz - u % nz;
        if (cost + w + 1 > B) break;
        const long long t = std::min(avail, B - cost - w);
        cost += w + t;
        u += t;
        if (t < avail) break;
      }
      if (out) out->push_back(Range{(int)u0, (int)(u - u0)});
      ++n;
    }
    return n;
  };
  // hi: whole columns, ceil(ncol / slots) of them per CTA, always fits
  long long lo = std::max<long long>(w + 1, (U + slots - 1) / slots + w);
  long long hi = std::max(lo, ((ncol + slots - 1) / slots) * (nz + w));
  while (lo < hi) {
    const long long mid = (lo + hi) / 2;
    if (pack(mid, nullptr) <= slots)
      hi = mid;
    else
      lo = mid + 1;
  }
  std::vector<Range> out;
  pack(lo, &out);
  return out;
}

}  // namespace sched
}  // namespace sx
