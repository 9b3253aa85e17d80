"""Work orders of the stencil backend's multi-unit launches (csrc/sx_schedule.h), compiled for the host.

The balanced schedule of small lattices cuts the column-plane units into one contiguous range per
resident CTA; it must cover every unit exactly once within the CTA slots.  The overlapped two-pass
launch takes predictor and corrector units from one queue, and the pipelined
host-array step issues predictor and corrector passes over z chunks while the uploads and downloads of
other chunks are in flight.  Both are correct only if every unit appears once and every corrector unit
comes after the predictor units of its S~ halo (the 3 x 3 neighbouring columns in the chunks z - 1 ..
z + 1, wrapped on periodic axes, absent beyond open faces), and, in the first host-array step, every
predictor waits for the uploads of the chunks it reads.  Checked here on every small geometry and
boundary combination and on the 1024^3 bench geometry."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2605_26016_gb300", "csrc")

DRIVER = r"""
#include <stdio.h>
#include <vector>
#include "sx_schedule.h"
using namespace sx::sched;

// the chunks (or columns) a unit's halo touches, restated: positions c - 1 .. c + 1 on an axis of n
static std::vector<int> near(int c, int n, int per) {
  std::vector<int> out;
  for (int d = -1; d <= 1; ++d) {
    int q = c + d;
    if (q < 0 || q >= n) {
      if (!per) continue;
      q = (q + n) % n;
    }
    out.push_back(q);
  }
  return out;
}

static int check_queue(int ncx, int ncy, int K, int px, int py, int pz, long long lag) {
  const int ncol = ncx * ncy;
  const std::vector<int> q = overlap_order(ncx, ncy, K, px, py, pz, lag);
  std::vector<long long> pos_pred(K * ncol, -1), pos_corr(K * ncol, -1);
  if ((long long)q.size() != 2LL * K * ncol) return 1;
  for (long long i = 0; i < (long long)q.size(); ++i) {
    const int idx = q[i] & (kUnitCorr - 1);
    if (idx < 0 || idx >= K * ncol) return 2;
    std::vector<long long> &pos = (q[i] & kUnitCorr) ? pos_corr : pos_pred;
    if (pos[idx] >= 0) return 3;  // twice
    pos[idx] = i;
  }
  for (int z = 0; z < K; ++z)
    for (int cy = 0; cy < ncy; ++cy)
      for (int cx = 0; cx < ncx; ++cx) {
        const long long at = pos_corr[z * ncol + cy * ncx + cx];
        for (int zz : near(z, K, pz))
          for (int yy : near(cy, ncy, py))
            for (int xx : near(cx, ncx, px))
              if (pos_pred[zz * ncol + yy * ncx + xx] > at) return 4;  // a dependency after its user
      }
  return 0;
}

static int check_host(int K, bool pz, bool first, bool last) {
  const std::vector<ChunkOp> ops = host_step_ops(K, pz, first, last);
  std::vector<int> pred_at(K, -1), corr_at(K, -1);
  if ((int)ops.size() != 2 * K) return 11;
  for (int i = 0; i < (int)ops.size(); ++i) {
    const ChunkOp &o = ops[i];
    if (o.z < 0 || o.z >= K) return 12;
    int &at = o.corr ? corr_at[o.z] : pred_at[o.z];
    if (at >= 0) return 13;
    at = i;
    if (!o.corr && first)
      for (int q : near(o.z, K, pz))
        if (o.wait < q) return 14;  // uploads run in chunk order: chunks 0 .. wait are in place
    if (!o.corr && !first && o.wait != -1) return 15;
    if (o.corr && o.wait != -1) return 16;
  }
  for (int z = 0; z < K; ++z)
    for (int q : near(z, K, pz))
      if (pred_at[q] > corr_at[z]) return 17;
  return 0;
}

struct Rg {
  int x, y;
};

// ranges tile [0, U) in order, at most `slots` of them, each costing (planes + w per column segment,
// columns of nz units) no more than `bound`
static int check_ranges(const std::vector<Rg> &rs, const std::vector<long long> &ncol, const std::vector<int> &nz,
                        long long slots, long long w, long long bound) {
  std::vector<long long> off(ncol.size() + 1, 0);
  for (size_t r = 0; r < ncol.size(); ++r) off[r + 1] = off[r] + ncol[r] * nz[r];
  const long long U = off.back();
  if ((long long)rs.size() > slots) return 21;
  long long u = 0;
  for (const Rg &g : rs) {
    if (g.x != u || g.y < 1) return 22;
    long long cost = 0, v = g.x;
    size_t r = 0;
    while (v < (long long)g.x + g.y) {
      while (v >= off[r + 1]) ++r;
      const long long end = std::min<long long>((long long)g.x + g.y, off[r] + ((v - off[r]) / nz[r] + 1) * nz[r]);
      cost += w + (end - v);  // one column segment
      v = end;
    }
    if (cost > bound) return 23;
    u += g.y;
  }
  return u == U ? 0 : 24;
}

int main(void) {
  long n = 0;
  for (int R = 1; R <= 2; ++R)
    for (long long ncol : {1LL, 3LL, 32LL, 100LL, 151LL})
      for (int nz : {1, 2, 5, 17, 64, 128})
        for (long long slots : {1LL, 7LL, 152LL, 304LL}) {
          const long long w = 2 * R;
          const std::vector<Rg> rs = balanced_schedule<Rg>(ncol, nz, R, slots);
          const long long hi = std::max<long long>(std::max<long long>(w + 1, (ncol * nz + slots - 1) / slots + w),
                                                   ((ncol + slots - 1) / slots) * (nz + w));
          const int r = check_ranges(rs, {ncol}, {nz}, slots, w, hi);
          if (r) { printf("balanced %lld %d %d %lld: %d\n", ncol, nz, R, slots, r); return 1; }
          ++n;
        }
  {  // replicas of different sizes, the units of one after the other's
    const std::vector<long long> ncol = {4, 12, 1, 30};
    const std::vector<int> nz = {24, 48, 7, 96};
    for (long long slots : {1LL, 5LL, 152LL}) {
      const std::vector<Rg> rs = balanced_schedule_multi<Rg>(ncol, nz, 2, slots);
      long long U = 0, cols = 0;
      for (size_t r = 0; r < ncol.size(); ++r) { U += ncol[r] * nz[r]; cols += ncol[r]; }
      const int r = check_ranges(rs, ncol, nz, slots, 4, U + 4 * cols);
      if (r) { printf("multi %lld: %d\n", slots, r); return 1; }
      ++n;
    }
  }
  // the point of the schedule: 32 columns of 128 planes over 152 CTAs cost far less than whole columns
  {
    const std::vector<Rg> rs = balanced_schedule<Rg>(32, 128, 2, 152);
    if (check_ranges(rs, {32}, {128}, 152, 4, 4 * 4 + 128 * 32 / 152 + 1) != 0) { printf("not balanced\n"); return 1; }
  }
  for (int ncx = 1; ncx <= 4; ++ncx)
    for (int ncy = 1; ncy <= 4; ++ncy)
      for (int K = 1; K <= 5; ++K)
        for (int b = 0; b < 8; ++b)
          for (long long lag : {0LL, 1LL, 5LL, 1000LL}) {
            const int r = check_queue(ncx, ncy, K, b & 1, (b >> 1) & 1, (b >> 2) & 1, lag);
            if (r) { printf("queue %d %d %d %d %lld: %d\n", ncx, ncy, K, b, lag, r); return 1; }
            ++n;
          }
  for (int b = 0; b < 8; b += 7) {  // the 1024^3 bench geometry: 32 x 64 columns, chunks of 64 planes
    const int r = check_queue(32, 64, 16, b & 1, (b >> 1) & 1, (b >> 2) & 1, 304);
    if (r) { printf("queue bench %d: %d\n", b, r); return 1; }
    ++n;
  }
  for (int K : {1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 20, 31, 32, 63, 64})
    for (int pz = 0; pz < 2; ++pz)
      for (int f = 0; f < 2; ++f)
        for (int l = 0; l < 2; ++l) {
          const int r = check_host(K, pz, f, l);
          if (r) { printf("host %d %d %d %d: %d\n", K, pz, f, l, r); return 1; }
          ++n;
        }
  // the first and last step of a one-step call overlap: some corrector comes before the last predictor
  const std::vector<ChunkOp> one = host_step_ops(64, true, true, true);
  int first_corr = -1, last_pred = -1;
  for (int i = 0; i < (int)one.size(); ++i) {
    if (one[i].corr && first_corr < 0) first_corr = i;
    if (!one[i].corr) last_pred = i;
  }
  if (first_corr < 0 || first_corr > last_pred) { printf("no overlap\n"); return 1; }
  printf("%ld\n", n);
  return 0;
}
"""


def test_work_orders_respect_their_dependencies(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "drv.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "drv"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert int(out.stdout.split()[-1]) > 2000
