"""The fixed-point part of the FP64 state renormalisation (csrc/sx_fixed.h), compiled for the host.

For x = S + d with S on the unit sphere and a step d, the library forms x in FP64, takes
eps = |x|^2 - 1 and t = (1 + eps)^(-1/2) - 1 in 64-bit fixed point, and returns S' = x + x t with
one FP64 fused multiply-add per component.  Checked here against x / |x| in extended precision
(long double) on a million seeded cases: unit spheres of every orientation, steps from 1e-9 to
the 2^-10 limit of eps, zero and tiny components, and the out-of-range inputs that must fall back."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2605_26016_gb300", "csrc")

DRIVER = r"""
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include "sx_fixed.h"

static uint64_t st = 0x9E3779B97F4A7C15ull;
static double urand() {  /* splitmix64 -> [0, 1) */
  uint64_t z = (st += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1p-53;
}

int main(void) {
  long n = 0, fast = 0;
  double worst_c = 0.0, worst_n = 0.0, worst_t = 0.0;
  for (long k = 0; k < 1000000; ++k) {
    double S[3];
    const double z = 2.0 * urand() - 1.0, ph = 2.0 * M_PI * urand(), r = sqrt(1.0 - z * z);
    S[0] = r * cos(ph); S[1] = r * sin(ph); S[2] = z;
    if (k % 7 == 0) S[k % 3] = 0.0;                                  /* exact zero component */
    if (k % 11 == 0) S[(k + 1) % 3] *= 1e-20;                        /* tiny component */
    const long double ns = sqrtl((long double)S[0] * S[0] + (long double)S[1] * S[1] + (long double)S[2] * S[2]);
    for (int c = 0; c < 3; ++c) S[c] = (double)(S[c] / ns);
    const double scale = pow(10.0, -9.0 + 7.5 * urand());           /* |d| from 1e-9 to ~3e-2 */
    float d[3];
    for (int c = 0; c < 3; ++c) d[c] = (float)(scale * (2.0 * urand() - 1.0));
    double x[3];
    for (int c = 0; c < 3; ++c) x[c] = S[c] + (double)d[c];
    double t;
    const long double n2 = (long double)x[0] * x[0] + (long double)x[1] * x[1] + (long double)x[2] * x[2];
    const long double eps = n2 - 1.0L;
    const int ok = sx::fx::t_of_x(sx::fx::dbits(x[0]), sx::fx::dbits(x[1]), sx::fx::dbits(x[2]), t);
    ++n;
    if (fabsl(eps) < 0x1p-10L * 0.999L && !ok) { printf("MISSED %Lg\n", eps); return 1; }
    if (fabsl(eps) >= 0x1p-10L * 1.001L && ok) { printf("WRONGLY FAST %Lg\n", eps); return 1; }
    if (!ok) continue;
    ++fast;
    const long double tref = 1.0L / sqrtl(n2) - 1.0L;
    const double et = (double)fabsl((long double)t - tref);
    if (et > worst_t) worst_t = et;
    double o[3];
    long double on2 = 0.0L;
    for (int c = 0; c < 3; ++c) {
      o[c] = fma(x[c], t, x[c]);
      const double e = (double)fabsl((long double)o[c] - (long double)x[c] / sqrtl(n2));
      if (e > worst_c) worst_c = e;
      on2 += (long double)o[c] * o[c];
    }
    const double en = (double)fabsl(on2 - 1.0L);
    if (en > worst_n) worst_n = en;
  }
  /* out of range: NaN, infinity, |x_c| >= 2 */
  double t = 0.0;
  const double bad[3][3] = {{NAN, 0.0, 1.0}, {INFINITY, 0.0, 0.0}, {2.0, 0.0, 0.0}};
  for (int k = 0; k < 3; ++k)
    if (sx::fx::t_of_x(sx::fx::dbits(bad[k][0]), sx::fx::dbits(bad[k][1]), sx::fx::dbits(bad[k][2]), t)) {
      printf("ACCEPTED BAD %d\n", k);
      return 1;
    }
  printf("%ld %ld %.3e %.3e %.3e\n", n, fast, worst_t, worst_c, worst_n);
  return 0;
}
"""


def test_fixed_point_renormalisation_against_extended_precision(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "drv.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "drv"
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    n, fast, worst_t, worst_c, worst_n = out.stdout.split()
    print(out.stdout)
    assert int(fast) > 0.75 * int(n)                      # the fast path covers all but the largest steps
    assert float(worst_t) < 2.0 ** -56                    # t to better than FP64 rounding of 1
    assert float(worst_c) <= 2.0 ** -52                   # every component within one unit of 2^-52
    assert float(worst_n) <= 4.5e-16                      # |S'|^2 - 1: FP64 rounding of the three products
