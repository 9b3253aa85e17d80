"""Throughput of the GB300 pipes the kernel design rests on, measured on the device.

The library keeps FP64 work off its hot paths (integer-bit conversions, fixed-point renormalisation)
because FP64 arithmetic runs far below the FP32 rate on this part.  This test measures that ratio
with a small probe (independent FMA chains per thread, CUDA-event timing, no memory traffic), prints
the rates, and fails if FP64 were ever within a factor 20 of FP32, which would invalidate the design.
The FP64 rate it prints is the ALU peak that bench.py's roofline block uses."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PROBE = r"""
#include <cstdio>
#include <cuda_runtime.h>
constexpr int kIter = 2048, kChains = 8, kThreads = 256;
__device__ double g_d[1 << 16];
__device__ float g_f[1 << 16];
__device__ unsigned g_u[1 << 16];

__global__ void k_dfma(double seed) {
  double a[kChains];
  for (int i = 0; i < kChains; ++i) a[i] = seed + i + threadIdx.x;
  for (int it = 0; it < kIter; ++it)
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], 0.99999999, 1e-9);
  double s = 0.0;
  for (int i = 0; i < kChains; ++i) s += a[i];
  g_d[(blockIdx.x * kThreads + threadIdx.x) & 0xFFFF] = s;
}
__global__ void k_ffma(float seed) {
  float a[kChains];
  for (int i = 0; i < kChains; ++i) a[i] = seed + i + threadIdx.x;
  for (int it = 0; it < kIter; ++it)
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], 0.9999999f, 1e-7f);
  float s = 0.0f;
  for (int i = 0; i < kChains; ++i) s += a[i];
  g_f[(blockIdx.x * kThreads + threadIdx.x) & 0xFFFF] = s;
}
__global__ void k_imad(unsigned seed) {
  unsigned a[kChains];
  for (int i = 0; i < kChains; ++i) a[i] = seed + i + threadIdx.x;
  for (int it = 0; it < kIter; ++it)
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = a[i] * (a[i] | 1u) + 0x7F4A7C15u;  // quadratic: not foldable
  unsigned s = 0;
  for (int i = 0; i < kChains; ++i) s ^= a[i];
  g_u[(blockIdx.x * kThreads + threadIdx.x) & 0xFFFF] = s;
}

template <class F>
static double rate(F launch, int blocks) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  launch(blocks);
  cudaEventRecord(e0);
  for (int r = 0; r < 5; ++r) launch(blocks);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  return 5.0 * blocks * kThreads * (double)kIter * kChains / (ms * 1e-3);
}

int main() {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const int blocks = sms * 16;
  const double d = rate([](int b) { k_dfma<<<b, kThreads>>>(1.0); }, blocks);
  const double f = rate([](int b) { k_ffma<<<b, kThreads>>>(1.0f); }, blocks);
  const double u = rate([](int b) { k_imad<<<b, kThreads>>>(1u); }, blocks);
  if (cudaDeviceSynchronize() != cudaSuccess) return 1;
  printf("%.6e %.6e %.6e\n", d, f, u);
  return 0;
}
"""


def test_fp64_rate_is_far_below_fp32(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = tmp_path / "probe.cu"
    src.write_text(PROBE)
    exe = tmp_path / "probe"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    dfma, ffma, imad = (float(v) for v in out.stdout.split())
    print(f"FP64 FMA {dfma / 1e9:.0f} G/s, FP32 FMA {ffma / 1e9:.0f} G/s, INT32 IMAD {imad / 1e9:.0f} G/s "
          f"(thread operations), FP32/FP64 = {ffma / dfma:.1f}")
    assert ffma > 20.0 * dfma
    assert imad > 5.0 * dfma
