// Pipe-rate microbenchmark: warp-level throughput of FP64 FMA/ADD, FP32 FMA (scalar and packed f32x2),
// integer ops, f64<->f32 conversion, MUFU rsqrt, shared-memory loads, and an HBM copy.  Every access
// stays in bounds.  Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o pipe_rates pipe_rates.cu
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("CUDA %s at %d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)
constexpr int ITER = 4096;
__device__ unsigned long long g_cyc[4096];
__device__ double g_sinkd[1<<20];
__device__ float g_sinkf[1<<20];

__global__ void k_dfma(double a0) {
  double a[8]; for (int i=0;i<8;i++) a[i]=a0+i+threadIdx.x;
  double b=1.0000001, c=1e-9;
  unsigned long long t0=clock64();
  for (int it=0; it<ITER; it++) {
#pragma unroll
    for (int i=0;i<8;i++) a[i]=fma(a[i],b,c);
  }
  unsigned long long t1=clock64();
  double s=0; for(int i=0;i<8;i++) s+=a[i];
  g_sinkd[(blockIdx.x*blockDim.x+threadIdx.x)&((1<<20)-1)]=s;
  if(threadIdx.x==0) g_cyc[blockIdx.x]=t1-t0;
}
__global__ void k_dadd(double a0) {
  double a[8]; for (int i=0;i<8;i++) a[i]=a0+i+threadIdx.x;
  double c=1e-9;
  unsigned long long t0=clock64();
  for (int it=0; it<ITER; it++) {
#pragma unroll
    for (int i=0;i<8;i++) a[i]=a[i]+c;
  }
  unsigned long long t1=clock64();
  double s=0; for(int i=0;i<8;i++) s+=a[i];
  g_sinkd[(blockIdx.x*blockDim.x+threadIdx.x)&((1<<20)-1)]=s;
  if(threadIdx.x==0) g_cyc[blockIdx.x]=t1-t0;
}
__global__ void k_ffma(float a0) {
  float a[8]; for (int i=0;i<8;i++) a[i]=a0+i+threadIdx.x;
  float b=1.0000001f, c=1e-9f;
  unsigned long long t0=clock64();
  for (int it=0; it<ITER; it++) {
#pragma unroll
    for (int i=0;i<8;i++) a[i]=fmaf(a[i],b,c);
  }
  unsigned long long t1=clock64();
  float s=0; for(int i=0;i<8;i++) s+=a[i];
  g_sinkf[(blockIdx.x*blockDim.x+threadIdx.x)&((1<<20)-1)]=s;
  if(threadIdx.x==0) g_cyc[blockIdx.x]=t1-t0;
}
// packed f32x2 FMA (PTX fma.rn.f32x2 on sm_100+)
__global__ void k_ffma2(float a0) {
  unsigned long long a[8]; 
  for (int i=0;i<8;i++){ float2 v=make_float2(a0+i, a0+threadIdx.x); a[i]=*reinterpret_cast<unsigned long long*>(&v);} 
  float2 bb=make_float2(1.0000001f,1.0000001f), cc=make_float2(1e-9f,1e-9f);
  unsigned long long b=*reinterpret_cast<unsigned long long*>(&bb), c=*reinterpret_cast<unsigned long long*>(&cc);
  unsigned long long t0=clock64();
  for (int it=0; it<ITER; it++) {
#pragma unroll
    for (int i=0;i<8;i++) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[i]) : "l"(b), "l"(c));
  }
  unsigned long long t1=clock64();
  float s=0; for(int i=0;i<8;i++){ float2 v=*reinterpret_cast<float2*>(&a[i]); s+=v.x+v.y;}
  g_sinkf[(blockIdx.x*blockDim.x+threadIdx.x)&((1<<20)-1)]=s;
  if(threadIdx.x==0) g_cyc[blockIdx.x]=t1-t0;
}
__global__ void k_imad(int a0) {
  unsigned a[8]; for (int i=0;i<8;i++) a[i]=a0+i+threadIdx.x;
  unsigned b=1664525u, c=1013904223u;
  unsigned long long t0=clock64();
  for (int it=0; it<ITER; it++) {
#pragma unroll
    for (int i=0;i<8;i++) a[i]=a[i]*b+c;
  }
  unsigned long long t1=clock64();
  unsigned s=0; for(int i=0;i<8;i++) s^=a[i];
  g_sinkf[(blockIdx.x*blockDim.x+threadIdx.x)&((1<<20)-1)]=(float)s;
  if(threadIdx.x==0) g_cyc[blockIdx.x]=t1-t0;
}
__global__ void k_iadd3(int a0) {
  unsigned a[8]; for (int i=0;i<8;i++) a[i]=a0+i+threadIdx.x;
  unsigned b=1664525u;
  unsigned long long t0=clock64();
  for (int it=0; it<ITER; it++) {
#pragma unroll
    for (int i=0;i<8;i++) a[i]=(a[i]^b)+ (a[(i+1)&7]>>3);
  }
  unsigned long long t1=clock64();
  unsigned s=0; for(int i=0;i<8;i++) s^=a[i];
  g_sinkf[(blockIdx.x*blockDim.x+threadIdx.x)&((1<<20)-1)]=(float)s;
  if(threadIdx.x==0) g_cyc[blockIdx.x]=t1-t0;
}
// f64 -> f32 -> f64 round trip: 2 conversions per element-iteration
__global__ void k_cvt(double a0) {
  double a[8]; for (int i=0;i<8;i++) a[i]=a0+i*0.1+threadIdx.x;
  unsigned long long t0=clock64();
  for (int it=0; it<ITER; it++) {
#pragma unroll
    for (int i=0;i<8;i++) { float f; asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(f) : "d"(a[i])); asm volatile("cvt.f64.f32 %0, %1;" : "=d"(a[i]) : "f"(f)); }
  }
  unsigned long long t1=clock64();
  double s=0; for(int i=0;i<8;i++) s+=a[i];
  g_sinkd[(blockIdx.x*blockDim.x+threadIdx.x)&((1<<20)-1)]=s;
  if(threadIdx.x==0) g_cyc[blockIdx.x]=t1-t0;
}
__global__ void k_rsq(float a0) {
  float a[8]; for (int i=0;i<8;i++) a[i]=a0+i+threadIdx.x;
  unsigned long long t0=clock64();
  for (int it=0; it<ITER; it++) {
#pragma unroll
    for (int i=0;i<8;i++) asm volatile("rsqrt.approx.f32 %0, %0;" : "+f"(a[i]));
  }
  unsigned long long t1=clock64();
  float s=0; for(int i=0;i<8;i++) s+=a[i];
  g_sinkf[(blockIdx.x*blockDim.x+threadIdx.x)&((1<<20)-1)]=s;
  if(threadIdx.x==0) g_cyc[blockIdx.x]=t1-t0;
}
// LDS.128 bandwidth: each thread reads float4 from smem (conflict-free: consecutive 16B per lane)
__global__ void k_lds128(int salt) {
  __shared__ float4 sm[2048];
  for (int i=threadIdx.x;i<2048;i+=blockDim.x) sm[i]=make_float4(i,i+1,i+2,i+salt);
  __syncthreads();
  float4 acc=make_float4(0,0,0,0);
  int base=threadIdx.x & 1023;
  unsigned long long t0=clock64();
  for (int it=0; it<ITER; it++) {
#pragma unroll
    for (int i=0;i<8;i++) { float4 v=sm[(base + i*32 + (it&7)*128) & 2047]; acc.x+=v.x; acc.y+=v.y; acc.z+=v.z; acc.w+=v.w; }
  }
  unsigned long long t1=clock64();
  g_sinkf[(blockIdx.x*blockDim.x+threadIdx.x)&((1<<20)-1)]=acc.x+acc.y+acc.z+acc.w;
  if(threadIdx.x==0) g_cyc[blockIdx.x]=t1-t0;
}
__global__ void k_lds32(int salt) {
  __shared__ float sm[8192];
  for (int i=threadIdx.x;i<8192;i+=blockDim.x) sm[i]=i+salt;
  __syncthreads();
  float acc0=0,acc1=0;
  int base=threadIdx.x & 1023;
  unsigned long long t0=clock64();
  for (int it=0; it<ITER; it++) {
#pragma unroll
    for (int i=0;i<8;i++) { float v=sm[(base + i*32 + (it&7)*1024) & 8191]; if(i&1) acc0+=v; else acc1+=v; }
  }
  unsigned long long t1=clock64();
  g_sinkf[(blockIdx.x*blockDim.x+threadIdx.x)&((1<<20)-1)]=acc0+acc1;
  if(threadIdx.x==0) g_cyc[blockIdx.x]=t1-t0;
}
// HBM stream copy
__global__ void k_copy(const double4_32a* __restrict__ a, double4_32a* __restrict__ b, size_t n) {
  for (size_t i=blockIdx.x*(size_t)blockDim.x+threadIdx.x;i<n;i+=(size_t)gridDim.x*blockDim.x) b[i]=a[i];
}

template<typename F, typename A>
int run(const char* name, F kern, A arg, int blocks, int threads, double ops_per_thread_iter, int nsm) {
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  kern<<<blocks,threads>>>(arg); CK(cudaDeviceSynchronize());
  cudaEventRecord(e0); kern<<<blocks,threads>>>(arg); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
  float ms; cudaEventElapsedTime(&ms,e0,e1);
  static unsigned long long cyc[4096]; CK(cudaMemcpyFromSymbol(cyc,g_cyc,sizeof(unsigned long long)*blocks));
  double mc=0; for(int i=0;i<blocks;i++) mc+=cyc[i]; mc/=blocks;
  double total_ops = (double)blocks*threads*ITER*ops_per_thread_iter;
  double per_sm_cycle = total_ops / nsm / mc;   // assumes all blocks co-resident
  printf("%-8s  %8.3f ms  %10.3f Gop/s   %7.2f op/SM/clk (cycles/block %.0f)\n", name, ms, total_ops/ms/1e6, per_sm_cycle, mc);
  return 0;
}
int main(){
  cudaDeviceProp p; CK(cudaGetDeviceProperties(&p,0));
  int nsm=p.multiProcessorCount;
  int clk=0, memclk=0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0); cudaDeviceGetAttribute(&memclk, cudaDevAttrMemoryClockRate, 0);
  printf("%s sm_%d%d SMs=%d L2=%d B smemPerBlockOptin=%zu clk=%d kHz memclk=%d kHz totalMem=%.1f GB\n", p.name, p.major,p.minor,nsm,p.l2CacheSize,p.sharedMemPerBlockOptin, clk, memclk, p.totalGlobalMem/1e9);
  size_t fr,to; cudaMemGetInfo(&fr,&to); printf("free %.1f GB of %.1f GB\n", fr/1e9,to/1e9);
  int B=nsm*4, T=256;
  run("dfma", k_dfma, 1.0, B, T, 8, nsm);
  run("dadd", k_dadd, 1.0, B, T, 8, nsm);
  run("ffma", k_ffma, 1.0f, B, T, 8, nsm);
  run("ffma2", k_ffma2, 1.0f, B, T, 8, nsm);
  run("imad", k_imad, 1, B, T, 8, nsm);
  run("iadd/lop", k_iadd3, 1, B, T, 16, nsm);
  run("cvt64-32", k_cvt, 1.0, B, T, 16, nsm);
  run("rsqrt", k_rsq, 1.0f, B, T, 8, nsm);
  run("lds128", k_lds128, 1, B, T, 8, nsm);
  run("lds32", k_lds32, 1, B, T, 8, nsm);
  // HBM copy 2 GiB each way
  size_t n = (size_t)1<<26; double4_32a *a,*b; CK(cudaMalloc(&a,n*32)); CK(cudaMalloc(&b,n*32));
  cudaMemset(a,0,n*32); cudaMemset(b,0,n*32);
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  k_copy<<<nsm*8,512>>>(a,b,n); CK(cudaDeviceSynchronize());
  float best=1e9; for(int r=0;r<5;r++){cudaEventRecord(e0); k_copy<<<nsm*8,512>>>(a,b,n); cudaEventRecord(e1); cudaEventSynchronize(e1); float ms; cudaEventElapsedTime(&ms,e0,e1); if(ms<best)best=ms;}
  printf("copy 2x%.2f GB: %.3f ms -> %.1f GB/s\n", n*32/1e9, best, 2.0*n*32/best/1e6);
  cudaFree(a); cudaFree(b);
  return 0;
}
