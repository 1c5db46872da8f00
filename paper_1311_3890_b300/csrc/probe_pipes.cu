// Throughput probe of the pipes the pair passes use: MUFU ex2 results, FP32
// FFMA, packed FP32x2 FMA (two FMAs per instruction, counted as two) and
// int32 -> FP32 conversions per SM per clock (8 independent chains per
// thread, 8 blocks of 1024 threads per SM).  The measured MUFU rate is the denominator of the
// MUFU side of the force pass's roofline.  Build and run: python -m
// paper_1311_3890_b300.probe
#include <cstdio>
#include <cuda_runtime.h>
__global__ void k_ex2(float* out, int iters, float seed) {
  float a0 = seed + threadIdx.x * 1e-6f, a1 = a0 + 0.1f, a2 = a0 + 0.2f, a3 = a0 + 0.3f;
  float a4 = a0 + 0.4f, a5 = a0 + 0.5f, a6 = a0 + 0.6f, a7 = a0 + 0.7f;
  for (int i = 0; i < iters; ++i) {
#define E(a) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(a));
    E(a0) E(a1) E(a2) E(a3) E(a4) E(a5) E(a6) E(a7)
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}
__global__ void k_ffma(float* out, int iters, float seed) {
  float a[8];
  for (int k = 0; k < 8; ++k) a[k] = seed + k + threadIdx.x * 1e-6f;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], 0.9999f, 1e-7f);
  float s = 0; for (int k = 0; k < 8; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void k_i2f(float* out, int iters, int seed) {
  int a[8];
  for (int k = 0; k < 8; ++k) a[k] = seed + k + threadIdx.x;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) asm volatile("cvt.rn.f32.s32 %0, %0;" : "+r"(a[k]));
  int s = 0; for (int k = 0; k < 8; ++k) s ^= a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}
__global__ void k_ffma2(float* out, int iters, float seed) {
  unsigned long long a[4];
  const unsigned long long m = 0x3f7ff972u | ((unsigned long long)0x3f7ff972u << 32);  // 0.9999f x2
  const unsigned long long c = 0x33d6bf95u | ((unsigned long long)0x33d6bf95u << 32);  // 1e-7f x2
  for (int k = 0; k < 4; ++k) {
    const float lo = seed + 2 * k + threadIdx.x * 1e-6f, hi = lo + 1.f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a[k]) : "f"(lo), "f"(hi));
  }
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(m), "l"(c));
  float s = 0;
  for (int k = 0; k < 4; ++k) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[k]));
    s += lo + hi;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
int main() {
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  int clk; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  float* out; cudaMalloc(&out, sizeof(float) * sms * 8 * 1024);
  cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
  const int iters = 20000, blocks = sms * 8, threads = 1024;
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(a); k_ex2<<<blocks, threads>>>(out, iters, 0.5f); cudaEventRecord(b); cudaEventSynchronize(b);
    float ms; cudaEventElapsedTime(&ms, a, b);
    double ops = (double)blocks * threads * iters * 8;
    printf("ex2: %.3e ops/s  = %.2f per SM per clock at max clock %d MHz\n", ops / (ms * 1e-3), ops / (ms * 1e-3) / sms / (clk * 1e3), clk / 1000);
    cudaEventRecord(a); k_ffma<<<blocks, threads>>>(out, iters, 0.5f); cudaEventRecord(b); cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    printf("ffma: %.3e ops/s = %.2f per SM per clock\n", ops / (ms * 1e-3), ops / (ms * 1e-3) / sms / (clk * 1e3));
    cudaEventRecord(a); k_ffma2<<<blocks, threads>>>(out, iters, 0.5f); cudaEventRecord(b); cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    printf("ffma2: %.3e FMA/s = %.2f per SM per clock (each instruction two FMAs)\n", ops / (ms * 1e-3), ops / (ms * 1e-3) / sms / (clk * 1e3));
    cudaEventRecord(a); k_i2f<<<blocks, threads>>>(out, iters, 3); cudaEventRecord(b); cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    printf("i2f: %.3e ops/s = %.2f per SM per clock\n", ops / (ms * 1e-3), ops / (ms * 1e-3) / sms / (clk * 1e3));
  }
  printf("SMs %d\n", sms);
  return 0;
}
