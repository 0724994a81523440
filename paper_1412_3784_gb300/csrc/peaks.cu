// peaks.cu -- the library's own peak microbenchmarks: FP32 FMA issue rate
// (scalar and paired f32x2), FP64 FMA rate and device-to-device copy
// bandwidth.  Used to state the denominators of the roofline next to the
// measured copy / GEMM peaks.  Every kernel is a bounded loop.
#include <stdio.h>

#include "nemd_internal.cuh"

namespace {

constexpr int kChains = 8;

__global__ void k_ffma(float *out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) x[k] = threadIdx.x * 1e-3f + k;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}

__global__ void k_ffma2(float *out, int iters, float a, float b) {
  unsigned long long x[kChains];
  const unsigned long long A = pack2(a, a), B = pack2(b, b);
#pragma unroll
  for (int k = 0; k < kChains; k++) x[k] = pack2(threadIdx.x * 1e-3f + k, k * 0.5f);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < kChains; k++) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[k]) : "l"(A), "l"(B));
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; k++) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[k]));
    s += lo + hi;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dfma(double *out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) x[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_copy(const float4 *__restrict__ a, float4 *__restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

template <class F>
float time_ms(F launch, int reps) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  launch();  // warm-up
  cudaEventRecord(e0);
  for (int r = 0; r < reps; r++) launch();
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / reps;
}

}  // namespace

extern "C" int nemd_measure_peaks(int device, double *out) {
  if (!out) return NEMD_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return NEMD_ERR_CUDA;
  int sms = 0, clk = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, device);
  const int threads = 256, blocks = sms * 8, iters = 4096;
  float *fo = nullptr;
  double *dout = nullptr;
  if (cudaMalloc(&fo, sizeof(float) * threads * blocks) != cudaSuccess ||
      cudaMalloc(&dout, sizeof(double) * threads * blocks) != cudaSuccess) {
    cudaFree(fo);
    return NEMD_ERR_NOMEM;
  }
  const double lanes = (double)threads * blocks * kChains * iters;
  float ms = time_ms([&] { k_ffma<<<blocks, threads>>>(fo, iters, 0.999f, 1e-3f); }, 5);
  out[0] = lanes / (ms * 1e-3);
  ms = time_ms([&] { k_ffma2<<<blocks, threads>>>(fo, iters, 0.999f, 1e-3f); }, 5);
  out[1] = 2.0 * lanes / (ms * 1e-3);
  const int diters = 256;
  ms = time_ms([&] { k_dfma<<<blocks, threads>>>(dout, diters, 0.999, 1e-3); }, 3);
  out[2] = (double)threads * blocks * kChains * diters / (ms * 1e-3);
  const size_t nbytes = (size_t)1 << 30;
  float4 *a = nullptr, *b = nullptr;
  out[3] = 0.0;
  if (cudaMalloc(&a, nbytes) == cudaSuccess && cudaMalloc(&b, nbytes) == cudaSuccess) {
    cudaMemset(a, 0, nbytes);
    const size_t n4 = nbytes / sizeof(float4);
    ms = time_ms([&] { k_copy<<<sms * 16, 512>>>(a, b, n4); }, 10);
    out[3] = 2.0 * nbytes / (ms * 1e-3);
  }
  cudaGetLastError();
  if (a) cudaFree(a);
  if (b) cudaFree(b);
  cudaFree(fo);
  cudaFree(dout);
  out[4] = sms;
  out[5] = clk;
  return cudaGetLastError() == cudaSuccess ? NEMD_OK : NEMD_ERR_CUDA;
}
