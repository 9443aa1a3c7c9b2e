// Arithmetic-peak probes of the current device (cl_measure_peak): every thread
// runs independent multiply-add chains (or FP64 MMA chains per warp) so the
// pipe, not latency, bounds the rate.  Used as the roofline denominator of the
// FP64 front kernels, which have no vendor-measured figure on this part.
#include <cuda_runtime.h>

#include "clselinv.h"

namespace {
constexpr int kIters = 4096;

__global__ void p_dfma(double* out, double a, double b) {
  double x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = threadIdx.x * 1e-9 + j;
  for (int i = 0; i < kIters; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
  double s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void p_ffma(double* out, float a, float b) {
  float x[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) x[j] = threadIdx.x * 1e-6f + j;
  for (int i = 0; i < kIters; ++i)
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = fmaf(x[j], a, b);
  float s = 0;
#pragma unroll
  for (int j = 0; j < 16; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void p_dmma(double* out) {
  double a = 1e-3 * threadIdx.x, b = 2e-3;
  double c[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
  for (int i = 0; i < kIters / 4; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[q][0]), "+d"(c[q][1])
                   : "d"(a), "d"(b));
  double s = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) s += c[q][0] + c[q][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace

extern "C" int cl_measure_peak(int unit, double* gflops) {
  if (!gflops || unit < 0 || unit > 2) return CL_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256, n = blocks * threads;
  double* buf = nullptr;
  if (cudaMalloc(&buf, n * sizeof(double)) != cudaSuccess) return CL_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 0;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    double flops;
    if (unit == 0) {
      p_dmma<<<blocks, threads>>>(buf);
      flops = 2.0 * 8 * 8 * 4 * 4 * (kIters / 4) * (double)(n / 32);
    } else if (unit == 1) {
      p_dfma<<<blocks, threads>>>(buf, 0.999, 1e-3);
      flops = 2.0 * 8 * kIters * (double)n;
    } else {
      p_ffma<<<blocks, threads>>>(buf, 0.999f, 1e-3f);
      flops = 2.0 * 16 * kIters * (double)n;
    }
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms > 0 && flops / ms / 1e6 > best) best = flops / ms / 1e6;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (err != cudaSuccess) return CL_ERR_CUDA;
  *gflops = best;
  return CL_OK;
}
