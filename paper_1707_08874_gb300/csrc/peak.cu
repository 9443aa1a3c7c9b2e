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
// BF16 tensor MMA (mma.sync m16n8k16, FP32 accumulate); every chain gets its
// own operand registers so no two MMAs are identical
__global__ void p_bmma(double* out) {
  const unsigned lane = threadIdx.x & 31;
  unsigned a[4][4], b[4][2];
  float c[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
#pragma unroll
    for (int i = 0; i < 4; ++i) a[q][i] = 0x3c003c00u + lane * 7u + q * 131u + i * 17u;
    b[q][0] = 0x3b803b80u + lane * 3u + q * 11u;
    b[q][1] = 0x3b803b80u + lane * 5u + q * 13u;
#pragma unroll
    for (int i = 0; i < 4; ++i) c[q][i] = 0.f;
  }
  for (int it = 0; it < kIters / 4; ++it)
#pragma unroll
    for (int q = 0; q < 4; ++q)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};"
          : "+f"(c[q][0]), "+f"(c[q][1]), "+f"(c[q][2]), "+f"(c[q][3])
          : "r"(a[q][0]), "r"(a[q][1]), "r"(a[q][2]), "r"(a[q][3]), "r"(b[q][0]), "r"(b[q][1]));
  double s = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int i = 0; i < 4; ++i) s += c[q][i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
// INT8 tensor MMA (mma.sync m16n8k32, INT32 accumulate), distinct operands per chain
__global__ void p_imma(double* out) {
  const unsigned lane = threadIdx.x & 31;
  unsigned a[4][4], b[4][2];
  int c[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
#pragma unroll
    for (int i = 0; i < 4; ++i) a[q][i] = 0x01020304u * (lane + 1) + q * 0x01010101u + i;
    b[q][0] = 0x02030405u * (lane + 3) + q;
    b[q][1] = 0x03040506u * (lane + 5) + q;
#pragma unroll
    for (int i = 0; i < 4; ++i) c[q][i] = 0;
  }
  for (int it = 0; it < kIters / 4; ++it)
#pragma unroll
    for (int q = 0; q < 4; ++q)
      asm volatile(
          "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};"
          : "+r"(c[q][0]), "+r"(c[q][1]), "+r"(c[q][2]), "+r"(c[q][3])
          : "r"(a[q][0]), "r"(a[q][1]), "r"(a[q][2]), "r"(a[q][3]), "r"(b[q][0]), "r"(b[q][1]));
  double s = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int i = 0; i < 4; ++i) s += c[q][i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace

extern "C" int cl_measure_peak(int unit, double* gflops) {
  if (!gflops || unit < 0 || unit > 4) return CL_ERR_INVALID_ARG;
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
    } else if (unit == 2) {
      p_ffma<<<blocks, threads>>>(buf, 0.999f, 1e-3f);
      flops = 2.0 * 16 * kIters * (double)n;
    } else if (unit == 3) {
      p_bmma<<<blocks, threads>>>(buf);
      flops = 2.0 * 16 * 8 * 16 * 4 * (kIters / 4) * (double)(n / 32);
    } else {
      p_imma<<<blocks, threads>>>(buf);
      flops = 2.0 * 16 * 8 * 32 * 4 * (kIters / 4) * (double)(n / 32);
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
