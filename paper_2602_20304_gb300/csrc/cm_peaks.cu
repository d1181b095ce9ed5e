// cm_peaks.cu -- throughput probes of the two pipes the manifold kernels run on:
// FP32 fused multiply-add and the MUFU (XU) transcendental unit (ex2.approx).
// Eight independent dependency chains per thread keep both pipes issue-bound.
#include <cuda_runtime.h>

#include "contact_manifold.h"
#include "cm_math.cuh"

namespace {

__global__ void fma_probe(float* sink, int iters, float a, float b) {
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = threadIdx.x * 1e-3f + j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fmaf(x[j], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == 1234.5f) sink[threadIdx.x] = s;  // never true; keeps the chains alive
}

__global__ void ex2_probe(float* sink, int iters) {
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = -(threadIdx.x & 7) * 0.01f - j * 0.1f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = -cm::ex2(x[j]);  // stays in (-1, 0)
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == 1234.5f) sink[threadIdx.x] = s;
}

template <class F>
float time_ms(F launch) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  launch();  // warm-up
  cudaEventRecord(a);
  launch();
  cudaEventRecord(b);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms;
}

}  // namespace

extern "C" cm_status cm_measure_pipe_peaks(int device, double* fma_flops, double* mufu_ops) {
  if (!fma_flops || !mufu_ops) return CM_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return CM_ERR_CUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  float* sink = nullptr;
  if (cudaMalloc(&sink, 1024 * sizeof(float)) != cudaSuccess) return CM_ERR_OOM;
  const int threads = 512, blocks = sms * 4, iters = 4096;
  float ms_fma = time_ms([&] { fma_probe<<<blocks, threads>>>(sink, iters, 0.999f, 1e-3f); });
  float ms_ex2 = time_ms([&] { ex2_probe<<<blocks, threads>>>(sink, iters / 4); });
  cudaError_t e = cudaGetLastError();
  cudaFree(sink);
  if (e != cudaSuccess) return CM_ERR_CUDA;
  const double n = (double)blocks * threads * 8.0;
  *fma_flops = 2.0 * n * iters / (ms_fma * 1e-3);
  *mufu_ops = n * (iters / 4) / (ms_ex2 * 1e-3);
  return CM_OK;
}
