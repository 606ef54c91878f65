// daba_probe.cu -- measured fused multiply-add rates of the current GPU, the denominators of the
// roofline of the library's arithmetic-bound kernels (the FP64 path is bound by the FP64 pipe).
// Every thread runs kChains independent FMA chains for `iters` steps; the chains are summed into
// one value per thread at the end so that the compiler keeps them. Timed with CUDA events.
#include <cuda_runtime.h>

#include "../../include/daba_probe.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fma_f32(int iters, float a, float b, float* out) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = float(threadIdx.x + c);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_fma_f32x2(int iters, float a, float b, float* out) {
  float2 x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = make_float2(float(threadIdx.x + c), float(threadIdx.x - c));
  const float2 A = make_float2(a, a), B = make_float2(b, b);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], A, B);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_fma_f64(int iters, double a, double b, float* out) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = double(threadIdx.x + c);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = float(s);
}

}  // namespace

extern "C" int daba_probe_fma_rate(int kind, double* flops_per_s) {
  if (!flops_per_s || kind < 0 || kind > 2) return 1;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 2;
  }
  const int blocks = n_sm * 8;
  const int iters = kind == 2 ? 2048 : 16384;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return 3;
  }
  int rc = 0;
  float best = 1e30f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = 2;
  for (int rep = 0; rc == 0 && rep < 4; ++rep) {   // the first launch warms up; the best of the rest counts
    cudaEventRecord(e0);
    if (kind == 0) k_fma_f32<<<blocks, kThreads>>>(iters, 0.999999f, 1e-7f, out);
    if (kind == 1) k_fma_f32x2<<<blocks, kThreads>>>(iters, 0.999999f, 1e-7f, out);
    if (kind == 2) k_fma_f64<<<blocks, kThreads>>>(iters, 0.9999999999, 1e-12, out);
    cudaEventRecord(e1);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = 2;
      break;
    }
    if (rep > 0 && ms < best) best = ms;
  }
  if (rc == 0) {
    const double fma_per_thread = (double)iters * kChains * (kind == 1 ? 2 : 1);
    *flops_per_s = 2.0 * fma_per_thread * blocks * kThreads / (best * 1e-3);
  }
  cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}
