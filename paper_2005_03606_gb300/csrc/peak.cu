// Throughput probes of the arithmetic pipes the kernels of this library are
// bound by (mg_measure_peak in include/mg.h): FP32 and FP64 fused
// multiply-add, and the FP32 exponential (the special-function unit the
// lognormal fields' integration uses once per sample).  Each thread runs
// kChains independent dependency chains so that the pipe, not the latency of
// one operation, sets the rate; the grid fills every SM several times over.
#include "mg_internal.cuh"
#include "mg.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(int iters, T a, T b, T* __restrict__ out) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-12345.0) out[blockIdx.x] = s;   // keeps the chains alive; never true for these inputs
}

__global__ void __launch_bounds__(kThreads) exp_chain_kernel(int iters, float a, float* __restrict__ out) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = __expf(x[c] * a);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -12345.f) out[blockIdx.x] = s;
}

}  // namespace

extern "C" mg_status mg_measure_peak(int kind, double* ops_per_s) {
  if (!ops_per_s || kind < 0 || kind > 2) {
    mg::set_error("mg_measure_peak: bad arguments");
    return MG_ERR_INVALID;
  }
  int dev = 0, nsm = 0;
  if (!mg::cuda_ok(cudaGetDevice(&dev), "device") ||
      !mg::cuda_ok(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "attribute"))
    return MG_ERR_CUDA;
  const int blocks = nsm * 8;
  const int iters = kind == 1 ? 2048 : (kind == 2 ? 4096 : 16384);
  void* out = nullptr;
  if (!mg::cuda_ok(cudaMalloc(&out, sizeof(double) * blocks), "buffer")) return MG_ERR_CUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&]() {
    if (kind == 0) fma_chain_kernel<float><<<blocks, kThreads>>>(iters, 0.9999f, 1e-4f, (float*)out);
    else if (kind == 1) fma_chain_kernel<double><<<blocks, kThreads>>>(iters, 0.9999, 1e-4, (double*)out);
    else exp_chain_kernel<<<blocks, kThreads>>>(iters, -0.5f, (float*)out);
    mg::count_launches(1);
  };
  for (int w = 0; w < 2; ++w) launch();
  cudaEventRecord(e0);
  const int reps = 5;
  for (int r = 0; r < reps; ++r) launch();
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (!mg::cuda_ok(e, "peak probe")) return MG_ERR_CUDA;
  // operations: one FMA (two flops, counted as one operation) or one exp per chain step
  const double ops = (double)reps * blocks * kThreads * kChains * (double)iters;
  *ops_per_s = ops / (ms * 1e-3);
  return MG_OK;
}
