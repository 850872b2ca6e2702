// FP64 pipe probe: the roofline denominator of the FP64-bound kernels.
//
// Every thread runs eight independent dependency chains of one FP64
// instruction kind (fused multiply-add, add or multiply) over runtime
// operands, so the compiler can neither fold nor shorten them and the FP64
// pipe, not latency, limits the rate.  The chains stay in normal range
// (multiplier 1 - 2^-30, addend 2^-40), and every thread stores its sum so
// that nothing is dead code.  The host times one launch of
// 4 x SMs CTAs x 256 threads with CUDA events after a warm-up launch.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/imex.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_fp64_probe(int iters, double a, double b, double* out) {
  double c[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) c[k] = 1.0 + (threadIdx.x + k) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      if (KIND == 0) c[k] = fma(c[k], a, b);
      else if (KIND == 1) c[k] = c[k] + b;
      else c[k] = c[k] * a;
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += c[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int imex_probe_fp64(int kind, int iters, double* lane_ops_per_s, double* seconds) {
  if (kind < 0 || kind > 2 || iters < 1 || !lane_ops_per_s) return IMEX_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IMEX_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return IMEX_ERR_CUDA;
  const int blocks = 4 * sms;
  double* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * kProbeThreads * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return IMEX_ERR_ALLOC;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const double a = 1.0 - 1.0 / (double)(1u << 30), b = 1.0 / (double)(1ull << 40);
  auto launch = [&](int n) {
    if (kind == 0) k_fp64_probe<0><<<blocks, kProbeThreads>>>(n, a, b, out);
    else if (kind == 1) k_fp64_probe<1><<<blocks, kProbeThreads>>>(n, a, b, out);
    else k_fp64_probe<2><<<blocks, kProbeThreads>>>(n, a, b, out);
    return cudaGetLastError();
  };
  float ms = 0.f;
  if (e == cudaSuccess) e = launch(iters / 8 + 1);   // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, nullptr);
  if (e == cudaSuccess) e = launch(iters);
  if (e == cudaSuccess) e = cudaEventRecord(e1, nullptr);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess || ms <= 0.f) return IMEX_ERR_CUDA;
  const double ops = (double)blocks * kProbeThreads * kChains * (double)iters;
  *lane_ops_per_s = ops / (ms * 1e-3);
  if (seconds) *seconds = ms * 1e-3;
  return IMEX_OK;
}
