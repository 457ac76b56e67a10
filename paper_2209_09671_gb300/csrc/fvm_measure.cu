// Measurement aid: the fused multiply-add throughput of this GPU in double
// and in float, for the rooflines of kernels bound by arithmetic rather than
// by memory (the FP64 pressure residual, the reverse-mode flux kernels).
// Each thread runs eight independent FMA chains in registers, so the pipe,
// not the latency of one chain, sets the rate; nothing touches memory except
// one guarded store that keeps the chains alive.
#include "fvm_internal.h"

namespace fvm {
namespace {

__device__ double g_fma_sink64;
__device__ float g_fma_sink32;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T a, T b, T* sink) {
  T x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = T(threadIdx.x + q) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int q = 0; q < 8; ++q) x[q] = fma(x[q], a, b);
    }
  }
  T s = T(0);
#pragma unroll
  for (int q = 0; q < 8; ++q) s += x[q];
  if (s == T(-1234.5)) *sink = s;   // never true for these inputs; keeps the chains
}

}  // namespace
}  // namespace fvm

using namespace fvm;

extern "C" fvm_status fvm_fma_peak(int precision, void* cuda_stream, double* tflops, double* ms) {
  if (!tflops || !ms || (precision != FVM_F64 && precision != FVM_MIXED)) return FVM_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return FVM_ECUDA;
  }
  const int threads = 256, blocks = sms * 8;
  const int iters = precision == FVM_F64 ? 2048 : 32768;
  void* sink = nullptr;
  cudaError_t e = precision == FVM_F64 ? cudaGetSymbolAddress(&sink, g_fma_sink64)
                                       : cudaGetSymbolAddress(&sink, g_fma_sink32);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FVM_ECUDA;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return FVM_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return FVM_ECUDA;
  }
  float best = 0.f;
  for (int rep = 0; rep < 4; ++rep) {   // the first launch warms the clocks
    cudaEventRecord(e0, s);
    if (precision == FVM_F64)
      k_fma_chains<double><<<blocks, threads, 0, s>>>(iters, 0.999999, 1e-7, (double*)sink);
    else
      k_fma_chains<float><<<blocks, threads, 0, s>>>(iters, 0.9999f, 1e-5f, (float*)sink);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (rep > 0 && (best == 0.f || t < best)) best = t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess || best <= 0.f) return FVM_ECUDA;
  const double flops = 2.0 * 8.0 * 4.0 * (double)iters * (double)threads * (double)blocks;
  *ms = best;
  *tflops = flops / (best * 1e-3) / 1e12;
  return FVM_OK;
}
