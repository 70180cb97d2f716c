// FP64 throughput probe: the denominator of the ALU roofline that the solve
// and recombination kernels are measured against.  Every thread runs eight
// independent fused multiply-add chains (enough instruction-level parallelism
// to cover the FMA latency); the grid fills every SM several times over.  The
// only memory access is one store that the chains' values never trigger, so
// the timing is of the FP64 pipe alone.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/matex.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeIters = 2048;

__global__ void __launch_bounds__(kProbeThreads)
fp64_fma_probe(double mul, double add, double* __restrict__ sink) {
  double a0 = threadIdx.x * 1e-3, a1 = a0 + 0.1, a2 = a0 + 0.2, a3 = a0 + 0.3;
  double a4 = a0 + 0.4, a5 = a0 + 0.5, a6 = a0 + 0.6, a7 = a0 + 0.7;
#pragma unroll 4
  for (int i = 0; i < kProbeIters; ++i) {
    a0 = fma(a0, mul, add);
    a1 = fma(a1, mul, add);
    a2 = fma(a2, mul, add);
    a3 = fma(a3, mul, add);
    a4 = fma(a4, mul, add);
    a5 = fma(a5, mul, add);
    a6 = fma(a6, mul, add);
    a7 = fma(a7, mul, add);
  }
  const double s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
  if (s == -1.0) sink[0] = s;  // the chains stay positive: never taken
}

}  // namespace

extern "C" matex_status matex_measure_fp64_peak(int32_t reps, double* tflops, double* ms) {
  if (!tflops || reps <= 0) return MATEX_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return MATEX_ERR_CUDA;
  }
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&sink, sizeof(double)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    return MATEX_ERR_CUDA;
  }
  const int blocks = sms * 16;
  const double flops = 2.0 * 8.0 * kProbeIters * (double)blocks * kProbeThreads;
  fp64_fma_probe<<<blocks, kProbeThreads>>>(0.999999, 1e-7, sink);  // warm-up
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0);
    fp64_fma_probe<<<blocks, kProbeThreads>>>(0.999999, 1e-7, sink);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    best = std::min(best, t);
  }
  const bool ok = cudaGetLastError() == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (!ok) return MATEX_ERR_CUDA;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms) *ms = best;
  return MATEX_OK;
}
