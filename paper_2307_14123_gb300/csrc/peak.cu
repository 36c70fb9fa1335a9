// Arithmetic-rate probes (measurement support, not part of the method): the
// FP32 and FP64 fused multiply-add rates of the CUDA cores, which bound the
// kernels of the hot path that run on them (the message contraction, the
// determinant jets).  Each thread runs kFmaChains independent dependency
// chains of FMAs, so every warp scheduler has independent instructions to
// issue; the chains' results are summed into `sink` so nothing is dropped.
#include <cuda_runtime.h>

#include "dqmc.h"

namespace {

constexpr int kFmaChains = 8;
constexpr int kFmaThreads = 256;

template <class T>
__global__ void __launch_bounds__(kFmaThreads) fma_rate_kernel(int iters, T a, T b, T* __restrict__ sink) {
  T x[kFmaChains];
#pragma unroll
  for (int c = 0; c < kFmaChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int c = 0; c < kFmaChains; ++c) x[c] = x[c] * a + b;
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kFmaChains; ++c) s += x[c];
  if (s == (T)12345.678) sink[blockIdx.x] = s;  // never true for the probe's inputs; keeps the chains live
}

}  // namespace

extern "C" dq_status dq_fma_rate_probe(int32_t kind, int32_t blocks, int32_t iters, void* sink, void* stream,
                                       double* flops) {
  if (blocks <= 0 || iters <= 0 || sink == nullptr || (kind != 0 && kind != 1)) return DQ_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (kind == 0)
    fma_rate_kernel<float><<<blocks, kFmaThreads, 0, s>>>(iters, 0.999f, 1e-4f, static_cast<float*>(sink));
  else
    fma_rate_kernel<double><<<blocks, kFmaThreads, 0, s>>>(iters, 0.999, 1e-4, static_cast<double*>(sink));
  if (cudaGetLastError() != cudaSuccess) return DQ_ERR_CUDA;
  if (flops) *flops = 2.0 * kFmaChains * 16 * (double)iters * kFmaThreads * (double)blocks;
  return DQ_OK;
}
