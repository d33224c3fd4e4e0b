// FP64 fused multiply-add throughput probe.
//
// The linearisation and cost kernels compute the geometry, residuals and cost in FP64
// on a part whose FP64 rate is a small fraction of its FP32 rate, so their roofline is
// the FP64 pipe.  Its denominator is measured on the part itself with this kernel:
// every thread runs eight independent chains of dependent FMAs (enough chains per
// warp to keep the pipe busy at full occupancy), with operands that keep the values
// finite, and writes one sum so that nothing is optimised away.
#include <cuda_runtime.h>

#include "gpo.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) k_fp64_fma_probe(int iters, double seed, double* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = seed + 1e-3 * (double)(t + k);
  // a <- a * m + c converges to c / (1 - m) = 1.0 and never overflows
  const double m = 0.9999999, c = 1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[t] = s;
}

}  // namespace

extern "C" gpo_status gpo_fp64_fma_probe(void* cuda_stream, int32_t n_ctas, int32_t iters, double* out) {
  if (n_ctas <= 0 || iters <= 0 || out == nullptr) return GPO_ERR_ARG;
  k_fp64_fma_probe<<<n_ctas, kProbeThreads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(iters, 0.5, out);
  return cudaGetLastError() == cudaSuccess ? GPO_OK : GPO_ERR_CUDA;
}
