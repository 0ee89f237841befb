// FP64 fused multiply-add rate of the device: the denominator of the roofline
// of the FP64-bound kernels (the paper has no counterpart; it is a measurement).
//
// Every thread runs 8 independent dependent chains x <- x * a + b, so the FP64
// pipe, not latency, limits the rate. Work per launch: blocks x kProbeThreads
// threads x 8 chains x iters FMAs = 2 x that many flops.
#include "sp_internal.h"

namespace {

constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_dfma_probe(double* out, int iters, double a, double b) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1e-3 * (tid + k);
  for (int i = 0; i < iters; i += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[tid] = s;  // keeps the chains live
}

}  // namespace

extern "C" sp_status sp_probe_fp64_fma(double* out, int blocks, int iters, void* stream) {
  if (!out || blocks < 1 || iters < 4 || (iters & 3)) return SP_EINVAL;
  k_dfma_probe<<<blocks, kProbeThreads, 0, (cudaStream_t)stream>>>(out, iters, 0.999999999, 1e-9);
  return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}
