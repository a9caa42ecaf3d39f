// ch_peak.cu -- ch_fma_peak: fused multiply-add throughput of this GPU's FP64 or FP32 pipe.
//
// The roofline of the FP64 path is its FP64 pipe (GB300 issues 2 DFMA per SM per clock),
// and the on-chip FP32 kernels are bound by instruction issue rather than by HBM; their
// fractions are stated against this measured rate instead of a nominal one.  Every thread
// runs kChains independent FMA chains x <- x m + c (m just below 1, so the values stay
// near c / (1 - m) and never overflow or turn subnormal), which keeps the pipe busy with
// no memory traffic; the result is written only if it takes a value it cannot take, so the
// compiler keeps every FMA.
#include <cstdint>

#include <cuda_runtime.h>

#include "ch.h"

namespace chk {
void record_error(const char* msg);  // ch_api.cu
}

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(1024) fma_peak_kernel(int64_t iters, double* sink) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
  const T m = T(0.999999), c = T(1e-6);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], m, c);
    }
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == T(-1)) sink[0] = (double)s;  // never true: keeps the chains live
}

}  // namespace

extern "C" int ch_fma_peak(int precision, int blocks, int threads, int64_t iters, double* sink, void* stream,
                           double* flops) {
  if (blocks < 1 || threads < 32 || threads > 1024 || threads % 32 || iters < 1 || !sink || !flops) {
    chk::record_error("ch_fma_peak: bad launch shape, iteration count or NULL pointer");
    return CH_EINVAL;
  }
  if (precision != CH_FP64 && precision != CH_FP32) {
    chk::record_error("ch_fma_peak: precision must be CH_FP64 or CH_FP32");
    return CH_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (precision == CH_FP64)
    fma_peak_kernel<double><<<blocks, threads, 0, st>>>(iters, sink);
  else
    fma_peak_kernel<float><<<blocks, threads, 0, st>>>(iters, sink);
  if (cudaPeekAtLastError() != cudaSuccess) {
    chk::record_error("ch_fma_peak: launch failed");
    return CH_ECUDA;
  }
  *flops = 2.0 * kChains * 16.0 * (double)iters * (double)threads * (double)blocks;
  return CH_OK;
}
