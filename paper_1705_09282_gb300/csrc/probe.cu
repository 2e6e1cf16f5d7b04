// Arithmetic-peak probe: the measured denominator of the roofline fractions that the
// benchmark reports for kernels bound by FP64 or FP32 multiply-add issue.  Not on the
// solver's path.
#include <cuda_runtime.h>

#include "igamg.h"

namespace {

// CH independent multiply-add chains per thread, ITERS rounds: 2 * CH * ITERS flops per
// thread.  The chains start from distinct values and the sum is stored, so nothing folds.
template <typename T, int CH>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T a, T b, T* out) {
  T x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int igamg_probe_fma(int fp64, int blocks, int iters, void* out, void* cuda_stream,
                               double* flops) {
  if (blocks <= 0 || iters <= 0 || !out) return IGAMG_EINVAL;
  constexpr int kThreads = 256, kChains = 8;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (fp64)
    k_fma_chains<double, kChains><<<blocks, kThreads, 0, s>>>(iters, 0.999999, 1e-7, (double*)out);
  else
    k_fma_chains<float, kChains><<<blocks, kThreads, 0, s>>>(iters, 0.999999f, 1e-7f, (float*)out);
  if (flops) *flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
  return cudaGetLastError() == cudaSuccess ? IGAMG_OK : IGAMG_ECUDA;
}
