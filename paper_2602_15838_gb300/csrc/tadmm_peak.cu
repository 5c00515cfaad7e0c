// FMA throughput probe: the measured FP64 / FP32 arithmetic roof against which
// the solver's kernels (FP64-pipe bound, no tensor cores) are rated.  Every
// thread runs kChains independent fused multiply-add chains held in
// registers; the grid fills every SM with `blocks_per_sm` CTAs of 256 threads.
// The chains' final values are summed and compared with a value they cannot
// reach (they stay in [0, 8]), with a store to a device variable behind the
// comparison, so that the compiler keeps the work.
#include <cuda_runtime.h>

#include "tadmm_impl.h"

namespace tadmm {

constexpr int kChains = 8;

__device__ double g_probe_sink;

template <typename F>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, F mul, F add) {
  F v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = F(threadIdx.x + c) * F(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], mul, add);
  }
  F acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += v[c];
  if (acc == F(-12345.0)) g_probe_sink = double(acc);
}

}  // namespace tadmm

extern "C" int tadmm_fma_probe(int32_t precision, int32_t iters, int32_t blocks_per_sm, double* flops, void* stream) {
  using tadmm::set_error;
  if (precision != 64 && precision != 32) return set_error(TADMM_EINVAL, "precision must be 64 or 32");
  if (iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 8) return set_error(TADMM_EINVAL, "need iters >= 1, 1 <= blocks_per_sm <= 8");
  int dev = 0, sms = 0;
  int rc = tadmm::cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (!rc) rc = tadmm::cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  if (rc) return rc;
  const int grid = sms * blocks_per_sm;
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == 64)
    tadmm::k_fma_probe<double><<<grid, 256, 0, st>>>(iters, 0.999999999, 1e-9);
  else
    tadmm::k_fma_probe<float><<<grid, 256, 0, st>>>(iters, 0.9999999f, 1e-7f);
  if (flops) *flops = 2.0 * tadmm::kChains * (double)iters * 256.0 * grid;
  return tadmm::cuda_check(cudaGetLastError(), "fma probe launch");
}
