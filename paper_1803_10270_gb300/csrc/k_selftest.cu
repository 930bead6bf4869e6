// Diagnostic entry point: evaluates the FP64 reciprocal and reciprocal-square-root helpers of
// common.cuh (FP32 seed plus a truncated series correction) beside CUDA's own 1.0 / x and
// rsqrt(x), so a test can measure their error in units in the last place.
#include "common.cuh"

namespace {

__global__ void fastmath_kernel(const double* __restrict__ x, double* __restrict__ out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double v = x[i];
    out[4 * (long long)i + 0] = htg_rcp_fast(v);
    out[4 * (long long)i + 1] = 1.0 / v;
    out[4 * (long long)i + 2] = htg_rsqrt_fast(v);
    out[4 * (long long)i + 3] = rsqrt(v);
  }
}

}  // namespace

extern "C" int ht_selftest_fastmath(const double* x_dev, double* out_dev, int n, void* stream) {
  if (n < 0 || (n > 0 && (!x_dev || !out_dev))) return HT_ERR_ARG;
  if (n == 0) return HT_OK;
  const int threads = 256, blocks = htg_min(htg_cdiv(n, threads), 1024);
  fastmath_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(x_dev, out_dev, n);
  return cudaGetLastError() == cudaSuccess ? HT_OK : HT_ERR_CUDA;
}
