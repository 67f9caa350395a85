// teno_probe.cu -- FP64 throughput probe used by the benchmark to check the
// FP64 roofline denominator on the running GPU (no counterpart in the paper).
// Each thread runs 8 independent fused multiply-add chains, so the kernel is
// bound by the FP64 pipe alone; flops = 2 * 8 * iters per thread.
#include <cstdint>
#include <cuda_runtime.h>

#include "teno.h"
#include "teno_device.cuh"

namespace {

__global__ void __launch_bounds__(256) fp64_fma_chains(double* out, int64_t iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3 + k;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" teno_status teno_probe_fp64(double* out_dev, int64_t blocks, int64_t iters, void* stream) {
  if (!out_dev || blocks < 1 || blocks > (1 << 20) || iters < 1) return TENO_ERR_INVALID_ARG;
  fp64_fma_chains<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      out_dev, iters, 0.999999999, 1e-9);
  return cudaGetLastError() == cudaSuccess ? TENO_OK : TENO_ERR_CUDA;
}

namespace {

// out = [recip_pos(x) | 1.0 / x], n entries each
__global__ void __launch_bounds__(256) recip_probe(const double* __restrict__ x, double* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    out[i] = teno::recip_pos(v);
    out[n + i] = 1.0 / v;
  }
}

}  // namespace

extern "C" teno_status teno_probe_recip(const double* x_dev, double* out_dev, int64_t n, void* stream) {
  if (!x_dev || !out_dev || n < 1 || n > (int64_t(1) << 32)) return TENO_ERR_INVALID_ARG;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  recip_probe<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(x_dev, out_dev, n);
  return cudaGetLastError() == cudaSuccess ? TENO_OK : TENO_ERR_CUDA;
}
