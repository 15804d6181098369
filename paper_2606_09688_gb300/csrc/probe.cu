// Arithmetic peak probes: sustained FP64 and FP32 fused multiply-add rates of
// the device, measured with CUDA events on the caller's stream.  They are
// the denominators of the roofline fractions of kernels bound by the FP64 or
// FP32 pipes (the combination sum, the time transforms, the FP64 stencils).
#include <cuda_runtime.h>

#include "../../include/st_probe.h"

namespace {

constexpr int kChains = 8;  // independent FMA chains per thread

// Every thread runs kChains independent chains x <- x * a + b.  With a slightly
// below one and b small the values stay bounded; the final sum is written, so
// no chain can be removed by the compiler.
template <typename R>
__global__ void __launch_bounds__(256) k_fma_probe(R* out, int iters, R a, R b) {
  R x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (R)(threadIdx.x + k) * (R)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
  }
  R s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename R>
st_status run_probe(int iters, double* gflops, cudaStream_t s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ST_ERR_CUDA;
  const int threads = 256, blocks = sms * 8;  // 2048 threads per SM
  R* out = nullptr;
  if (cudaMallocAsync(&out, sizeof(R) * (size_t)threads * blocks, s) != cudaSuccess) return ST_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const R a = (R)0.999999, b = (R)1e-6;
  k_fma_probe<R><<<blocks, threads, 0, s>>>(out, iters / 8 + 1, a, b);  // warm-up
  cudaEventRecord(e0, s);
  k_fma_probe<R><<<blocks, threads, 0, s>>>(out, iters, a, b);
  cudaEventRecord(e1, s);
  st_status st = ST_OK;
  if (cudaEventSynchronize(e1) != cudaSuccess) {
    st = ST_ERR_CUDA;
  } else {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * kChains * 16.0 * (double)iters * threads * (double)blocks;
    *gflops = flops / ((double)ms * 1e6);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, s);
  if (cudaGetLastError() != cudaSuccess) st = ST_ERR_CUDA;
  return st;
}

}  // namespace

extern "C" st_status st_probe_fma(int precision, int iters, double* gflops, void* stream) {
  if (gflops == nullptr || iters < 1 || iters > (1 << 24) || (precision != 0 && precision != 1)) return ST_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return precision == 0 ? run_probe<double>(iters, gflops, s) : run_probe<float>(iters, gflops, s);
}
