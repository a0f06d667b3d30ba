// Test-only probe: FP64 fused multiply-add throughput of the GPU, the ceiling of the FP64 stage kernel.
// Built by tests/test_device_math_gpu.py with nvcc; not part of the library.
#include <cuda_runtime.h>

constexpr int CHAINS = 8;  // independent FMA chains per thread, so that latency never limits issue

__global__ void dfma_loop(double* out, int iters, double a, double b) {
  double x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = 1e-3 * (threadIdx.x + c);
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);  // contracts toward b / (1 - a) = 1
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FP64 FMAs per second over one launch of `blocks_per_sm` CTAs of 256 threads per SM, after one warm-up
// launch; *nsm receives the SM count. Returns 0 on success.
extern "C" int fp64_rate(int iters, int blocks_per_sm, double* fma_per_s, int* nsm) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 2;
  const int threads = 256, blocks = *nsm * blocks_per_sm;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * (size_t)blocks * threads) != cudaSuccess) return 3;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  dfma_loop<<<blocks, threads>>>(out, iters, 0.999999, 1e-6);
  cudaEventRecord(e0);
  dfma_loop<<<blocks, threads>>>(out, iters, 0.999999, 1e-6);
  cudaEventRecord(e1);
  int rc = cudaEventSynchronize(e1) == cudaSuccess ? 0 : 4;
  float ms = 0.f;
  if (rc == 0 && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = 5;
  if (rc == 0) *fma_per_s = (double)blocks * threads * iters * CHAINS / (ms * 1e-3);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}
