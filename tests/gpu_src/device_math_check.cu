// Test-only shim: evaluates the library's device reciprocal, WENO5 interface values (FP64 and double-float
// limiter) and double-float split on host-provided inputs.
// Built by tests/test_device_math_gpu.py with nvcc; not part of the library.
#include <cuda_runtime.h>

#include "../../paper_1608_03004_gb300/csrc/rlb_device_math.cuh"

__global__ void rcp_kernel(const double* d, double* out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = rlbdev::rcp_nr(d[i]);
}

// which = 1: wind toward increasing index, samples in memory order = wind order;
// which = 2: wind toward decreasing index, samples in memory order (interface between m1 and m2);
// which = 3, 4: the same with the double-float limiter of the FP64 stage kernel.
__global__ void weno_kernel(const double* v, double* out, int n, bool fwd, bool df) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double* w = v + 5 * i;
    out[i] = df ? rlbdev::weno5_interface_df(w[0], w[1], w[2], w[3], w[4], fwd)
                : rlbdev::weno5_interface(w[0], w[1], w[2], w[3], w[4], fwd);
  }
}

// which = 5: df_split then the two halves widened and summed in FP64 (the split's round trip)
__global__ void split_kernel(const double* v, double* out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const rlbdev::DF q = rlbdev::df_split(v[i]);
    out[i] = rlbdev::df_widen(q.hi) + rlbdev::df_widen(q.lo);
  }
}

extern "C" int dm_eval(int which, const double* in, double* out, int n) {
  double *din = nullptr, *dout = nullptr;
  const size_t nin = (size_t)n * ((which == 0 || which == 5) ? 1 : 5);
  if (cudaMalloc(&din, nin * sizeof(double)) != cudaSuccess) return 1;
  if (cudaMalloc(&dout, (size_t)n * sizeof(double)) != cudaSuccess) return 2;
  cudaMemcpy(din, in, nin * sizeof(double), cudaMemcpyHostToDevice);
  const int nb = (n + 255) / 256;
  if (which == 0)
    rcp_kernel<<<nb, 256>>>(din, dout, n);
  else if (which == 5)
    split_kernel<<<nb, 256>>>(din, dout, n);
  else
    weno_kernel<<<nb, 256>>>(din, dout, n, which == 1 || which == 3, which >= 3);
  cudaError_t e = cudaMemcpy(out, dout, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(din);
  cudaFree(dout);
  return e == cudaSuccess ? 0 : 3;
}
