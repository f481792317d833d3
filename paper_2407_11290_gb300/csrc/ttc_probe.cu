// ttc_probe.cu -- FMA-throughput loop used to measure the FP64 / FP32 pipe
// peaks that the screen's roofline fraction is reported against.
#include <cuda_runtime.h>

#include "ttcross_probe.h"

namespace {

template <class T>
__global__ void k_fma_loop(T *out, int64_t iters, T a, T b) {
  T x0 = (T)threadIdx.x, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int64_t i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  const T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
  if (s == (T)-1.2345) out[blockIdx.x] = s;  // keeps the loop alive
}

}  // namespace

extern "C" int ttcross_probe_fma_peak(int fp64, int blocks_per_sm, int64_t iters,
                                      double *fma_per_s, double *ms) {
  if (blocks_per_sm < 1 || blocks_per_sm > 32 || iters < 1 || !fma_per_s || !ms) return 1;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 6;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 6;
  const int grid = nsm * blocks_per_sm, block = 256;
  void *out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * grid) != cudaSuccess) return 6;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // warm-up, then the timed launch
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(e0);
    if (fp64)
      k_fma_loop<double><<<grid, block>>>((double *)out, iters, 0.9999999, 1e-7);
    else
      k_fma_loop<float><<<grid, block>>>((float *)out, iters, 0.9999f, 1e-4f);
    cudaEventRecord(e1);
  }
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return 6;
  *ms = t;
  *fma_per_s = (double)grid * block * 8.0 * (double)iters / (t * 1e-3);
  return 0;
}
