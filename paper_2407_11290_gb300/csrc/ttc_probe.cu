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

// dependent FMA chains of warps < nchain on lanes < active; warps >= nchain
// load the SM's FP64 units with independent chains; thread t writes out[t]
__global__ void k_fp64_chain(double *out, long long *cyc, int64_t iters, int nchain, int active) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double a = 1.0000001 + 1e-9 * threadIdx.x, b = 1e-9;
  double acc = 0.5;
  __syncthreads();
  const long long t0 = clock64();
  if (warp < nchain) {
    if (lane < active)
      for (int64_t i = 0; i < iters; ++i) acc = fma(acc, a, b);
  } else {
    double x0 = acc, x1 = acc + 1.0, x2 = acc + 2.0, x3 = acc + 3.0;
    for (int64_t i = 0; i < iters; ++i) {
      x0 = fma(x0, a, b);
      x1 = fma(x1, a, b);
      x2 = fma(x2, a, b);
      x3 = fma(x3, a, b);
    }
    acc = (x0 + x1) + (x2 + x3);
  }
  const long long t1 = clock64();
  out[threadIdx.x] = acc;
  if (threadIdx.x == 0) *cyc = t1 - t0;
}

// K independent FMA chains per lane; thread t writes out[t]
template <int K>
__global__ void k_fp64_ilp(double *out, long long *cyc, int64_t iters) {
  const double a = 1.0000001 + 1e-9 * threadIdx.x, b = 1e-9;
  double x[K];
#pragma unroll
  for (int k = 0; k < K; ++k) x[k] = 0.5 + k;
  __syncthreads();
  const long long t0 = clock64();
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < K; ++k) x[k] = fma(x[k], a, b);
  }
  const long long t1 = clock64();
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) s += x[k];
  out[threadIdx.x] = s;
  if (threadIdx.x == 0) *cyc = t1 - t0;
}

}  // namespace

extern "C" int ttcross_probe_fp64_ilp(int warps, int chains, int64_t iters, double *cycles) {
  if (warps < 1 || warps > 32 || !(chains == 1 || chains == 2 || chains == 4 || chains == 8) ||
      iters < 1 || iters > ((int64_t)1 << 30) || !cycles)
    return 1;
  const int threads = 32 * warps;
  void *buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * threads + sizeof(long long)) != cudaSuccess) return 6;
  double *out = (double *)buf;
  long long *cyc = (long long *)(out + threads);
  for (int rep = 0; rep < 2; ++rep) {  // warm-up, then the measured launch
    if (chains == 1) k_fp64_ilp<1><<<1, threads>>>(out, cyc, iters);
    if (chains == 2) k_fp64_ilp<2><<<1, threads>>>(out, cyc, iters);
    if (chains == 4) k_fp64_ilp<4><<<1, threads>>>(out, cyc, iters);
    if (chains == 8) k_fp64_ilp<8><<<1, threads>>>(out, cyc, iters);
  }
  long long h = 0;
  cudaError_t e = cudaMemcpy(&h, cyc, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return 6;
  *cycles = (double)h / ((double)iters * chains);
  return 0;
}

extern "C" int ttcross_probe_fp64_chain(int chain_warps, int active_lanes, int busy_warps,
                                        int64_t iters, double *cycles) {
  if (chain_warps < 1 || busy_warps < 0 || chain_warps + busy_warps > 32 || active_lanes < 1 ||
      active_lanes > 32 || iters < 1 || iters > ((int64_t)1 << 30) || !cycles)
    return 1;
  const int threads = 32 * (chain_warps + busy_warps);
  void *buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * threads + sizeof(long long)) != cudaSuccess) return 6;
  double *out = (double *)buf;
  long long *cyc = (long long *)(out + threads);
  long long h = 0;
  for (int rep = 0; rep < 2; ++rep)  // warm-up, then the measured launch
    k_fp64_chain<<<1, threads>>>(out, cyc, iters, chain_warps, active_lanes);
  cudaError_t e = cudaMemcpy(&h, cyc, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return 6;
  *cycles = (double)h / (double)iters;
  return 0;
}

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
