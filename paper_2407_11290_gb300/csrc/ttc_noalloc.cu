// ttc_noalloc.cu -- sampled relative error of a TT without any allocation.
//
// Callers that must not allocate device memory (code running inside a custom
// allocator or memory-pool callback, a pre-sized real-time or embedded
// process whose whole GPU memory budget is fixed at start-up, a plugin whose
// host forbids cudaMalloc after initialisation) can still check a TT
// against its function with ttcross_sampled_error_noalloc.  It is a variant
// of the error evaluation that ttcross_run performs: the per-chunk partial
// sums it needs live in the file-scope array below, not in memory from
// cudaMalloc.
//
// The array is a fixed 64 KiB per GPU: every device that loads the library
// holds it until the process exits.  All calls share it, and each call
// overwrites every slot it later reads, so nothing has to be cleared; but two
// calls whose kernels overlap on the GPU (different streams, or different
// host threads on one device) race on it and must be ordered by the caller.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "ttcross.h"

namespace ttc {
void set_last_error(const char *msg);  // ttc_api.cu: shared with ttcross_last_error_string
}

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int64_t kChunk = 4096;          // samples per partial-sum slot
constexpr int kMaxChunks = 4096;          // slots -> at most 16,777,216 samples
constexpr int kMaxRank = 256;             // core sizes s_m: 8 register slots per lane
constexpr int kMaxD = 16;
constexpr int kMaxDevices = 64;

// (sum (X - X~)^2, sum X^2) of every chunk of samples
static __device__ __align__(256) double g_chunk_sums[2 * kMaxChunks];

struct ErrArgs {
  int32_t d;
  int32_t gen;
  int64_t n[kMaxD];
  const double *core[kMaxD];  // core m: [s_m][n_m][s_{m+1}] row-major (device)
  int32_t s[kMaxD + 1];
  int32_t dx, dv;
  double a_rho, a_u, a_T, vmin, vmax;
  int64_t nsamples;
  int32_t exhaustive;
  uint64_t seed;
};

__device__ __forceinline__ uint64_t mix_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// index of mode m of sample k (SplitMix64 counter form, sample-major,
// mode-minor, index = floor(x n / 2^64); entry k in column-major order when
// every entry is used); computed alone, so no index array lives in memory
__device__ __forceinline__ int32_t coord(const ErrArgs &a, int64_t k, int m) {
  if (a.exhaustive) {
    int64_t l = k;
    for (int j = 0; j < m; ++j) l /= a.n[j];
    return (int32_t)(l % a.n[m]);
  }
  return (int32_t)__umul64hi(mix_at(a.seed, (uint64_t)(k * a.d + m)), (uint64_t)a.n[m]);
}

__device__ __forceinline__ double x_at(const ErrArgs &a, int64_t k, int m) {
  const double two_pi = 6.283185307179586476925286766559;
  return __dmul_rn(two_pi, (double)coord(a, k, m)) / (double)a.n[m];
}

// X at sample k: the Hilbert tensor or the Maxwellian of the generator
__device__ double entry(const ErrArgs &a, int64_t k) {
  if (a.gen == TTC_GEN_HILBERT) {
    int64_t s = 1;
    for (int m = 0; m < a.d; ++m) s += coord(a, k, m);
    return 1.0 / (double)s;
  }
  const double two_pi = 6.283185307179586476925286766559;
  double prod_sin = 1.0, sum_x = 0.0;
  for (int m = 0; m < a.dx; ++m) {
    const double x = x_at(a, k, m);
    prod_sin = __dmul_rn(prod_sin, sin(x));
    sum_x = __dadd_rn(sum_x, x);
  }
  const double rho = __dadd_rn(1.0, __dmul_rn(a.a_rho, prod_sin));
  const double T = __dadd_rn(1.0, __dmul_rn(a.a_T, cos(sum_x)));
  double q = 0.0;
  for (int j = 0; j < a.dv; ++j) {
    const int m = a.dx + j;
    const double v = __dadd_rn(
        a.vmin, __dmul_rn(__dsub_rn(a.vmax, a.vmin), (double)coord(a, k, m)) / (double)(a.n[m] - 1));
    const double u = __dmul_rn(a.a_u, cos(x_at(a, k, (j + 1) % a.dx)));
    const double dvu = __dsub_rn(v, u);
    q = __dadd_rn(q, __dmul_rn(dvu, dvu));
  }
  return __dmul_rn(rho / pow(__dmul_rn(two_pi, T), 0.5 * (double)a.dv), exp(-q / __dmul_rn(2.0, T)));
}

// X~ at sample k by one warp: X~ = G_1(i_1) ... G_d(i_d), left to right.
// Lane l keeps v[32 j + l] (j < K) in registers; each output w[u] of a core
// is the serial FMA chain over p = 0, 1, ... of v[p] G(p, i, u), v[p]
// broadcast from its lane, so the order of the operations is that of a plain
// per-sample loop and no vector lives in local memory.  Every lane returns
// the value.
template <int K>
__device__ double tt_value_warp(const ErrArgs &a, int64_t k) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  double v[K], w[K];
  int rl = a.s[1];
  {
    const double *G = a.core[0] + (int64_t)coord(a, k, 0) * rl;
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = 32 * j + lane < rl ? G[32 * j + lane] : 0.0;
  }
  for (int m = 1; m < a.d; ++m) {
    const int rr = a.s[m + 1];
    const int64_t ld = a.n[m] * rr;
    const double *G = a.core[m] + (int64_t)coord(a, k, m) * rr;
#pragma unroll
    for (int j = 0; j < K; ++j) w[j] = 0.0;
#pragma unroll
    for (int jp = 0; jp < K; ++jp) {
      if (32 * jp >= rl) break;
      const int lim = min(32, rl - 32 * jp);
      for (int l = 0; l < lim; ++l) {
        const int p = 32 * jp + l;
        const double vp = __shfl_sync(FULL, v[jp], l);
#pragma unroll
        for (int j = 0; j < K; ++j) {
          const int u = 32 * j + lane;
          if (u < rr) w[j] = __fma_rn(vp, G[p * ld + u], w[j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = w[j];
    rl = rr;
  }
  return __shfl_sync(FULL, v[0], 0);
}

__device__ double block_sum(double v, double *red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kWarps; ++i) s += red[i];
  __syncthreads();
  return s;
}

// one slot per chunk of kChunk samples (a warp per sample, warp w of the
// CTA taking samples w, w + 8, ... of the chunk): the result does not depend
// on the grid, so it is the same on any GPU
template <int K>
__global__ void __launch_bounds__(kThreads) k_chunk_sums(ErrArgs a, int64_t nchunks, double *sums) {
  __shared__ double red[kWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int64_t k0 = c * kChunk, k1 = min(a.nsamples, k0 + kChunk);
    double num = 0.0, den = 0.0;
    for (int64_t k = k0 + warp; k < k1; k += kWarps) {
      const double xt = tt_value_warp<K>(a, k);
      if (lane == 0) {
        const double x = entry(a, k);
        const double e = __dsub_rn(x, xt);
        num = __fma_rn(e, e, num);
        den = __fma_rn(x, x, den);
      }
    }
    const double sn = block_sum(num, red);
    const double sd = block_sum(den, red);
    if (threadIdx.x == 0) {
      sums[2 * c] = sn;
      sums[2 * c + 1] = sd;
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_finish(const double *sums, int64_t nchunks, double *out) {
  __shared__ double red[kWarps];
  double num = 0.0, den = 0.0;
  for (int64_t c = threadIdx.x; c < nchunks; c += kThreads) {
    num += sums[2 * c];
    den += sums[2 * c + 1];
  }
  const double sn = block_sum(num, red);
  const double sd = block_sum(den, red);
  if (threadIdx.x == 0) *out = sqrt(sn / sd);
}

ttc_status bad(ttc_status s, const char *msg) {
  ttc::set_last_error(msg);
  return s;
}

std::mutex g_mu;
double *g_sums[kMaxDevices] = {};

// Device address of g_chunk_sums on device dev (the current device).  The
// first call on a device looks it up and keeps it, so that a later call made
// while the stream is being captured needs no lookup.  Calls outside a
// capture look it up again: after cudaDeviceReset the module is loaded anew
// and the array may sit elsewhere.
ttc_status scratch_on(int dev, bool capturing, double **out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_sums[dev] || !capturing) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_chunk_sums);
    if (e != cudaSuccess || !p) {
      if (capturing) return bad(TTC_ERR_CUDA, "scratch address unknown: make a first call before capture");
      return bad(TTC_ERR_CUDA, "cudaGetSymbolAddress of the scratch failed");
    }
    g_sums[dev] = static_cast<double *>(p);
  }
  *out = g_sums[dev];
  return TTC_OK;
}

template <int K>
cudaError_t launch_sums(const ErrArgs &a, int64_t nchunks, int64_t grid, double *sums,
                        cudaStream_t cs) {
  k_chunk_sums<K><<<(unsigned)grid, kThreads, 0, cs>>>(a, nchunks, sums);
  return cudaGetLastError();
}

}  // namespace

extern "C" ttc_status ttcross_sampled_error_noalloc(int d, const int64_t *n, const ttc_generator *gen,
                                                    const double *const *cores, const int64_t *s,
                                                    int64_t nsamples, uint64_t seed, double *err,
                                                    void *stream) {
  ttc::set_last_error("");
  if (d < 2 || d > kMaxD) return bad(TTC_ERR_INVALID_ARG, "d outside [2,16]");
  if (!n || !gen || !cores || !s || !err) return bad(TTC_ERR_INVALID_ARG, "null argument");
  if (gen->kind != TTC_GEN_HILBERT && gen->kind != TTC_GEN_MAXWELLIAN)
    return bad(TTC_ERR_INVALID_ARG,
               "this entry point evaluates the Hilbert and Maxwellian generators only");
  ErrArgs a{};
  a.d = d;
  a.gen = gen->kind;
  int64_t total = 1;
  bool big = false;
  for (int m = 0; m < d; ++m) {
    if (n[m] < 1 || n[m] > (1 << 24)) return bad(TTC_ERR_INVALID_ARG, "mode size outside [1,2^24]");
    a.n[m] = n[m];
    if (total > ((int64_t)1 << 62) / n[m]) big = true; else total *= n[m];
    if (!cores[m]) return bad(TTC_ERR_INVALID_ARG, "null core pointer");
    a.core[m] = cores[m];
  }
  if (s[0] != 1 || s[d] != 1) return bad(TTC_ERR_INVALID_ARG, "core sizes must start and end with 1");
  for (int m = 0; m <= d; ++m) {
    if (s[m] < 1 || s[m] > kMaxRank) return bad(TTC_ERR_INVALID_ARG, "core size outside [1,256]");
    a.s[m] = (int32_t)s[m];
  }
  int smax = 1;
  for (int m = 0; m <= d; ++m) smax = std::max(smax, a.s[m]);
  if (gen->kind == TTC_GEN_MAXWELLIAN) {
    if (gen->dx < 1 || gen->dv < 1 || gen->dx + gen->dv != d)
      return bad(TTC_ERR_INVALID_ARG, "Maxwellian needs dx, dv >= 1 and dx + dv = d");
    for (int m = gen->dx; m < d; ++m)
      if (n[m] < 2) return bad(TTC_ERR_INVALID_ARG, "velocity modes need n >= 2");
    a.dx = gen->dx;
    a.dv = gen->dv;
    a.a_rho = gen->a_rho;
    a.a_u = gen->a_u;
    a.a_T = gen->a_T;
    a.vmin = gen->vmin;
    a.vmax = gen->vmax;
  }
  a.exhaustive = (nsamples <= 0 || (!big && nsamples >= total)) ? 1 : 0;
  a.nsamples = a.exhaustive ? total : nsamples;
  if (a.exhaustive && big) return bad(TTC_ERR_INVALID_ARG, "every-entry error on more than 2^62 entries");
  const int64_t nchunks = (a.nsamples + kChunk - 1) / kChunk;
  if (nchunks > kMaxChunks) {
    char msg[160];
    snprintf(msg, sizeof msg,
             "%lld samples exceed the static scratch of this entry point (at most %lld)",
             (long long)a.nsamples, (long long)kChunk * kMaxChunks);
    return bad(TTC_ERR_INVALID_ARG, msg);
  }
  a.seed = seed;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return bad(TTC_ERR_CUDA, "no usable current device");
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return bad(TTC_ERR_CUDA, "device query failed");
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(cs, &cap) != cudaSuccess) return bad(TTC_ERR_CUDA, "stream query failed");
  double *sums = nullptr;
  ttc_status st = scratch_on(dev, cap != cudaStreamCaptureStatusNone, &sums);
  if (st != TTC_OK) return st;
  const int64_t grid = std::min<int64_t>(nchunks, (int64_t)nsm * 4);
  cudaError_t e;
  if (smax <= 32)
    e = launch_sums<1>(a, nchunks, grid, sums, cs);
  else if (smax <= 64)
    e = launch_sums<2>(a, nchunks, grid, sums, cs);
  else if (smax <= 128)
    e = launch_sums<4>(a, nchunks, grid, sums, cs);
  else
    e = launch_sums<8>(a, nchunks, grid, sums, cs);
  if (e == cudaSuccess) {
    k_finish<<<1, kThreads, 0, cs>>>(sums, nchunks, err);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return bad(TTC_ERR_CUDA, cudaGetErrorString(e));
  return TTC_OK;
}
