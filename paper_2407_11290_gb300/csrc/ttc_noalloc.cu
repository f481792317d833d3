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
constexpr int64_t kChunk = 4096;          // samples per partial-sum slot
constexpr int kMaxChunks = 4096;          // slots -> at most 16,777,216 samples
constexpr int kMaxRank = 128;
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

__device__ double entry(const ErrArgs &a, const int32_t *idx) {
  if (a.gen == TTC_GEN_HILBERT) {
    int64_t s = 1;
    for (int m = 0; m < a.d; ++m) s += idx[m];
    return 1.0 / (double)s;
  }
  const double two_pi = 6.283185307179586476925286766559;
  double x[kMaxD];
  double prod_sin = 1.0, sum_x = 0.0;
  for (int m = 0; m < a.dx; ++m) {
    x[m] = __dmul_rn(two_pi, (double)idx[m]) / (double)a.n[m];
    prod_sin = __dmul_rn(prod_sin, sin(x[m]));
    sum_x = __dadd_rn(sum_x, x[m]);
  }
  const double rho = __dadd_rn(1.0, __dmul_rn(a.a_rho, prod_sin));
  const double T = __dadd_rn(1.0, __dmul_rn(a.a_T, cos(sum_x)));
  double q = 0.0;
  for (int j = 0; j < a.dv; ++j) {
    const int m = a.dx + j;
    const double v =
        __dadd_rn(a.vmin, __dmul_rn(__dsub_rn(a.vmax, a.vmin), (double)idx[m]) / (double)(a.n[m] - 1));
    const double u = __dmul_rn(a.a_u, cos(x[(j + 1) % a.dx]));
    const double dvu = __dsub_rn(v, u);
    q = __dadd_rn(q, __dmul_rn(dvu, dvu));
  }
  return __dmul_rn(rho / pow(__dmul_rn(two_pi, T), 0.5 * (double)a.dv), exp(-q / __dmul_rn(2.0, T)));
}

// X~(i) = G_1(i_1) ... G_d(i_d), each dot product a serial FMA chain
__device__ double tt_value(const ErrArgs &a, const int32_t *idx) {
  double v[kMaxRank], w[kMaxRank];
  int rl = a.s[1];
  for (int t = 0; t < rl; ++t) v[t] = a.core[0][(int64_t)idx[0] * rl + t];
  for (int m = 1; m < a.d; ++m) {
    const int rr = a.s[m + 1];
    const double *G = a.core[m] + (int64_t)idx[m] * rr;
    const int64_t ld = a.n[m] * rr;
    for (int u = 0; u < rr; ++u) {
      double acc = 0.0;
      for (int p = 0; p < rl; ++p) acc = __fma_rn(v[p], G[p * ld + u], acc);
      w[u] = acc;
    }
    for (int u = 0; u < rr; ++u) v[u] = w[u];
    rl = rr;
  }
  return v[0];
}

__device__ double block_sum(double v, double *red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kThreads / 32; ++i) s += red[i];
  __syncthreads();
  return s;
}

// one slot per chunk of kChunk samples: the result does not depend on the
// grid, so it is the same on any GPU
__global__ void __launch_bounds__(kThreads) k_chunk_sums(ErrArgs a, int64_t nchunks, double *sums) {
  __shared__ double red[kThreads / 32];
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int64_t k0 = c * kChunk, k1 = min(a.nsamples, k0 + kChunk);
    double num = 0.0, den = 0.0;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += kThreads) {
      int32_t idx[kMaxD];
      if (a.exhaustive) {
        int64_t l = k;
        for (int m = 0; m < a.d; ++m) {
          idx[m] = (int32_t)(l % a.n[m]);
          l /= a.n[m];
        }
      } else {
        for (int m = 0; m < a.d; ++m)
          idx[m] = (int32_t)__umul64hi(mix_at(a.seed, (uint64_t)(k * a.d + m)), (uint64_t)a.n[m]);
      }
      const double x = entry(a, idx);
      const double e = __dsub_rn(x, tt_value(a, idx));
      num = __fma_rn(e, e, num);
      den = __fma_rn(x, x, den);
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
  __shared__ double red[kThreads / 32];
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

// Device address of g_chunk_sums on the current device, looked up once per
// device (the first call on each device does it).
ttc_status scratch_on(int dev, double **out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_sums[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_chunk_sums);
    if (e != cudaSuccess || !p) return bad(TTC_ERR_CUDA, "cudaGetSymbolAddress of the scratch failed");
    g_sums[dev] = static_cast<double *>(p);
  }
  *out = g_sums[dev];
  return TTC_OK;
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
    if (s[m] < 1 || s[m] > kMaxRank) return bad(TTC_ERR_INVALID_ARG, "core size outside [1,128]");
    a.s[m] = (int32_t)s[m];
  }
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
  double *sums = nullptr;
  ttc_status st = scratch_on(dev, &sums);
  if (st != TTC_OK) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const int64_t grid = std::min<int64_t>(nchunks, (int64_t)nsm * 4);
  k_chunk_sums<<<(unsigned)grid, kThreads, 0, cs>>>(a, nchunks, sums);
  k_finish<<<1, kThreads, 0, cs>>>(sums, nchunks, err);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bad(TTC_ERR_CUDA, cudaGetErrorString(e));
  return TTC_OK;
}
