// ttc_api.cu -- the C ABI of include/ttcross.h: argument checks, the device
// memory of an instance (one pooled allocation), and the launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ttc_internal.cuh"
#include "ttc_launch.h"
#include "ttcross.h"

using namespace ttc;

namespace {

thread_local std::string g_err;

ttc_status fail(ttc_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CU(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(e_ == cudaErrorMemoryAllocation ? TTC_ERR_OOM : TTC_ERR_CUDA,      \
                  "%s failed: %s", #call, cudaGetErrorString(e_));                   \
  } while (0)

// Two-pass carving of one device allocation: the first pass (base == nullptr)
// only measures, the second hands out 256-byte aligned pieces.
struct Carver {
  char *base = nullptr;
  size_t off = 0;
  template <class T>
  T *take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += sizeof(T) * (count ? count : 1);
    return p;
  }
};

}  // namespace

namespace ttc {
void set_last_error(const char *msg) { g_err = msg; }
}  // namespace ttc

struct ttc_handle {
  int d = 0, nb = 0;
  int64_t n[TTC_MAXD] = {};
  ttc_options opt{};
  int32_t bond_cap[TTC_MAXB] = {};
  int device = 0;
  int grid = 0;
  InstDev hi{};                 // host copy of the device descriptor
  InstDev *d_inst = nullptr;
  InstDev **d_list = nullptr;   // [1] = d_inst, for single runs
  InstDev **blist = nullptr;    // the instance list of batches led by this handle
  int64_t blist_cap = 0;
  bool captured = false;        // a run of this handle was captured in a CUDA graph:
                                // every sync reads the device (replays bypass the host)
  Ctrl *d_ctrl = nullptr;
  Barrier *d_bar = nullptr;
  int32_t *d_smid = nullptr;
  Ctrl h_ctrl{};
  void *pool = nullptr;
  size_t pool_bytes = 0;
  void *estore = nullptr;       // stored-residual form: E, ew, erow of every bond
  size_t estore_bytes = 0;
  Cand *cand = nullptr;
  int64_t cand_cap = 0;
  int64_t bond_cand_cap[TTC_MAXB] = {};
  double *core_stage = nullptr;
  int64_t core_stage_cap = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool ran = false;
  bool events_ok = false;
  // user generator: the callback, the superblock entry cache, the staging
  // buffers of the multi-indices and values handed to the callback
  ttc_user_fn user_fn = nullptr;
  void *user = nullptr;
  void *acache = nullptr;
  int32_t *ustage_idx = nullptr;
  double *ustage_val = nullptr;
  int64_t ustage_cap = 0;
  int64_t *ucounts = nullptr;   // device [TTC_MAXD + 1]
  int32_t plan_te = 0, plan_qsplit = 0;  // ttcross_set_plan
  double *rebuild_scratch = nullptr;     // ttcross_rebuild_cores: pivot rows' T
  cudaEvent_t ev2 = nullptr, ev3 = nullptr;  // around the last core rebuild
  bool rebuilt = false;
  bool synced = false;          // h_ctrl holds the finished last run
  ttc_status sync_status = TTC_OK;
  std::string sync_msg;
  std::vector<double> tt_cores;
  std::vector<int32_t> tt_ranks;
};

namespace {

__global__ void k_set_ctrl(Ctrl *dst, Ctrl v) { *dst = v; }

// a chunk of the instance list, passed by value as a kernel parameter (so
// that a captured launch keeps the pointers it was given)
constexpr int BATCH_CHUNK = 256;
struct BatchList {
  InstDev *p[BATCH_CHUNK];
};

// candidate slots of bond b for rank caps capL / capR of its neighbours:
// one per 64 x 64 tile at the caps, at least 8192 (room for the 32 x 32 tiles
// the kernels switch to when a sweep has fewer than two waves of tiles), and
// four per tile in the stored form
int64_t cand_slots(int64_t n_b, int64_t n_b1, int64_t capL, int64_t capR, int32_t pr, int32_t pc,
                   bool stored) {
  const int64_t need = std::max<int64_t>(host_tiles(n_b, n_b1, capL, capR, pr, pc), 8192);
  return stored ? 4 * need : need;
}

int64_t cand_need(const ttc_handle *h, int b, const int32_t *grid) {
  const int64_t capL = b == 0 ? 1 : h->bond_cap[b - 1];
  const int64_t capR = b == h->nb - 1 ? 1 : h->bond_cap[b + 1];
  const int32_t pr = grid ? grid[b] : 0, pc = grid ? grid[b + 1] : 0;
  return cand_slots(h->n[b], h->n[b + 1], capL, capR, pr, pc, h->hi.stored != 0);
}

// the candidate slots of a run with this grid fit the current allocation
bool cands_fit(const ttc_handle *h, const int32_t *grid) {
  if (!h->cand) return false;
  for (int b = 0; b < h->nb; ++b)
    if (cand_need(h, b, grid) > h->bond_cand_cap[b]) return false;
  return true;
}

// the stream is capturing into a CUDA graph (errors read as not capturing)
bool stream_capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
  return cs != cudaStreamCaptureStatusNone;
}

__global__ void k_set_list(InstDev **dst, BatchList src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src.p[i];
}

ttc_status ensure_cands(ttc_handle *h, const int32_t *grid) {
  int64_t need[TTC_MAXB], total = 0;
  bool grow = false;
  for (int b = 0; b < h->nb; ++b) {
    need[b] = cand_need(h, b, grid);
    if (need[b] > h->bond_cand_cap[b]) grow = true;
  }
  if (!grow && h->cand) return TTC_OK;
  for (int b = 0; b < h->nb; ++b) {
    need[b] = std::max(need[b], h->bond_cand_cap[b]);
    total += need[b];
  }
  if (h->cand) {
    CU(cudaDeviceSynchronize());
    CU(cudaFree(h->cand));
    h->cand = nullptr;
  }
  // one allocation: FP64 candidates, mixed candidates, refinement list and results
  const size_t bytes = (sizeof(Cand) + sizeof(MCand) + 2 * sizeof(int32_t) + sizeof(Cand)) *
                       (size_t)total;
  CU(cudaMalloc(&h->cand, bytes));
  // all bits set: an unwritten slot reads as row -1 with a NaN key, which the
  // merges count (ttc_stats.unscreened_slots) instead of trusting
  CU(cudaMemset(h->cand, 0xFF, bytes));
  h->cand_cap = total;
  char *base = reinterpret_cast<char *>(h->cand);
  h->hi.mcand = reinterpret_cast<MCand *>(base + sizeof(Cand) * total);
  h->hi.refine_cand = reinterpret_cast<Cand *>(base + (sizeof(Cand) + sizeof(MCand)) * total);
  h->hi.refine_list =
      reinterpret_cast<int32_t *>(base + (2 * sizeof(Cand) + sizeof(MCand)) * total);
  int64_t off = 0;
  for (int b = 0; b < h->nb; ++b) {
    h->bond_cand_cap[b] = need[b];
    h->hi.bond[b].cand_base = off;
    h->hi.bond[b].cand_cap = need[b];
    off += need[b];
  }
  h->hi.cand = h->cand;
  CU(cudaMemcpy(h->d_inst, &h->hi, sizeof(InstDev), cudaMemcpyHostToDevice));
  // the memset and the copy ran on the legacy stream, which does not order
  // against the caller's (possibly non-blocking) stream, and a pageable copy
  // may return before its DMA lands: finish both before any launch
  CU(cudaDeviceSynchronize());
  return TTC_OK;
}

ttc_status check_handle(const ttc_handle *h) {
  if (!h) return fail(TTC_ERR_INVALID_ARG, "null handle");
  return TTC_OK;
}

Ctrl make_ctrl(const ttc_handle *h, double eps, int max_rank, const int32_t *grid) {
  Ctrl c;
  std::memset(&c, 0, sizeof c);
  c.state = ST_SCREEN;
  c.status = TTC_OK;
  for (int b = 0; b < h->nb; ++b) {
    int cap = h->bond_cap[b];
    if (max_rank > 0 && max_rank < cap) cap = max_rank;
    c.maxr[b] = cap;
  }
  c.eps = eps;
  c.tau = eps;
  c.max_refine = h->opt.max_refine;
  for (int m = 0; m < h->d; ++m) c.grid[m] = grid ? grid[m] : 0;
  c.force_te = h->plan_te;
  c.qsplit = h->plan_qsplit;
  return c;
}

// user generator: room for cnt multi-indices and values in the staging buffers
ttc_status user_stage(ttc_handle *h, int64_t cnt, cudaStream_t s) {
  if (cnt <= h->ustage_cap) return TTC_OK;
  CU(cudaStreamSynchronize(s));
  const int64_t cap = std::max<int64_t>(cnt, 2 * h->ustage_cap);
  cudaFree(h->ustage_idx);
  cudaFree(h->ustage_val);
  h->ustage_idx = nullptr;
  h->ustage_val = nullptr;
  h->ustage_cap = 0;
  CU(cudaMalloc(&h->ustage_idx, sizeof(int32_t) * h->d * cap));
  CU(cudaMalloc(&h->ustage_val, sizeof(double) * cap));
  h->ustage_cap = cap;
  return TTC_OK;
}

// user generator: the entries that entered the superblocks in the last
// decision (first: every entry of the rank-one superblocks) through the
// callback into the cache, in stream order
ttc_status user_fill(ttc_handle *h, int first, cudaStream_t s) {
  CU(launch_user_count(h->d_inst, first, h->ucounts, s));
  int64_t tot = 0;
  CU(cudaMemcpyAsync(&tot, h->ucounts + h->nb, sizeof tot, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (tot == 0) return TTC_OK;
  ttc_status st = user_stage(h, tot, s);
  if (st) return st;
  CU(launch_user_gather(h->d_inst, first, h->ucounts, h->ustage_idx, s));
  h->user_fn(h->ustage_idx, tot, h->ustage_val, h->user, s);
  CU(cudaGetLastError());
  CU(launch_user_scatter(h->d_inst, first, h->ucounts, h->ustage_val, s));
  return TTC_OK;
}

// user generator: X at the error samples and at the origin into xs
ttc_status user_samples(ttc_handle *h, cudaStream_t s) {
  const int64_t cnt = h->hi.nsamples + 1;
  ttc_status st = user_stage(h, cnt, s);
  if (st) return st;
  CU(launch_user_samples(h->d_inst, h->ustage_idx, s));
  h->user_fn(h->ustage_idx, cnt, h->ustage_val, h->user, s);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(h->hi.xs, h->ustage_val, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, s));
  return TTC_OK;
}

ttc_status launch_run(ttc_handle *const *hs, int count, InstDev *const *d_list, cudaStream_t s) {
  ttc_handle *h0 = hs[0];
  RunArgs ra;
  ra.insts = d_list;
  ra.count = count;
  ra.bar = h0->d_bar;
  ra.smid = h0->d_smid;
  ra.wait_ns = (int64_t)(h0->opt.wait_limit_s * 1e9);
  const bool user = count == 1 && h0->user_fn;  // host-stepped with the callback
  ra.persistent = (h0->opt.host_loop || user) ? 0 : 1;
  ra.mixed = 0;
  ra.sampled = 0;
  ra.max_rook = 0;
  for (int i = 0; i < count; ++i)
    if (hs[i]->hi.nl > 0) {
      ra.sampled = 1;
      ra.max_rook = std::max(ra.max_rook, hs[i]->hi.max_rook);
    }
  for (int i = 0; i < count; ++i)
    if (hs[i]->hi.prec != P_FP64 && !hs[i]->hi.stored) ra.mixed = 1;  // refinement phases
  int64_t iters = 0;
  for (int i = 0; i < count; ++i) {
    int64_t s = hs[i]->opt.max_refine + 4;
    for (int b = 0; b < hs[i]->nb; ++b) s += hs[i]->bond_cap[b];
    iters = std::max(iters, s);
  }
  ra.max_iters = (int32_t)iters;
  CU(cudaMemsetAsync(h0->d_bar, 0, sizeof(Barrier), s));
  if (ra.persistent) {
    CU(launch_persistent(ra, h0->grid, s));
    return TTC_OK;
  }
  // host-stepped: the same phases as separate launches, state read per sweep
  ttc_status us;
  if (user && (us = user_samples(h0, s))) return us;
  CU(launch_phase(PH_INIT1, ra, h0->grid, s));
  CU(launch_phase(PH_INIT2, ra, h0->grid, s));
  if (user && (us = user_fill(h0, 1, s))) return us;
  CU(launch_phase(PH_INIT3, ra, h0->grid, s));
  for (int64_t it = 0; it <= ra.max_iters; ++it) {
    bool done = true;
    for (int i = 0; i < count; ++i) {
      int32_t st = 0;
      CU(cudaMemcpyAsync(&st, &hs[i]->d_ctrl->state, sizeof st, cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      if (st != ST_DONE) done = false;
    }
    if (done) return TTC_OK;
    CU(launch_phase(PH_SCREEN, ra, h0->grid, s));
    CU(launch_phase(PH_DECIDE, ra, h0->grid, s));
    if (ra.sampled) {
      // refinement rounds: a phase pair per step (no-ops once every bond is done)
      for (int k = 0; k < 2 * ra.max_rook; ++k) {
        CU(launch_phase(PH_ROOK_SCAN, ra, h0->grid, s));
        CU(launch_phase(PH_ROOK_DECIDE, ra, h0->grid, s));
      }
      CU(launch_phase(PH_FINALIZE, ra, h0->grid, s));
    }
    if (ra.mixed) {
      CU(launch_phase(PH_REFINE, ra, h0->grid, s));
      CU(launch_phase(PH_DECIDE2, ra, h0->grid, s));
    }
    if (user && (us = user_fill(h0, 0, s))) return us;
    CU(launch_phase(PH_TABLES, ra, h0->grid, s));
    CU(launch_phase(PH_UPDATE, ra, h0->grid, s));
  }
  return fail(TTC_ERR_CUDA, "host-stepped run did not finish");
}

}  // namespace

extern "C" {

ttc_status ttcross_default_options(ttc_options *opt) {
  if (!opt) return fail(TTC_ERR_INVALID_ARG, "null options");
  std::memset(opt, 0, sizeof *opt);
  opt->max_rank = 64;
  opt->bond_max_rank = nullptr;
  opt->precision = TTC_PREC_FP64;
  opt->nsamples = 1000000;
  opt->seed = 20240715ull;
  opt->max_refine = 6;
  opt->topk = 8;
  opt->host_loop = 0;
  opt->grid_ctas = 0;
  opt->wait_limit_s = 2.0;
  opt->residual = TTC_RESIDUAL_RECOMPUTE;
  opt->screen_samples = 0;
  opt->screen_seed = 20240715ull;
  opt->rook_rounds = 8;
  return TTC_OK;
}

const char *ttcross_last_error_string(void) { return g_err.c_str(); }

ttc_status ttcross_create(int d, const int64_t *n, const ttc_generator *gen, const ttc_options *opt,
                          ttc_handle **out) {
  g_err.clear();
  if (!out) return fail(TTC_ERR_INVALID_ARG, "null output handle");
  *out = nullptr;
  if (d < 2 || d > TTC_MAXD) return fail(TTC_ERR_INVALID_ARG, "d=%d outside [2,%d]", d, TTC_MAXD);
  if (!n || !gen) return fail(TTC_ERR_INVALID_ARG, "null n or generator");
  ttc_options o;
  if (opt) o = *opt; else ttcross_default_options(&o);
  if (o.max_rank < 1 || o.max_rank > RCAP)
    return fail(TTC_ERR_INVALID_ARG, "max_rank=%d outside [1,%d]", o.max_rank, RCAP);
  if (o.precision < TTC_PREC_FP64 || o.precision > TTC_PREC_AUTO)
    return fail(TTC_ERR_INVALID_ARG, "unknown precision %d", o.precision);
  if (o.topk < 1 || o.topk > 16) return fail(TTC_ERR_INVALID_ARG, "topk outside [1,16]");
  if (o.max_refine < 0) return fail(TTC_ERR_INVALID_ARG, "max_refine < 0");
  if (!(o.wait_limit_s > 0.0) || o.wait_limit_s > 600.0)
    return fail(TTC_ERR_INVALID_ARG, "wait_limit_s must be in (0, 600]");
  if (o.grid_ctas < 0 || o.grid_ctas > GRID_CAP)
    return fail(TTC_ERR_INVALID_ARG, "grid_ctas outside [0,%d]", GRID_CAP);
  if (o.residual != TTC_RESIDUAL_RECOMPUTE && o.residual != TTC_RESIDUAL_STORED)
    return fail(TTC_ERR_INVALID_ARG, "unknown residual form %d", o.residual);
  if (o.screen_samples < 0 || o.screen_samples > ((int64_t)1 << 40) || o.rook_rounds < 0 ||
      o.rook_rounds > 64)
    return fail(TTC_ERR_INVALID_ARG, "screen_samples / rook_rounds out of range");
  if (o.screen_samples > 0 &&
      (o.residual != TTC_RESIDUAL_RECOMPUTE || o.precision != TTC_PREC_FP64))
    return fail(TTC_ERR_INVALID_ARG,
                "a sampled screen needs the recompute residual form and FP64 precision");
  int64_t total = 1;
  bool overflow = false;
  int64_t hsum = 0;
  for (int m = 0; m < d; ++m) {
    if (n[m] < 1 || n[m] > (1 << 24)) return fail(TTC_ERR_INVALID_ARG, "n[%d]=%lld", m, (long long)n[m]);
    if (total > ((int64_t)1 << 62) / n[m]) overflow = true; else total *= n[m];
    hsum += n[m] - 1;
  }
  if (gen->kind == TTC_GEN_HILBERT) {
    if (hsum > (1 << 26)) return fail(TTC_ERR_INVALID_ARG, "Hilbert index sum too large");
  } else if (gen->kind == TTC_GEN_TT) {
    if (!gen->tt_ranks || !gen->tt_cores) return fail(TTC_ERR_INVALID_ARG, "TT generator without cores");
    if (gen->tt_ranks[0] != 1 || gen->tt_ranks[d] != 1)
      return fail(TTC_ERR_INVALID_ARG, "TT ranks must start and end with 1");
    for (int m = 1; m < d; ++m)
      if (gen->tt_ranks[m] < 1 || gen->tt_ranks[m] > TT_GEN_RMAX)
        return fail(TTC_ERR_INVALID_ARG, "TT generator ranks must be in [1,%d]", TT_GEN_RMAX);
  } else if (gen->kind == TTC_GEN_MAXWELLIAN) {
    if (gen->dx < 1 || gen->dv < 1 || gen->dx + gen->dv != d)
      return fail(TTC_ERR_INVALID_ARG, "Maxwellian needs dx, dv >= 1 and dx + dv = d");
    for (int m = gen->dx; m < d; ++m)
      if (n[m] < 2) return fail(TTC_ERR_INVALID_ARG, "velocity modes need n >= 2");
  } else if (gen->kind == TTC_GEN_USER) {
    if (!gen->user_fn) return fail(TTC_ERR_INVALID_ARG, "user generator without a callback");
    if (o.screen_samples > 0)
      return fail(TTC_ERR_INVALID_ARG, "a sampled screen with the user generator is not supported");
    if (o.precision != TTC_PREC_FP64 && o.residual != TTC_RESIDUAL_STORED)
      return fail(TTC_ERR_INVALID_ARG, "the user generator's mixed precision needs the stored form");
  } else if (gen->kind == TTC_GEN_MAXWELLIAN_XV) {
    if (gen->dx < 1 || gen->dv != gen->dx || 2 * gen->dx != d)
      return fail(TTC_ERR_INVALID_ARG, "the interleaved Maxwellian needs dx = dv = d / 2");
    for (int m = 0; m < d; ++m)
      if (n[m] < 2) return fail(TTC_ERR_INVALID_ARG, "its modes need n >= 2");
    if (!(std::fabs(gen->a_T) < 0.5)) return fail(TTC_ERR_INVALID_ARG, "need |a_T| < 1/2");
  } else {
    return fail(TTC_ERR_INVALID_ARG, "unknown generator kind %d", gen->kind);
  }
  if (overflow) return fail(TTC_ERR_INVALID_ARG, "more than 2^62 entries: linear index overflows");
  const bool exhaustive = o.nsamples <= 0 || (!overflow && o.nsamples >= total);
  if (exhaustive && (overflow || total > (int64_t)1 << 30))
    return fail(TTC_ERR_INVALID_ARG, "every-entry error on %s entries", overflow ? "> 2^63" : "> 2^30");
  const int64_t ns = exhaustive ? total : o.nsamples;

  ttc_handle *h = new ttc_handle();
  h->d = d;
  h->nb = d - 1;
  for (int m = 0; m < d; ++m) h->n[m] = n[m];
  h->opt = o;
  for (int b = 0; b < d - 1; ++b) {
    int cap = o.max_rank;
    if (o.bond_max_rank) {
      if (o.bond_max_rank[b] < 1 || o.bond_max_rank[b] > RCAP) {
        delete h;
        return fail(TTC_ERR_INVALID_ARG, "bond_max_rank[%d]=%d", b, o.bond_max_rank[b]);
      }
      cap = std::max(cap, (int)o.bond_max_rank[b]);
    }
    h->bond_cap[b] = cap;
  }
  for (int b = 0; b < d - 1; ++b) {
    // superblock rows / columns are 32-bit in the tile plan
    const int64_t capL = b == 0 ? 1 : h->bond_cap[b - 1];
    const int64_t capR = b == d - 2 ? 1 : h->bond_cap[b + 1];
    if (capL * n[b] >= ((int64_t)1 << 31) || capR * n[b + 1] >= ((int64_t)1 << 31)) {
      delete h;
      return fail(TTC_ERR_INVALID_ARG, "bond %d: rank cap x mode size reaches 2^31", b + 1);
    }
  }
  h->opt.bond_max_rank = nullptr;
  std::vector<int32_t> bcaps;
  if (o.bond_max_rank) bcaps.assign(o.bond_max_rank, o.bond_max_rank + d - 1);
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return fail(TTC_ERR_CUDA, "no CUDA device");
  }
  // persistent grid: one wave at full occupancy
  int bps = 0, nsm = 0;
  cudaError_t ce = persistent_occupancy(&bps);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
  if (ce != cudaSuccess || bps < 1) {
    delete h;
    return fail(TTC_ERR_CUDA, "occupancy query failed: %s", cudaGetErrorString(ce));
  }
  h->grid = std::min(bps * nsm, GRID_CAP);
  if (o.grid_ctas > 0) h->grid = std::min(h->grid, o.grid_ctas);

  // ---- device memory: one pool ----
  InstDev &I = h->hi;
  std::memset(&I, 0, sizeof I);
  I.d = d;
  I.nb = d - 1;
  int64_t st = 1;
  for (int m = 0; m < d; ++m) {
    I.n[m] = n[m];
    I.stride[m] = st;
    st = overflow ? st : st * n[m];
  }
  I.gen = gen->kind;
  // AUTO: the float-float screen; plain FP32 resolves residuals only down to
  // about 1e-7 of the largest entries, which the stop thresholds here undercut
  I.prec = o.precision == TTC_PREC_AUTO ? P_SPLIT : o.precision;
  I.topk = o.topk;
  I.nl = o.screen_samples;
  I.lseed = o.screen_seed;
  I.max_rook = o.rook_rounds;
  I.nsamples = ns;
  I.exhaustive = exhaustive ? 1 : 0;
  I.seed = o.seed;
  if (gen->kind == TTC_GEN_MAXWELLIAN || gen->kind == TTC_GEN_MAXWELLIAN_XV) {
    I.dx = gen->dx; I.dv = gen->dv;
    I.a_rho = gen->a_rho; I.a_u = gen->a_u; I.a_T = gen->a_T;
    I.vmin = gen->vmin; I.vmax = gen->vmax;
  }
  int64_t tt_total = 0;
  if (gen->kind == TTC_GEN_TT) {
    for (int m = 0; m <= d; ++m) I.rho[m] = gen->tt_ranks[m];
    for (int m = 0; m < d; ++m) {
      I.core_off[m] = tt_total;
      tt_total += (int64_t)I.rho[m] * n[m] * I.rho[m + 1];
    }
  }
  const int64_t hlen = gen->kind == TTC_GEN_HILBERT ? hsum + 1 : 1;
  int64_t ncombo = 1, ncos = 1;
  if (gen->kind == TTC_GEN_MAXWELLIAN) {
    ncos = 0;
    for (int m = 0; m < gen->dx; ++m) {
      I.mx_stride[m] = ncombo;
      I.mx_off[m] = ncos;
      ncombo *= n[m];
      ncos += n[m];
    }
    if (ncombo > ((int64_t)1 << 27)) {
      delete h;
      return fail(TTC_ERR_INVALID_ARG, "Maxwellian x grid too large (%lld index combinations)",
                  (long long)ncombo);
    }
  }
  const bool xv = gen->kind == TTC_GEN_MAXWELLIAN_XV;
  if (xv) {
    // one table per mode: position modes rho / (2 sqrt(2 pi T)) and
    // 1 / (2 T), velocity modes the grid values (and zeros)
    ncombo = 0;
    for (int m = 0; m < d; ++m) {
      I.mx_off[m] = ncombo;
      ncombo += n[m];
    }
  }
  const bool mxtab = gen->kind == TTC_GEN_MAXWELLIAN || xv;
  int64_t core_cap = 0;
  for (int pass = 0; pass < 2; ++pass) {
    Carver cv;
    cv.base = static_cast<char *>(h->pool);
    Ctrl *ctrl = cv.take<Ctrl>(1);
    Barrier *bar = cv.take<Barrier>(1);
    InstDev *dinst = cv.take<InstDev>(1);
    InstDev **dlist = cv.take<InstDev *>(1);
    double *hilb = cv.take<double>(hlen);
    double *mxc = cv.take<double>(mxtab ? ncombo : 1);
    double *mxn = cv.take<double>(mxtab ? ncombo : 1);
    double *mxcos = cv.take<double>(ncos);
    float *hilb_hi = cv.take<float>(hlen);
    float *hilb_lo = cv.take<float>(hlen);
    double *tt = cv.take<double>(tt_total);
    double *xs = cv.take<double>(ns + 1);  // + the origin (user generator)
    double *errp = cv.take<double>(GRID_CAP);
    Cand *spart = cv.take<Cand>(GRID_CAP);
    int32_t *smid = cv.take<int32_t>(GRID_CAP);
    int64_t *ucnt = cv.take<int64_t>(TTC_MAXD + 1);
    int32_t *eidx = cv.take<int32_t>(TTC_MAXD);
    int64_t *elin = cv.take<int64_t>(1);
    int32_t *esum = cv.take<int32_t>(1);
    for (int b = 0; b < d - 1; ++b) {
      BondDev &B = I.bond[b];
      const int64_t cap = h->bond_cap[b];
      const int64_t capL = b == 0 ? 1 : h->bond_cap[b - 1];
      const int64_t capR = b == d - 2 ? 1 : h->bond_cap[b + 1];
      B.cap = (int32_t)cap;
      B.ldT = capL * n[b];
      B.ldR = n[b + 1] * capR;
      B.T = cv.take<double>(cap * B.ldT);
      B.R = cv.take<double>(cap * B.ldR);
      B.U = cv.take<double>(cap * cap);
      B.hpiv = cv.take<double>(cap * cap);
      B.hc = cv.take<double>(cap * cap);
      B.delta = cv.take<double>(cap);
      B.prow = cv.take<int32_t>(cap);
      B.pcol = cv.take<int32_t>(cap);
      B.I.width = b + 1;
      B.I.idx = cv.take<int32_t>(cap * (b + 1));
      B.I.lin = cv.take<int64_t>(cap);
      B.I.sum = cv.take<int32_t>(cap);
      B.J.width = d - 1 - b;
      B.J.idx = cv.take<int32_t>(cap * (d - 1 - b));
      B.J.lin = cv.take<int64_t>(cap);
      B.J.sum = cv.take<int32_t>(cap);
      B.Thi = B.Tlo = B.Rhi = B.Rlo = nullptr;
      if (I.prec != P_FP64) {
        B.Thi = cv.take<float>(cap * B.ldT);
        B.Tlo = cv.take<float>(cap * B.ldT);
        B.Rhi = cv.take<float>(cap * B.ldR);
        B.Rlo = cv.take<float>(cap * B.ldR);
      }
      core_cap = std::max(core_cap, B.ldT * cap);
    }
    core_cap = std::max(core_cap, h->bond_cap[d - 2] * n[d - 1]);
    double *stage = cv.take<double>(core_cap);
    // prefix / suffix tables of the error check: the longest prefix (suffix)
    // with at most max(nsamples, 4096) index combinations and 128 MiB
    int64_t tl = 0, trr = 0;
    {
      const int64_t lim = std::max<int64_t>(ns, 4096), bytes = (int64_t)128 << 20;
      int64_t N = n[0];
      for (int a = 2; a < d; ++a) {
        N *= n[a - 1];
        const int64_t c = N * h->bond_cap[a - 1];
        if (N > lim || c * 8 > bytes) break;
        tl = c;
      }
      N = n[d - 1];
      for (int c = 2; c < d; ++c) {
        N *= n[d - c];
        const int64_t cc = N * h->bond_cap[d - c - 1];
        if (N > lim || cc * 8 > bytes) break;
        trr = cc;
      }
    }
    double *tabL = cv.take<double>(tl);
    double *tabR = cv.take<double>(trr);
    if (pass == 0) {
      h->pool_bytes = cv.off;
      cudaError_t e = cudaMalloc(&h->pool, h->pool_bytes);
      if (e != cudaSuccess) {
        delete h;
        return fail(e == cudaErrorMemoryAllocation ? TTC_ERR_OOM : TTC_ERR_CUDA,
                    "cudaMalloc(%zu) failed: %s", cv.off, cudaGetErrorString(e));
      }
    } else {
      h->d_ctrl = ctrl;
      h->d_bar = bar;
      h->d_smid = smid;
      h->ucounts = ucnt;
      h->d_inst = dinst;
      h->d_list = dlist;
      I.hilb = hilb;
      I.mx_coef = mxc;
      I.mx_nh = mxn;
      I.mx_cos = mxcos;
      I.hilb_hi = hilb_hi;
      I.hilb_lo = hilb_lo;
      I.tt = tt;
      I.xs = xs;
      I.err_part = errp;
      I.start_part = spart;
      I.err_part_cap = GRID_CAP;
      I.empty.idx = eidx;
      I.empty.lin = elin;
      I.empty.sum = esum;
      I.empty.width = 0;
      I.ctrl = ctrl;
      h->core_stage = stage;
      h->core_stage_cap = core_cap;
      I.tabL = tabL;
      I.tabR = tabR;
      I.tabL_cap = tl;
      I.tabR_cap = trr;
    }
  }
  auto cleanup = [&](ttc_status s) {
    cudaFree(h->pool);
    if (h->cand) cudaFree(h->cand);
    if (h->estore) cudaFree(h->estore);
    if (h->acache) cudaFree(h->acache);
    delete h;
    return s;
  };
  if (o.residual == TTC_RESIDUAL_STORED) {
    // E [ldT][ldR], ew [ldT], erow [ldR] per bond, in one allocation of its own
    // (it dominates the footprint: 8 B per superblock entry at the rank caps)
    Carver ev;
    for (int pass = 0; pass < 2; ++pass) {
      ev.base = static_cast<char *>(h->estore);
      ev.off = 0;
      for (int b = 0; b < d - 1; ++b) {
        BondDev &B = I.bond[b];
        double *E = ev.take<double>((size_t)(B.ldT * B.ldR));
        double *ew = ev.take<double>((size_t)B.ldT);
        double *er = ev.take<double>((size_t)B.ldR);
        if (pass == 1) {
          B.E = E;
          B.ew = ew;
          B.erow = er;
        }
      }
      if (pass == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && ev.off > fr)
          return cleanup(fail(TTC_ERR_OOM, "stored residuals need %zu bytes, %zu free", ev.off, fr));
        h->estore_bytes = ev.off;
        cudaError_t e = cudaMalloc(&h->estore, ev.off);
        if (e != cudaSuccess)
          return cleanup(fail(e == cudaErrorMemoryAllocation ? TTC_ERR_OOM : TTC_ERR_CUDA,
                              "cudaMalloc(%zu) of the stored residuals failed: %s", ev.off,
                              cudaGetErrorString(e)));
      }
    }
    I.stored = 1;
  }
  if (gen->kind == TTC_GEN_USER) {
    // the entries of every superblock at the rank caps, as the stored residual
    size_t bytes = 0;
    for (int b = 0; b < d - 1; ++b)
      bytes += ((size_t)(I.bond[b].ldT * I.bond[b].ldR) * 8 + 255) & ~size_t(255);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && bytes > fr)
      return cleanup(fail(TTC_ERR_OOM, "the entry cache needs %zu bytes, %zu free", bytes, fr));
    if (cudaMalloc(&h->acache, bytes) != cudaSuccess)
      return cleanup(fail(TTC_ERR_OOM, "cudaMalloc(%zu) of the entry cache failed", bytes));
    char *p = static_cast<char *>(h->acache);
    for (int b = 0; b < d - 1; ++b) {
      I.bond[b].A = reinterpret_cast<double *>(p);
      p += ((size_t)(I.bond[b].ldT * I.bond[b].ldR) * 8 + 255) & ~size_t(255);
    }
    h->user_fn = gen->user_fn;
    h->user = gen->user;
  }
  if (cudaMemset(h->pool, 0, h->pool_bytes) != cudaSuccess)
    return cleanup(fail(TTC_ERR_CUDA, "cudaMemset failed"));
  if (gen->kind == TTC_GEN_HILBERT) {
    std::vector<double> tab(hlen);
    std::vector<float> thi(hlen), tlo(hlen);
    for (int64_t s = 0; s < hlen; ++s) {
      tab[s] = 1.0 / (double)(s + 1);
      thi[s] = (float)tab[s];
      tlo[s] = (float)(tab[s] - (double)thi[s]);
    }
    if (cudaMemcpy((void *)I.hilb, tab.data(), sizeof(double) * hlen, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy((void *)I.hilb_hi, thi.data(), sizeof(float) * hlen, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy((void *)I.hilb_lo, tlo.data(), sizeof(float) * hlen, cudaMemcpyHostToDevice) !=
            cudaSuccess)
      return cleanup(fail(TTC_ERR_CUDA, "copy of the Hilbert table failed"));
  }
  if (gen->kind == TTC_GEN_TT) {
    if (cudaMemcpy((void *)I.tt, gen->tt_cores, sizeof(double) * tt_total, cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return cleanup(fail(TTC_ERR_CUDA, "copy of the TT cores failed"));
  }
  InstDev *lst[1] = {h->d_inst};
  if (cudaMemcpy(h->d_list, lst, sizeof lst, cudaMemcpyHostToDevice) != cudaSuccess)
    return cleanup(fail(TTC_ERR_CUDA, "copy of the instance list failed"));
  ttc_status s = ensure_cands(h, nullptr);
  if (s != TTC_OK) return cleanup(s);
  if (mxtab) {
    if (launch_maxwellian_tables(h->d_inst, const_cast<double *>(I.mx_coef),
                                 const_cast<double *>(I.mx_nh),
                                 const_cast<double *>(I.mx_cos)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess)
      return cleanup(fail(TTC_ERR_CUDA, "Maxwellian tables failed"));
  }
  // every setup copy above is on the legacy stream: complete them before the
  // caller launches on a stream that does not order against it
  if (cudaDeviceSynchronize() != cudaSuccess)
    return cleanup(fail(TTC_ERR_CUDA, "setup did not complete"));
  if (cudaEventCreate(&h->ev0) == cudaSuccess && cudaEventCreate(&h->ev1) == cudaSuccess)
    h->events_ok = true;
  if (!bcaps.empty()) {
    // per-bond caps become the default caps of every run
    for (int b = 0; b < d - 1; ++b) h->bond_cap[b] = std::min(h->bond_cap[b], bcaps[b]);
  }
  *out = h;
  return TTC_OK;
}

ttc_status ttcross_run(ttc_handle *h, double eps, int max_rank, const int32_t *subtensor_grid,
                       void *stream) {
  g_err.clear();
  ttc_status s = check_handle(h);
  if (s) return s;
  if (!(eps >= 0.0) || !std::isfinite(eps) || eps >= 1.0)
    return fail(TTC_ERR_INVALID_ARG, "eps=%g must be in [0,1)", eps);
  if (subtensor_grid)
    for (int m = 0; m < h->d; ++m)
      if (subtensor_grid[m] < 1 || subtensor_grid[m] > h->n[m])
        return fail(TTC_ERR_INVALID_ARG, "subtensor_grid[%d]=%d outside [1,n]", m, subtensor_grid[m]);
  int dev = -1;
  CU(cudaGetDevice(&dev));
  if (dev != h->device) return fail(TTC_ERR_INVALID_ARG, "handle lives on device %d", h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool cap = stream_capturing(st);
  if (cap) {
    // a captured run issues stream work only: the persistent kernel, and
    // buffers already sized by an earlier run with this grid
    if (h->opt.host_loop || h->user_fn)
      return fail(TTC_ERR_INVALID_ARG, "a host-stepped run cannot be captured in a graph");
    if (!cands_fit(h, subtensor_grid))
      return fail(TTC_ERR_INVALID_ARG,
                  "run once with this subtensor grid before capturing (buffers would grow)");
  }
  s = ensure_cands(h, subtensor_grid);
  if (s) return s;
  Ctrl c = make_ctrl(h, eps, max_rank, subtensor_grid);
  k_set_ctrl<<<1, 1, 0, st>>>(h->d_ctrl, c);
  CU(cudaGetLastError());
  // (a captured run records no timing events: device_ms keeps the last
  // ordinary run's time)
  if (h->events_ok && !cap) CU(cudaEventRecord(h->ev0, st));
  ttc_handle *hs[1] = {h};
  s = launch_run(hs, 1, h->d_list, st);
  if (s) return s;
  if (h->events_ok && !cap) CU(cudaEventRecord(h->ev1, st));
  h->stream = st;
  h->ran = true;
  h->synced = false;
  if (cap) h->captured = true;
  return TTC_OK;
}

ttc_status ttcross_run_batch(ttc_handle *const *hs, int count, const double *eps,
                             const int32_t *max_rank, const int32_t *const *grids, void *stream) {
  g_err.clear();
  if (!hs || count < 1 || !eps) return fail(TTC_ERR_INVALID_ARG, "bad batch arguments");
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) return fail(TTC_ERR_INVALID_ARG, "null handle %d", i);
    if (!(eps[i] >= 0.0) || eps[i] >= 1.0) return fail(TTC_ERR_INVALID_ARG, "eps[%d]", i);
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(TTC_ERR_INVALID_ARG, "handle %d repeated", i);
    if (hs[i]->device != hs[0]->device) return fail(TTC_ERR_INVALID_ARG, "handles on different devices");
    const int32_t *gi = grids ? grids[i] : nullptr;
    if (gi)
      for (int m = 0; m < hs[i]->d; ++m)
        if (gi[m] < 1 || gi[m] > hs[i]->n[m])
          return fail(TTC_ERR_INVALID_ARG, "grids[%d][%d]=%d outside [1,n]", i, m, gi[m]);
    if (hs[i]->user_fn && count >= 2)
      return fail(TTC_ERR_INVALID_ARG, "instance %d: a user generator cannot be batched", i);
    // An FP32 / float-float recompute-form batch of non-Hilbert tensors ended
    // in an illegal address on the GPU twice; its cause is not found, so that
    // combination is refused here, before anything is launched.
    if (count >= 2 && hs[i]->hi.prec != P_FP64 && !hs[i]->hi.stored &&
        hs[i]->hi.gen != TTC_GEN_HILBERT)
      return fail(TTC_ERR_INVALID_ARG,
                  "instance %d: a mixed-precision recompute-form batch supports the Hilbert "
                  "generator only (use the stored residual form or FP64)", i);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ttc_handle *h0 = hs[0];
  const bool cap = stream_capturing(st);
  if (cap) {
    if (h0->blist_cap < count)
      return fail(TTC_ERR_INVALID_ARG,
                  "run a batch of this size led by this handle once before capturing");
    for (int i = 0; i < count; ++i)
      if (!cands_fit(hs[i], grids ? grids[i] : nullptr))
        return fail(TTC_ERR_INVALID_ARG, "instance %d: run it with this grid before capturing", i);
  }
  if (h0->blist_cap < count) {
    if (h0->blist) {
      CU(cudaDeviceSynchronize());
      CU(cudaFree(h0->blist));
      h0->blist = nullptr;
      h0->blist_cap = 0;
    }
    CU(cudaMalloc((void **)&h0->blist, sizeof(InstDev *) * count));
    h0->blist_cap = count;
  }
  for (int i = 0; i < count; ++i) {
    const int32_t *gi = grids ? grids[i] : nullptr;
    ttc_status s = ensure_cands(hs[i], gi);
    if (s) return s;
    Ctrl c = make_ctrl(hs[i], eps[i], max_rank ? max_rank[i] : 0, gi);
    k_set_ctrl<<<1, 1, 0, st>>>(hs[i]->d_ctrl, c);
    CU(cudaGetLastError());
  }
  // the instance list, written by kernels whose parameters carry the pointers
  for (int i0 = 0; i0 < count; i0 += BATCH_CHUNK) {
    BatchList bl{};
    const int nc = std::min(BATCH_CHUNK, count - i0);
    for (int i = 0; i < nc; ++i) bl.p[i] = hs[i0 + i]->d_inst;
    k_set_list<<<1, 256, 0, st>>>(h0->blist + i0, bl, nc);
    CU(cudaGetLastError());
  }
  InstDev **d_list = h0->blist;
  for (int i = 0; i < count; ++i)
    if (hs[i]->events_ok && !cap) CU(cudaEventRecord(hs[i]->ev0, st));
  ttc_status s = launch_run(hs, count, d_list, st);
  // every instance keeps its own copy of the launch's barrier words (abort
  // flag, phase times) and its own events, so that it can be synchronised,
  // queried or destroyed independently of the others
  for (int i = 1; i < count && s == TTC_OK; ++i)
    if (cudaMemcpyAsync(hs[i]->d_bar, h0->d_bar, sizeof(Barrier), cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
      s = fail(TTC_ERR_CUDA, "copy of the barrier words failed");
  for (int i = 0; i < count; ++i)
    if (hs[i]->events_ok && !cap) cudaEventRecord(hs[i]->ev1, st);
  if (s) return s;
  for (int i = 0; i < count; ++i) {
    hs[i]->stream = st;
    hs[i]->ran = true;
    hs[i]->synced = false;
    if (cap) hs[i]->captured = true;
  }
  return TTC_OK;
}

static ttc_status sync_run(ttc_handle *h);

ttc_status ttcross_set_plan(ttc_handle *h, int32_t tile_edge, int32_t queue_split) {
  g_err.clear();
  ttc_status s = check_handle(h);
  if (s) return s;
  if (tile_edge != 0 && tile_edge != 32 && tile_edge != 64)
    return fail(TTC_ERR_INVALID_ARG, "tile_edge %d: 0, 32 or 64", tile_edge);
  if (queue_split < 0 || queue_split > 7)
    return fail(TTC_ERR_INVALID_ARG, "queue_split %d outside [0,7]", queue_split);
  h->plan_te = tile_edge;
  h->plan_qsplit = queue_split;
  return TTC_OK;
}

ttc_status ttcross_autotune(ttc_handle *h, double eps, int max_rank, const int32_t *subtensor_grid,
                            void *stream, int32_t *tile_edge, int32_t *queue_split,
                            double *best_ms) {
  g_err.clear();
  ttc_status s = check_handle(h);
  if (s) return s;
  if (h->user_fn) return fail(TTC_ERR_INVALID_ARG, "the user generator runs host-stepped: no plan");
  if (!h->events_ok) return fail(TTC_ERR_CUDA, "no events to time the candidates");
  // the candidates: tile edge 32 / 64, and (stored form) 2, 4 or 6 eighths of
  // the CTAs starting the screen on the fresh queue; each is run twice and
  // timed by the device events around its launch, the faster time counts
  const int32_t edges[2] = {64, 32};
  const int32_t splits_stored[3] = {4, 2, 6}, splits_other[1] = {0};
  const int32_t *splits = h->hi.stored ? splits_stored : splits_other;
  const int nsplit = h->hi.stored ? 3 : 1;
  double best = 1e300;
  int32_t be = 0, bq = 0;
  for (int e = 0; e < 2; ++e)
    for (int q = 0; q < nsplit; ++q) {
      if ((s = ttcross_set_plan(h, edges[e], splits[q]))) return s;
      double t = 1e300;
      for (int rep = 0; rep < 2; ++rep) {
        if ((s = ttcross_run(h, eps, max_rank, subtensor_grid, stream))) return s;
        s = ttcross_sync(h);
        if (s != TTC_OK && s != TTC_NOT_CONVERGED) return s;
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
        t = std::min(t, (double)ms);
      }
      if (t < best) {
        best = t;
        be = edges[e];
        bq = splits[q];
      }
    }
  if ((s = ttcross_set_plan(h, be, bq))) return s;
  if (tile_edge) *tile_edge = be;
  if (queue_split) *queue_split = bq;
  if (best_ms) *best_ms = best;
  return TTC_OK;
}

ttc_status ttcross_sync(ttc_handle *h) {
  ttc_status s = check_handle(h);
  if (s) return s;
  if (!h->ran) return fail(TTC_ERR_INVALID_ARG, "no run to wait for");
  // the first wait after a run reads its control block; later calls (every
  // getter waits) return what it found without touching the device.  A
  // handle whose run was captured in a CUDA graph reads it every time: the
  // graph's replays do not pass through here.
  if (h->synced && !h->captured) {
    if (h->sync_status != TTC_OK && h->sync_status != TTC_NOT_CONVERGED)
      return fail(h->sync_status, "%s", h->sync_msg.c_str());
    return h->sync_status;
  }
  s = sync_run(h);
  if (s != TTC_ERR_CUDA || h->h_ctrl.state == ST_DONE) {
    h->synced = true;
    h->sync_status = s;
    h->sync_msg = g_err;
  }
  return s;
}

static ttc_status sync_run(ttc_handle *h) {
  CU(cudaStreamSynchronize(h->stream));
  CU(cudaMemcpy(&h->h_ctrl, h->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
  Barrier bar;
  CU(cudaMemcpy(&bar, h->d_bar, sizeof bar, cudaMemcpyDeviceToHost));
  if (bar.abort) {
    h->h_ctrl.status = TTC_ERR_DEVICE_TIMEOUT;
    return fail(TTC_ERR_DEVICE_TIMEOUT, "a device-side wait ran past %.3g s (wait %d)",
                h->opt.wait_limit_s, bar.where);
  }
  if (bar.overrun) return fail(TTC_ERR_CUDA, "sweep cap reached before the run finished");
  if (h->h_ctrl.state != ST_DONE)
    return fail(TTC_ERR_CUDA, "run ended without finishing (state %d)", h->h_ctrl.state);
  return (ttc_status)h->h_ctrl.status;
}

static ttc_status synced(ttc_handle *h) {
  ttc_status s = ttcross_sync(h);
  if (s == TTC_OK || s == TTC_NOT_CONVERGED) return TTC_OK;
  if (s == TTC_ERR_CUDA || s == TTC_ERR_INVALID_ARG) return s;
  return TTC_OK;  // device-side failures still leave a readable state
}

ttc_status ttcross_rebuild_cores(ttc_handle *h, void *stream) {
  ttc_status s = synced(h);
  if (s) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!h->rebuild_scratch)
    CU(cudaMalloc(&h->rebuild_scratch, sizeof(double) * (size_t)h->nb * RCAP * RCAP));
  if (!h->ev2) {
    CU(cudaEventCreate(&h->ev2));
    CU(cudaEventCreate(&h->ev3));
  }
  // the factors go, so that the cores come from the pivot sets alone
  for (int b = 0; b < h->nb; ++b) {
    const BondDev &B = h->hi.bond[b];
    CU(cudaMemsetAsync(B.T, 0, sizeof(double) * B.cap * B.ldT, st));
    CU(cudaMemsetAsync(B.hc, 0, sizeof(double) * B.cap * B.cap, st));
    CU(cudaMemsetAsync(B.hpiv, 0, sizeof(double) * B.cap * B.cap, st));
    CU(cudaMemsetAsync(B.delta, 0, sizeof(double) * B.cap, st));
  }
  const BondDev &BL = h->hi.bond[h->nb - 1];
  CU(cudaMemsetAsync(BL.R, 0, sizeof(double) * BL.cap * BL.ldR, st));
  CU(cudaEventRecord(h->ev2, st));
  CU(launch_rebuild_cores(h->d_inst, h->nb, h->rebuild_scratch, h->grid, st));
  CU(cudaEventRecord(h->ev3, st));
  h->rebuilt = true;
  return TTC_OK;
}

ttc_status ttcross_get_ranks(ttc_handle *h, int64_t *sz) {
  ttc_status s = synced(h);
  if (s) return s;
  if (!sz) return fail(TTC_ERR_INVALID_ARG, "null output");
  sz[0] = 1;
  for (int b = 0; b < h->nb; ++b) sz[b + 1] = h->h_ctrl.r[b];
  sz[h->d] = 1;
  return TTC_OK;
}

ttc_status ttcross_get_cores(ttc_handle *h, int k, double *dst, int dst_is_device, void *stream) {
  ttc_status s = synced(h);
  if (s) return s;
  if (k < 1 || k > h->d || !dst) return fail(TTC_ERR_INVALID_ARG, "core k=%d", k);
  const int m = k - 1;
  const int64_t sl = m == 0 ? 1 : h->h_ctrl.r[m - 1];
  const int64_t sr = m == h->d - 1 ? 1 : h->h_ctrl.r[m];
  const int64_t cnt = sl * h->n[m] * sr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dst_is_device) {
    CU(launch_core(h->d_inst, m, dst, st));
    return TTC_OK;
  }
  if (cnt > h->core_stage_cap) return fail(TTC_ERR_INVALID_ARG, "core larger than its capacity");
  CU(launch_core(h->d_inst, m, h->core_stage, st));
  CU(cudaMemcpyAsync(dst, h->core_stage, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  return TTC_OK;
}

ttc_status ttcross_get_pivots(ttc_handle *h, int k, int32_t *Iout, int32_t *Jout) {
  ttc_status s = synced(h);
  if (s) return s;
  if (k < 1 || k > h->nb) return fail(TTC_ERR_INVALID_ARG, "bond k=%d", k);
  const int b = k - 1;
  const int64_t r = h->h_ctrl.r[b];
  if (Iout) CU(cudaMemcpy(Iout, h->hi.bond[b].I.idx, sizeof(int32_t) * r * k, cudaMemcpyDeviceToHost));
  if (Jout)
    CU(cudaMemcpy(Jout, h->hi.bond[b].J.idx, sizeof(int32_t) * r * (h->d - k), cudaMemcpyDeviceToHost));
  return TTC_OK;
}

ttc_status ttcross_get_pivot_inverse(ttc_handle *h, int k, double *U) {
  ttc_status s = synced(h);
  if (s) return s;
  if (k < 1 || k > h->nb || !U) return fail(TTC_ERR_INVALID_ARG, "bond k=%d", k);
  const BondDev &B = h->hi.bond[k - 1];
  const int64_t r = h->h_ctrl.r[k - 1];
  CU(cudaMemcpy2D(U, sizeof(double) * r, B.U, sizeof(double) * B.cap, sizeof(double) * r, r,
                  cudaMemcpyDeviceToHost));
  return TTC_OK;
}

ttc_status ttcross_get_stats(ttc_handle *h, ttc_stats *out) {
  if (!h || !out) return fail(TTC_ERR_INVALID_ARG, "null argument");
  std::memset(out, 0, sizeof *out);
  ttc_status s = ttcross_sync(h);
  const Ctrl &c = h->h_ctrl;
  out->sweeps = c.sweeps;
  out->entries_screened = c.entries;
  out->refinements = c.refinements;
  out->tiles_refined = c.tiles_refined;
  out->unscreened_slots = c.unscreened;
  out->screen_fmas = c.screen_fmas;
  out->error_fmas = c.error_fmas;
  out->tau = c.tau;
  out->x_rms = c.xrms;
  out->err = c.err;
  out->status = s;
  out->entries_fresh = c.entries_fresh;
  out->stored_bytes = c.stored_bytes;
  if (h->rebuilt && cudaEventSynchronize(h->ev3) == cudaSuccess) {
    float rms = 0.f;
    if (cudaEventElapsedTime(&rms, h->ev2, h->ev3) == cudaSuccess) out->rebuild_ms = rms;
  }
  float ms = 0.f;
  if (h->events_ok && cudaEventElapsedTime(&ms, h->ev0, h->ev1) == cudaSuccess) out->device_ms = ms;
  Barrier bar;
  if (cudaMemcpy(&bar, h->d_bar, sizeof bar, cudaMemcpyDeviceToHost) == cudaSuccess) {
    out->device_error_where = bar.where;
    for (int i = 0; i < 6; ++i) out->phase_ms[i] = bar.phase_ns[i] * 1e-6;
  }
  return TTC_OK;
}

ttc_status ttcross_check_tiles(int d, const int64_t *n, const int32_t *r, const int32_t *caps,
                               const int32_t *r_stored, const int32_t *grid, int tile_edge,
                               int stored, int64_t *tiles, int64_t *cand_cap,
                               int64_t *violations) {
  if (d < 2 || d > TTC_MAXD) return fail(TTC_ERR_INVALID_ARG, "d=%d outside [2,%d]", d, TTC_MAXD);
  if (!n || !r || !caps || !violations) return fail(TTC_ERR_INVALID_ARG, "null array");
  if (tile_edge != 32 && tile_edge != 64) return fail(TTC_ERR_INVALID_ARG, "tile_edge not 32/64");
  for (int m = 0; m < d; ++m) {
    if (n[m] < 1 || n[m] > (1 << 20)) return fail(TTC_ERR_INVALID_ARG, "n[%d] outside [1,2^20]", m);
    if (grid && (grid[m] < 0 || grid[m] > n[m]))
      return fail(TTC_ERR_INVALID_ARG, "grid[%d] outside [0,n]", m);
  }
  for (int b = 0; b < d - 1; ++b) {
    if (caps[b] < 1 || caps[b] > RCAP) return fail(TTC_ERR_INVALID_ARG, "caps[%d] outside [1,%d]", b, RCAP);
    if (r[b] < 1 || r[b] > caps[b]) return fail(TTC_ERR_INVALID_ARG, "r[%d] outside [1,cap]", b);
    if (r_stored && (r_stored[b] < 1 || r_stored[b] > r[b]))
      return fail(TTC_ERR_INVALID_ARG, "r_stored[%d] outside [1,r]", b);
  }
  for (int b = 0; b < d - 1; ++b) {
    const int64_t rl = b == 0 ? 1 : r[b - 1], rr = b == d - 2 ? 1 : r[b + 1];
    if (rl * n[b] > (1 << 24) || rr * n[b + 1] > (1 << 24))
      return fail(TTC_ERR_INVALID_ARG, "superblock of bond %d above 2^24 rows or columns", b + 1);
  }
  *violations = 0;
  for (int b = 0; b < d - 1; ++b) {
    int64_t nt = 0;
    *violations += host_check_bond_tiles(d, n, r, r_stored, grid, b, tile_edge, &nt);
    if (tiles) tiles[b] = nt;
    if (cand_cap) {
      const int64_t capL = b == 0 ? 1 : caps[b - 1], capR = b == d - 2 ? 1 : caps[b + 1];
      cand_cap[b] = cand_slots(n[b], n[b + 1], capL, capR, grid ? grid[b] : 0,
                               grid ? grid[b + 1] : 0, stored != 0);
    }
  }
  return TTC_OK;
}

ttc_status ttcross_destroy(ttc_handle *h) {
  if (!h) return TTC_OK;
  if (h->ran) cudaStreamSynchronize(h->stream);
  if (h->events_ok) {
    cudaEventDestroy(h->ev0);
    cudaEventDestroy(h->ev1);
  }
  if (h->cand) cudaFree(h->cand);
  if (h->estore) cudaFree(h->estore);
  if (h->acache) cudaFree(h->acache);
  if (h->rebuild_scratch) cudaFree(h->rebuild_scratch);
  if (h->blist) cudaFree(h->blist);
  if (h->ev2) cudaEventDestroy(h->ev2);
  if (h->ev3) cudaEventDestroy(h->ev3);
  if (h->ustage_idx) cudaFree(h->ustage_idx);
  if (h->ustage_val) cudaFree(h->ustage_val);
  if (h->pool) cudaFree(h->pool);
  delete h;
  return TTC_OK;
}

}  // extern "C"
