/*
 * ttcross.h -- C ABI of the GB300 (sm_103a) adaptive tensor-train cross.
 *
 * Problem (paper: "Distributed memory parallel adaptive tensor-train cross
 * approximation", arXiv 2407.11290, Sec. 1 eq. FrobeniusNorm and Sec. 5 intro):
 * given a d-way tensor X of mode sizes n_1..n_d defined entry-wise by a
 * function (it is never formed), build TT cores G_1..G_d (Sec. 2.2) such that
 * the relative Frobenius error, estimated on random entries (Sec. 5), is at
 * most eps.
 *
 * Method (all steps run in CUDA kernels on one GPU):
 *   - every bond k = 1..d-1 screens its whole superblock
 *     X_k(I_{<=k-1} x I_k, I_{k+1} x J_{>k+1}) (Alg. 2) for the entry of
 *     largest residual |A - T_k R_k| (Alg. 1 with the sample set equal to the
 *     superblock); the paper's subtensor process grid (Sec. 3, Alg. 3) becomes
 *     a grid of CTAs, each taking a local argmax, followed by a device-side
 *     merge of the candidates (the Allgather of Alg. 3);
 *   - all bonds search simultaneously; pivots are appended with nestedness
 *     (eq. nestedpivots);
 *   - T_k = C_k P_k^{-1} is updated by eq. aca_approx_T_sub, rows entering a
 *     superblock are rebuilt by Alg. 4, and P_k^{-1} is bordered by the
 *     Sherman-Morrison step of Sec. 3.1.1, all in FP64;
 *   - cores follow eq. ttcross_build / corereshape; the sampled error is
 *     computed in FP64 on the GPU.
 *
 * Conventions
 *   - Indices are 0-based.  Bonds and cores use the paper's k: bonds
 *     1 <= k <= d-1, cores 1 <= k <= d.
 *   - The linear index used to break ties between equal residuals is the
 *     column-major one, lin = sum_m i_m prod_{l<m} n_l (Sec. 2.1 reshape).
 *   - `stream` arguments are cudaStream_t values passed as void*; NULL is the
 *     legacy default stream.
 *   - Every function returns a ttc_status; no exception crosses the ABI.
 *     On failure ttcross_last_error_string() (thread-local) describes it.
 *   - Handles own all of their device memory (allocated by ttcross_create,
 *     freed by ttcross_destroy).  Buffers passed by the caller stay owned by
 *     the caller and are not retained after the call returns.
 *   - A handle may be used by one host thread at a time.
 */
#ifndef TTCROSS_H
#define TTCROSS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TTC_OK = 0,
  TTC_ERR_INVALID_ARG = 1,   /* bad argument; nothing was launched */
  TTC_ERR_OOM = 2,           /* device allocation failed */
  TTC_ERR_ZERO_START = 3,    /* X is zero at the origin and at every error sample:
                                no start pivot (Alg. 1 line 1) */
  TTC_ERR_NONFINITE = 4,     /* a generated entry or residual was NaN/Inf */
  TTC_ERR_DEVICE_TIMEOUT = 5,/* a device-side wait ran past its limit */
  TTC_ERR_CUDA = 6,          /* a CUDA runtime call failed */
  TTC_NOT_CONVERGED = 7      /* rank caps or refinement limit reached with the
                                sampled error above eps; cores are valid */
} ttc_status;

typedef enum {
  TTC_GEN_HILBERT = 0,    /* X(i) = 1/(1 + i_1 + ... + i_d) (eq. HilbertTensor, 0-based) */
  TTC_GEN_TT = 1,         /* X given by TT cores (tests; exact recovery) */
  TTC_GEN_MAXWELLIAN = 2, /* f(x,v), see ttc_generator */
  TTC_GEN_MAXWELLIAN_XV = 3, /* the 2d2v / 3d3v distributions of Sec. 5.2
                               (eq. 2d2vFunction), modes interleaved
                               (x, v_x, y, v_y[, z, v_z]), see ttc_generator */
  TTC_GEN_USER = 4         /* entries from the caller's batch callback (Sec. 5
                               intro: the tensor is a function of its indices) */
} ttc_gen_kind;

/* Batch entry callback of TTC_GEN_USER.  It must set values[i] = X(i_1..i_d)
   with the multi-index idx[i*d + m] (0-based), for 0 <= i < count.  idx
   (int32, [count][d] row-major) and values (double, [count]) are device
   buffers owned by the library and valid until the callback's work on
   `stream` has run; `stream` is the run's stream (a cudaStream_t as void*).
   The callback enqueues its work on that stream (or finishes it before it
   returns); the library reads the values in stream order after it.  It is
   called on the host thread that called ttcross_run, between the run's
   kernels, never from device code.  user is the pointer of ttc_generator. */
typedef void (*ttc_user_fn)(const int32_t *idx, int64_t count, double *values, void *user,
                            void *stream);

/* Entry generator.  All pointers are host pointers, read during
   ttcross_create only (the data is copied to the device). */
typedef struct {
  int32_t kind; /* ttc_gen_kind */
  /* TTC_GEN_TT: ranks rho[0..d] with rho[0] = rho[d] = 1, 1 <= rho[m] <= 160
     (else TTC_ERR_INVALID_ARG), and the cores concatenated, core m laid out
     [rho_m][n_m][rho_{m+1}] row-major (doubles).  The entry is the
     left-to-right product of the core slices, each dot product a serial FMA
     chain. */
  const int32_t *tt_ranks;
  const double *tt_cores;
  /* TTC_GEN_MAXWELLIAN: modes ordered (x_0..x_{dx-1}, v_0..v_{dv-1});
     x_m = 2 pi i / n_m (periodic), v = vmin + (vmax - vmin) i / (n - 1);
     rho = 1 + a_rho prod_m sin x_m, u_j = a_u cos x_{(j+1) mod dx},
     T = 1 + a_T cos(sum_m x_m),
     f = rho (2 pi T)^{-dv/2} exp(-sum_j (v_j - u_j)^2 / (2 T)).
     TTC_GEN_MAXWELLIAN_XV (Sec. 5.2): dx = dv = D spatial dimensions, d = 2D,
     mode 2q the position s_q = -1/2 + i / (n - 1) on [-1/2, 1/2], mode 2q+1
     the velocity v_q = vmin + (vmax - vmin) i / (n - 1) (both grids include
     their end points); rho(s) = 1 + a_rho sin(2 pi s),
     T(s) = 1/2 + a_T sin(2 pi s) (need |a_T| < 1/2), shift a_u:
     f = sum_q rho(s_q) / (2 sqrt(2 pi T(s_q)))
         * (exp(-sum_q (v_q - a_u)^2 / (2 T(s_q))) + exp(-sum_q (v_q + a_u)^2 / (2 T(s_q)))).
     The paper's values: a_rho = 0.875, a_T = 0.4, a_u = 0.75, v on [-3, 3]. */
  int32_t dx, dv;
  double a_rho, a_u, a_T, vmin, vmax;
  /* TTC_GEN_USER: the callback and its pointer.  The entries are evaluated
     unfused: after every decision the library gathers the multi-indices of
     the entries that enter a superblock (and, at the start, of the error
     samples) into a device buffer, calls fn once for them, and scatters the
     values into a device cache of the superblocks (8 bytes per superblock
     entry at the rank caps, as the stored residual).  Such instances always
     run host-stepped (the phases as separate launches) and cannot be batched
     with run_batch. */
  ttc_user_fn user_fn;
  void *user;
} ttc_generator;

typedef enum {
  TTC_PREC_FP64 = 0,  /* FP64 screen; pivots bit-identical to the FP64 oracle */
  TTC_PREC_FP32 = 1,  /* FP32 screen, top-k re-scored in FP64 */
  TTC_PREC_SPLIT = 2, /* float-float (hi/lo FP32) screen, top-k re-scored in FP64 */
  TTC_PREC_AUTO = 3   /* FP32 for eps >= 1e-7 (of the entries' rms), else SPLIT */
} ttc_precision;

typedef enum {
  TTC_RESIDUAL_RECOMPUTE = 0, /* every screen forms E = A - T_k R_k afresh (Alg. 1) */
  TTC_RESIDUAL_STORED = 1     /* eq. aca_approx_E: E_k is kept in device memory and
                                 carried through each pivot's rank-one step
                                 E <- E - E(:,j*) E(i*,:) / E(i*,j*); only entries
                                 that enter a superblock are formed as A - T R.
                                 Needs 8 * rows_cap * cols_cap bytes per bond
                                 (rows_cap = cap_{k-1} n_k, cols_cap = n_{k+1}
                                 cap_{k+1}); pivots follow the stored values, so they
                                 may differ from the recompute form's at near-ties.
                                 With TTC_PREC_FP32 / SPLIT / AUTO the entries are
                                 formed and carried on the FP32 pipe as float-float
                                 pairs (the same 8 bytes), each bond's top-k
                                 candidates are re-scored in FP64, and T, R, P^-1 and
                                 the error stay FP64; where FP64 residuals tie, the
                                 pivot may be another of the tied entries. */
} ttc_residual;

typedef struct {
  int32_t max_rank;         /* rank capacity of every bond (default 64, <= 256); the
                               superblock extents cap * n must stay below 2^31 */
  const int32_t *bond_max_rank; /* nullable host array of d-1 per-bond rank caps
                               (prescribed ranks, e.g. (15,17,18,17,15)); copied */
  int32_t precision;        /* ttc_precision (default TTC_PREC_FP64) */
  int64_t nsamples;         /* error samples (default 1e6; <= 0: every entry) */
  uint64_t seed;            /* SplitMix64 seed of the error samples (default 20240715) */
  int32_t max_refine;       /* tau reductions before TTC_NOT_CONVERGED (default 6) */
  int32_t topk;             /* mixed forms: candidates re-scored in FP64 per tile (default 8) */
  int32_t host_loop;        /* 0: one persistent cooperative launch runs the whole cross
                               (default); 1: host-stepped phases (debugging) */
  int32_t grid_ctas;        /* persistent CTAs (0 = one wave at full occupancy) */
  double wait_limit_s;      /* limit of every device-side wait, seconds (default 2.0) */
  int32_t residual;         /* ttc_residual (default TTC_RESIDUAL_RECOMPUTE) */
  /* Alg. 1 with a random sample set L (Sec. 2.3) instead of the whole
     superblock, for superblocks too large to screen: screen_samples > 0
     entries of every bond's superblock are drawn per screen (with
     replacement; SplitMix64(screen_seed), sample j of bond k in screen t from
     outputs 2i and 2i+1, i = (t (d-1) + k-1) screen_samples + j, row / column
     = floor(x rows / 2^64) / floor(x' cols / 2^64)); their argmax (ties:
     lowest linear index) is refined as in the while loop of Alg. 1: the row
     moves to the argmax of the pivot's column, then the column to the argmax
     of its row, each only to a strictly larger |E|, for at most rook_rounds
     rounds or until a round moves neither.  Recompute form and FP64 only
     (else TTC_ERR_INVALID_ARG).  0 (default): the whole superblock. */
  int64_t screen_samples;
  uint64_t screen_seed;     /* default 20240715 */
  int32_t rook_rounds;      /* default 8, in [0, 64] */
} ttc_options;

typedef struct {
  int64_t sweeps;            /* residual screens (simultaneous over bonds) */
  int64_t entries_screened;  /* candidate entries screened, summed over sweeps */
  int64_t refinements;       /* tau reductions */
  int64_t tiles_refined;     /* mixed forms: screen tiles whose error bound could hide
                                the FP64 argmax and were re-screened in FP64 */
  int64_t unscreened_slots;  /* self-check: candidate slots a merge read that no screen
                                wrote in the same sweep (always 0) */
  int64_t screen_fmas;       /* algorithmic FMAs of the screens: sum over sweeps and
                                bonds of r_k * |superblock_k| */
  int64_t error_fmas;        /* algorithmic FMAs of the sampled-error evaluations */
  double tau;                /* final tau */
  double x_rms;              /* rms of X over the error samples */
  double err;                /* sampled relative Frobenius error */
  double device_ms;          /* GPU time of the last run (events around it) */
  double phase_ms[6];        /* persistent runs: GPU time per phase (init, screen,
                                decide, update, error verification, FP64 refinement) */
  int32_t status;            /* ttc_status of the last run */
  int32_t device_error_where;/* for TTC_ERR_DEVICE_TIMEOUT: the wait that gave up */
  int64_t entries_fresh;     /* screened entries formed as A - T R (all of them in the
                                recompute form; the rest were carried in storage) */
  int64_t stored_bytes;      /* stored form: bytes of E the screens read and wrote */
  double rebuild_ms;         /* GPU time of the last ttcross_rebuild_cores (0 if none) */
} ttc_stats;

typedef struct ttc_handle ttc_handle;

/* Fills *opt with the defaults listed above. */
ttc_status ttcross_default_options(ttc_options *opt);

/* Creates a TT-cross instance for a d-way tensor (2 <= d <= 16) with mode
   sizes n[0..d-1] >= 1 and the entry generator *gen.  opt may be NULL
   (defaults).  Allocates all device memory for rank capacity opt->max_rank on
   the current CUDA device.  Errors: INVALID_ARG (shape/generator/options),
   OOM, CUDA.  On success *out owns the instance. */
ttc_status ttcross_create(int d, const int64_t *n, const ttc_generator *gen,
                          const ttc_options *opt, ttc_handle **out);

/* Runs the adaptive cross to accuracy eps (Sec. 1 eq. FrobeniusNorm, error
   estimated as in Sec. 5).  Every bond starts from one pivot, the entry of
   largest |X| over the error samples and the origin (Alg. 1 line 1 with a
   zero approximation; ties to the lowest linear index), at rank 1.
   eps == 0 selects prescribed-rank mode: every bond grows to its cap.
   max_rank (<= the capacity; <= 0 means the capacity) caps every bond.
   subtensor_grid (nullable, d entries >= 1) splits every mode into that many
   pieces and makes the screen's CTA tiles follow the pieces (Sec. 3); the
   pivots do not depend on it (the global best is the best of the local bests,
   Sec. 3.2.1).  NULL lets the library choose the tiles.
   Asynchronous on `stream` unless opt->host_loop: it returns after the launch;
   ttcross_sync / the getters wait for it.  Errors detected on the host are
   returned at once; errors found on the device are reported by ttcross_sync.
   CUDA graphs: while `stream` is capturing, the call adds its work (a control
   block kernel, a memset and the persistent kernel) to the graph, so that
   replays rerun the whole cross.  It needs a persistent run (no host_loop, no
   user generator) and an earlier ordinary run with the same subtensor grid
   (a captured call allocates nothing; otherwise INVALID_ARG).  After a
   replay, wait for the replay's stream before ttcross_sync, which then reads
   the device on every call for this handle; device_ms keeps the last
   ordinary run's time. */
ttc_status ttcross_run(ttc_handle *h, double eps, int max_rank,
                       const int32_t *subtensor_grid, void *stream);

/* Runs count independent instances (each created by ttcross_create) in one
   persistent launch on `stream` (the batching of many tensors of uneven
   shape and rank in one launch; the paper runs one tensor at a time).
   eps[i], max_rank[i] (max_rank may be NULL: every instance's capacity) and
   grids[i] as eps, max_rank and subtensor_grid of ttcross_run; grids may be
   NULL, and so may any grids[i] (grids[i] has d_i entries).  The handles
   must be distinct and live on the current device.  Errors: INVALID_ARG
   (checked on the host before anything is launched; this includes a batch
   of two or more instances where an FP32 / float-float instance of the
   recompute form has a non-Hilbert generator, a combination that is not
   supported), CUDA, OOM.  The instance list lives with hs[0] (grown by
   ordinary calls).  CUDA graphs as for ttcross_run: a captured batch needs an
   earlier ordinary batch of at least count instances led by hs[0] and an
   earlier run of every instance with its grid; the list's pointers are
   captured by value, so a replay reruns these instances even after hs[0]
   led other batches. */
ttc_status ttcross_run_batch(ttc_handle *const *hs, int count, const double *eps,
                             const int32_t *max_rank, const int32_t *const *grids,
                             void *stream);

/* Schedule of the later runs of h (the paper picks its process-grid
   partitions by trying them, Sec. 5.1 testing setup; here the tile schedule):
   tile_edge 0 (the library's rule), 32 or 64 superblock rows / columns per
   CTA tile (FP64 and stored forms); queue_split 0 (half) or 1..7 eighths of
   the CTAs that start the stored screen on its queue of entries new to a
   superblock (the others start on the carried entries).  Pivots and results
   do not depend on it.  Errors: INVALID_ARG. */
ttc_status ttcross_set_plan(ttc_handle *h, int32_t tile_edge, int32_t queue_split);

/* Measures the candidate schedules of ttcross_set_plan on this instance (tile
   edge 64 and 32; queue split 4, 2, 6 eighths in the stored form), each by two
   runs of ttcross_run(eps, max_rank, subtensor_grid, stream) timed on the
   device, keeps the fastest for later runs and returns it (any output pointer
   may be NULL; best_ms is its device time).  Synchronous.  The caller may
   cache the choice per shape class and apply it with ttcross_set_plan.
   Errors: those of ttcross_run / ttcross_sync; INVALID_ARG for the user
   generator. */
ttc_status ttcross_autotune(ttc_handle *h, double eps, int max_rank, const int32_t *subtensor_grid,
                            void *stream, int32_t *tile_edge, int32_t *queue_split,
                            double *best_ms);

/* Waits for the last run of h and returns its device-side status. */
ttc_status ttcross_sync(ttc_handle *h);

/* TT core sizes s_0..s_d (s_0 = s_d = 1) after the last run.  Waits for it. */
ttc_status ttcross_get_ranks(ttc_handle *h, int64_t *s);

/* Core k (1 <= k <= d) as [s_{k-1}][n_k][s_k] row-major doubles into dst
   (s_{k-1} n_k s_k elements, caller-owned; device memory if dst_is_device,
   else host memory).  Waits for the last run. */
ttc_status ttcross_get_cores(ttc_handle *h, int k, double *dst, int dst_is_device,
                             void *stream);

/* Core construction from the pivot sets alone (Alg. 5, second loop; Sec.
   3.2.2, eq. corereshape): after the last run, every bond's history of
   Alg. 4 is rebuilt from the pivots (the pivot rows step by step, one CTA
   per bond), every superblock row of T_k is replayed from it (a row per
   warp, the rows sliced over the grid, as the paper's core-construction
   grids), and the last core X(I_{<=d-1}, :) is formed from the entries.  T,
   the history and the last bond's R are cleared first, so the cores read
   afterwards come from the pivots alone; by the arithmetic contract they
   equal the cores the sweeps kept, bit for bit.  Asynchronous on `stream`;
   its device time is ttc_stats.rebuild_ms.  Errors: those of ttcross_sync,
   OOM (a scratch of (d-1) * 256^2 doubles on first use), CUDA. */
ttc_status ttcross_rebuild_cores(ttc_handle *h, void *stream);

/* Pivot sets of bond k (1 <= k <= d-1) in insertion order: I_{<=k} as
   [r_k][k] and J_{>k} as [r_k][d-k] int32 host arrays (caller-owned). */
ttc_status ttcross_get_pivots(ttc_handle *h, int k, int32_t *I, int32_t *J);

/* Pivot inverse U_k = P_k^{-1} of bond k as [r_k][r_k] host doubles. */
ttc_status ttcross_get_pivot_inverse(ttc_handle *h, int k, double *U);

/* Statistics of the last run.  Waits for it. */
ttc_status ttcross_get_stats(ttc_handle *h, ttc_stats *st);

/* Frees the instance (waits for its last run).  NULL is accepted. */
ttc_status ttcross_destroy(ttc_handle *h);

/* Host-side check of the screens' tile arithmetic (Alg. 3's subtensors as
   CTA tiles, Sec. 3.2; no GPU and no handle needed).  For a d-mode tensor of
   mode sizes n[0..d-1] at bond ranks r[0..d-2] (bond k = r[k-1]), subtensor
   grid grid[0..d-1] (pieces per mode; NULL: library tiles) and tile edge
   tile_edge (32 or 64), it runs the kernels' own tile geometry on the host
   and counts in *violations the tiles that are empty, wider than the edge,
   outside their superblock or across a piece of the grid, plus every
   superblock row or column the tiles do not cover exactly once; with
   r_stored (nullable, d-1 ranks with 1 <= r_stored[b] <= r[b]: the ranks the
   stored residual was last written at) also every tile of the stored
   screen's carried rectangle that reaches outside the stored extent.  tiles[b]
   (may be NULL) receives bond b+1's tile count; cand_cap[b] (may be NULL)
   the candidate slots a run with rank caps caps[0..d-2] gives bond b+1
   (stored != 0: the stored form), which every tile count at ranks up to the
   caps must not exceed.  All arrays are caller-owned host memory.
   Errors: INVALID_ARG (d outside [2, TTC_MAXD], n[m] outside [1, 2^20],
   caps outside [1, 256], r[b] outside [1, caps[b]], r_stored[b] outside
   [1, r[b]], a grid entry outside [0, n[m]], a superblock above 2^24 rows or
   columns, a null array). */
ttc_status ttcross_check_tiles(int d, const int64_t *n, const int32_t *r, const int32_t *caps,
                               const int32_t *r_stored, const int32_t *grid, int tile_edge,
                               int stored, int64_t *tiles, int64_t *cand_cap,
                               int64_t *violations);

/* Sampled relative error of a TT, computed without allocating memory.
   The paper has no counterpart: this is for callers that cannot call
   cudaMalloc (a custom allocator or memory-pool callback, a process whose
   GPU memory budget is fixed at start-up, a host application that forbids
   allocation after initialisation).  It evaluates
   sqrt(sum (X - X~)^2 / sum X^2) over the same SplitMix64 samples as
   ttcross_run (all entries when nsamples <= 0 or >= prod n), where X is the
   Hilbert or Maxwellian generator *gen (TTC_GEN_TT is rejected: it would need
   device data) and X~ the TT whose core m (0-based) is the device array
   cores[m] laid out [s_m][n_m][s_{m+1}] row-major, as ttcross_get_cores
   writes it (s: host array of d+1 sizes, s_0 = s_d = 1, s_m <= 256).
   The result is written to *err, a caller-owned device double, in stream
   order on `stream`; the call returns after enqueueing two kernels.
   Scratch: a static 64 KiB device array per GPU holds one partial sum per
   chunk of 4096 samples, so nsamples is limited to 16,777,216 (larger
   requests return TTC_ERR_INVALID_ARG).  The first call on a device looks up
   that array's address; make it before any stream capture.  Calls outside a
   capture look it up again, so a call after cudaDeviceReset (which reloads
   the module) finds the array where it now is.  Every call uses
   the same array and overwrites what it reads, so calls whose kernels may
   overlap on the GPU (other streams or host threads) race and must be
   ordered by the caller.  No cudaMalloc, cudaFree or allocating library call
   is made.  Errors: INVALID_ARG, CUDA. */
ttc_status ttcross_sampled_error_noalloc(int d, const int64_t *n, const ttc_generator *gen,
                                         const double *const *cores, const int64_t *s,
                                         int64_t nsamples, uint64_t seed, double *err,
                                         void *stream);

/* Description of the last error on this host thread ("" if none). */
const char *ttcross_last_error_string(void);

#ifdef __cplusplus
}
#endif
#endif /* TTCROSS_H */
