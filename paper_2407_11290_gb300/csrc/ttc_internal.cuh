// ttc_internal.cuh -- device-side data layout and helpers of the TT cross.
//
// Layout in HBM (one instance; capacities fixed at create so one persistent
// launch can run the whole cross without reallocating):
//   bond b (paper's k = b+1), rank cap R_b, superblock rows a = p*n_b + i
//   (p indexes I_{<=k-1}), columns c = q*n_{b+1} + j (q indexes J_{>k+1}):
//     T  [R_b][ldT]  FP64, t-major: column t of T_k = C_k P_k^{-1} is contiguous
//     R  [R_b][ldR]  FP64: row t = X(I_{<=k}[t], superblock columns)
//     Thi/Tlo, Rhi/Rlo: FP32 (hi, lo) shadows of T and R for the mixed screens
//     U  [R_b][R_b]  P_k^{-1} (bordered Sherman-Morrison, Sec. 3.1.1)
//     hpiv/hc [R_b][R_b], delta[R_b]: pivot history replayed by Alg. 4
//     I, J: pivot multi-indices + column-major linear index + index sum
//     E  [ldT][ldR]  FP64, stored-residual form only: the residual of every
//        superblock entry, row-major (eq. aca_approx_E); ew [ldT] and
//        erow [ldR] hold the rank-one step of the last pivot
//   ldT = cap(R_{b-1}) * n_b and ldR = n_{b+1} * cap(R_{b+1}), so rows and
//   columns that enter the superblock later are appended, never moved.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define TTC_MAXD 16
#define TTC_MAXB (TTC_MAXD - 1)

namespace ttc {

constexpr int TT_GEN_RMAX = 160;  // largest TT rank of a TT-cores generator
constexpr int BM = 64, BN = 64;   // screen tile (superblock rows x columns)
constexpr int RCAP = 256;         // largest rank capacity the kernels accept
constexpr int GRID_CAP = 4096;    // largest persistent grid (partial-sum slots)

enum State : int32_t { ST_SCREEN = 0, ST_UPDATE = 1, ST_VERIFY = 2, ST_DONE = 3 };
enum Prec : int32_t { P_FP64 = 0, P_FP32 = 1, P_SPLIT = 2 };

struct SetDev {          // pivot index set I_{<=k} or J_{>k}
  int32_t *idx;          // [cap][width] mode indices
  int64_t *lin;          // [cap] part of the column-major linear index
  int32_t *sum;          // [cap] sum of the indices (Hilbert)
  int32_t width;
};

struct BondDev {
  int32_t cap;
  int64_t ldT, ldR;      // row / column capacity of the superblock
  double *T, *R, *U, *hpiv, *hc, *delta;
  float *Thi, *Tlo, *Rhi, *Rlo;
  int32_t *prow, *pcol;  // pivot superblock coordinates, insertion order
  double *E, *ew, *erow; // stored-residual form (null otherwise)
  double *A;             // user generator: the entries of the superblock [ldT][ldR]
  SetDev I, J;
  int64_t cand_base;     // first candidate slot of this bond
  int64_t cand_cap;      // candidate slots of this bond
};

// Per-instance control block; written by the device, read by the host.
struct Ctrl {
  int32_t state;
  int32_t status;
  int32_t r[TTC_MAXD];     // current ranks (bond b)
  int32_t r_old[TTC_MAXD]; // ranks before the last pivot step
  int32_t add[TTC_MAXD];   // bond added a pivot in the last decision
  int32_t maxr[TTC_MAXD];  // rank caps of this run
  int32_t ntiles[TTC_MAXD];// tiles screened for bond b in the last screen
  uint64_t best_key[TTC_MAXD];
  int64_t best_lin[TTC_MAXD];
  int32_t best_row[TTC_MAXD], best_col[TTC_MAXD];
  double eps, tau, xrms, den, err;
  int64_t sweeps, entries, refinements, tiles_refined;
  int64_t unscreened;        // candidate slots read by a merge that no screen wrote
  // tile schedule of the next screen (written by the instance's owner CTA
  // whenever its ranks change, read by every CTA): tile edge, and per bond
  // the superblock rows / columns and row / column tile counts
  int32_t plan_te;
  int32_t plan_rows[TTC_MAXD], plan_cols[TTC_MAXD];
  int32_t plan_nrt[TTC_MAXD], plan_nct[TTC_MAXD];
  int32_t screened;          // screened in this sweep (set by the screen, cleared by decide)
  int32_t pad2;
  int32_t pending[TTC_MAXD]; // mixed forms: bond merged, waiting for the refinement
  int32_t nrefine_bond[TTC_MAXD];
  int64_t screen_fmas, error_fmas;  // algorithmic FMAs of the screens / errors
  int32_t max_refine;
  int32_t grid[TTC_MAXD];  // subtensor pieces per mode (0 = library tiles)
  // plan of this run (ttcross_set_plan / the autotuner): tile edge (0 = the
  // library's rule, 32, 64) and the eighths of the CTAs that start the
  // stored screen on its fresh queue (0 = half)
  int32_t force_te, qsplit;
  int32_t pad;
  // stored-residual form, per bond: the stored extent (superblock rows /
  // columns as of the last screen) and whether the rank-one step of the last
  // pivot (ew, erow) is still to be applied by the next screen
  int32_t st_rows[TTC_MAXD], st_cols[TTC_MAXD];
  int32_t e_pend[TTC_MAXD];
  int32_t steal, steal2;     // stored form: items handed out by the running screen
                             // from its fresh / carried queues (cleared by the
                             // decide phase after it)
  int64_t entries_fresh;     // entries evaluated as A - T R (the rest carried)
  int64_t stored_bytes;      // bytes of E read and written by the screens
  // sampled screen: refinement step of each bond (0 none / done, 1 the
  // column of the pivot next, 2 its row next), rounds run, whether the
  // running round moved the pivot
  int32_t rook_stage[TTC_MAXD], rook_round[TTC_MAXD], rook_moved[TTC_MAXD];
  int64_t screen_t;          // sampled screen: screens run (the sample counter)
  int32_t dcount[TTC_MAXD];  // stored forms: parts of bond b's decide that have
                             // merged their share of the tile slots (the last
                             // one finishes the bond and clears it)
  int32_t dkind;             // work of the coming decide phases, fixed by the
                             // screen phase: DK_BONDS, DK_VERIFY or DK_NONE
  int32_t pad_dkind;
};

enum DecideKind { DK_NONE = 0, DK_BONDS = 1, DK_VERIFY = 2 };

struct InstDev {
  int32_t d, nb;
  int64_t n[TTC_MAXD], stride[TTC_MAXD];
  int32_t gen;                       // ttc_gen_kind
  const double *hilb;                // [sum_m (n_m-1) + 1] = 1/(s+1)
  const float *hilb_hi, *hilb_lo;    // its (hi, lo) FP32 split
  const double *tt;                  // TT cores
  int32_t rho[TTC_MAXD + 1];
  int64_t core_off[TTC_MAXD + 1];
  int32_t dx, dv;
  double a_rho, a_u, a_T, vmin, vmax;
  // Maxwellian tables (built on the device at create): for every combination
  // of the x indices, coef = rho / (2 pi T)^{dv/2} and nh = -1 / (2 T); and
  // cos x_m per x mode (mx_cos + mx_off[m])
  const double *mx_coef, *mx_nh, *mx_cos;
  int64_t mx_off[TTC_MAXD];
  int64_t mx_stride[TTC_MAXD];
  int32_t prec;
  int32_t topk;
  int32_t stored;                    // stored-residual screen
  // Alg. 1 with a random sample set: samples per bond and screen (0: the
  // whole superblock), their SplitMix64 seed, refinement rounds
  int64_t nl;
  uint64_t lseed;
  int32_t max_rook;
  BondDev bond[TTC_MAXB];
  SetDev empty;                      // I_{<=0} / J_{>d}: one empty multi-index
  double *xs;                        // X at the error samples
  double *tabL, *tabR;               // prefix / suffix contractions of the TT (error check)
  int64_t tabL_cap, tabR_cap;        // their capacities (doubles)
  int64_t nsamples;                  // samples used (== prod n when exhaustive)
  int32_t exhaustive;
  uint64_t seed;
  double *err_part;                  // [max grid] partial sums
  struct Cand *start_part;           // [max grid] per-CTA argmax |X| over the samples
  int32_t err_part_cap;
  struct Cand *cand;
  struct MCand *mcand;               // mixed-form tile candidates (same slots as cand)
  int32_t *refine_list;              // [cand capacity][2]: (bond, tile) to re-screen in FP64
  struct Cand *refine_cand;          // their FP64 results
  Ctrl *ctrl;
};

// Mixed-form tile candidate: the tile's best |E| in FP32 / float-float and
// bounds on the FP64 residual of the tile's entries:
//   |E64(best)| <= v * (1 + 4u) + eabs,  |E64(other)| <= rest * (1 + 4u) + eabs
struct MCand {
  float v, rest;
  double eabs;
  int64_t lin;
  int32_t row, col;
};

struct Cand {            // one screen candidate (max |E| of a tile, or top-k)
  uint64_t key;          // bits of |E| (FP64 or FP32 widened), larger wins
  int64_t lin;           // column-major linear index, smaller wins ties
  int32_t row, col;      // superblock coordinates
};

struct Barrier {
  unsigned int count;
  unsigned int gen;      // unused (the arrival count alone orders the barriers)
  int32_t abort;
  int32_t where;         // first wait that ran out
  int32_t overrun;       // the sweep cap was reached before every instance finished
  int32_t pad;
  uint64_t phase_ns[8];  // time per phase (CTA 0, barrier exit to barrier exit)
};

enum PhaseSlot { T_INIT = 0, T_SCREEN = 1, T_DECIDE = 2, T_UPDATE = 3, T_VERIFY = 4, T_REFINE = 5 };

// shadows of an FP64 value as (hi, lo) floats
__device__ __forceinline__ void split2(double x, float &hi, float &lo) {
  hi = __double2float_rn(x);
  lo = __double2float_rn(x - (double)hi);
}

struct RunArgs {
  InstDev *const *insts; // device array of instance pointers
  int32_t count;
  int32_t mixed;         // some instance screens in FP32 / float-float
  Barrier *bar;
  int64_t wait_ns;
  int32_t persistent;
  int32_t max_iters;     // sweep cap of the launch (sum of rank caps + refinements)
  int32_t *smid;         // [grid] the SM each CTA of a persistent launch runs on
  int32_t sampled;       // some instance screens a random sample set (Alg. 1)
  int32_t max_rook;      // the largest refinement round count of the instances
};

// ---------------------------------------------------------------------------
// small helpers

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Control words written by other CTAs earlier in the launch, read from L2:
// the grid barrier's fence orders the writes before the read, and the L2
// path skips this SM's L1 (which may hold a stale copy) without the
// system-scope ordering a volatile access carries.
__device__ __forceinline__ int32_t ld_cg(const int32_t &x) { return __ldcg(&x); }
__device__ __forceinline__ int64_t ld_cg(const int64_t &x) {
  return (int64_t)__ldcg(reinterpret_cast<const long long *>(&x));
}
__device__ __forceinline__ uint64_t ld_cg(const uint64_t &x) {
  return (uint64_t)__ldcg(reinterpret_cast<const unsigned long long *>(&x));
}
__device__ __forceinline__ double ld_cg(const double &x) { return __ldcg(&x); }

// key order: larger |E| first, then smaller linear index
__device__ __forceinline__ bool key_better(uint64_t k1, int64_t l1, uint64_t k2, int64_t l2) {
  return k1 > k2 || (k1 == k2 && l1 < l2);
}

// The bits of |e| (the order of the keys is the order of |e|), formed by an
// integer AND on the high word.  Written as a 64-bit mask the compiler may
// take the FP64 pipe for it (an add with an absolute-value operand); that
// pipe runs about two FMAs per clock per SM here and is the screens' binding
// resource, so the key stays on the integer pipe.
__device__ __forceinline__ uint64_t abs_key(double e) {
  uint32_t lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(e));
  asm("and.b32 %0, %0, 0x7FFFFFFF;" : "+r"(hi));
  return ((uint64_t)hi << 32) | lo;
}
// +Inf bit pattern: keys above it are NaN
constexpr uint64_t KEY_INF = 0x7FF0000000000000ull;

// The contract's dot product: acc = +0; acc = fma(x[t], y[t], acc), t = 0..K-1.
// Operands are loaded eight pairs at a time before their FMAs, so a chain
// over global memory waits for one round trip per eight terms, not per term;
// the FMAs still run in the serial order t = 0, 1, ...
__device__ __forceinline__ double chain(const double *x, int64_t sx, const double *y, int64_t sy,
                                        int K) {
  double acc = 0.0;
  int t = 0;
  for (; t + 8 <= K; t += 8) {
    double xv[8], yv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      xv[k] = x[(t + k) * sx];
      yv[k] = y[(t + k) * sy];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) acc = __fma_rn(xv[k], yv[k], acc);
  }
  for (; t < K; ++t) acc = __fma_rn(x[t * sx], y[t * sy], acc);
  return acc;
}

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ int64_t rows_of(const InstDev &in, const int32_t *r, int b) {
  return (int64_t)(b == 0 ? 1 : r[b - 1]) * in.n[b];
}
__host__ __device__ __forceinline__ int64_t cols_of(const InstDev &in, const int32_t *r, int b) {
  return in.n[b + 1] * (int64_t)(b == in.nb - 1 ? 1 : r[b + 1]);
}
__device__ __forceinline__ const SetDev &left_set(const InstDev &in, int b) {
  return b == 0 ? in.empty : in.bond[b - 1].I;
}
__device__ __forceinline__ const SetDev &right_set(const InstDev &in, int b) {
  return b == in.nb - 1 ? in.empty : in.bond[b + 1].J;
}

}  // namespace ttc
