// ttc_kernels.cu -- the hot path of the adaptive TT cross on sm_103a.
//
// One sweep (all bonds at once, Sec. 3.2.3) is three phases:
//   screen : every CTA takes superblock tiles of every bond (the paper's
//            subtensors of Alg. 3 become CTA tiles), generates the entries,
//            forms E = A - T R with the FP64 FMA chain of the arithmetic
//            contract (or the FP32 / float-float forms), and keeps the tile's
//            max |E| (ties: lowest column-major linear index);
//   decide : one CTA per instance merges the tile candidates (the Allgather
//            of Alg. 3), applies the stop test and appends the pivots:
//            nested index sets (eq. nestedpivots), pivot history, and the
//            bordered Sherman-Morrison update of P^{-1} (Sec. 3.1.1);
//   update : every CTA applies eq. aca_approx_T_sub to the old rows of T,
//            replays the pivot history on rows that entered the superblock
//            (Alg. 4), and generates the new rows / columns of R; or, when an
//            instance has converged at its threshold, evaluates the sampled
//            error of Sec. 5.
// The phases run either in one persistent cooperative launch separated by
// grid barriers (every wait bounded in time) or as separate launches.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <memory>
#include <vector>

#include "ttc_gen.cuh"
#include "ttc_internal.cuh"
#include "ttc_launch.h"

namespace ttc {

constexpr int NT = 256;  // threads per CTA
constexpr int KC = 32;   // depth of the T / R chunks staged in shared memory


struct ScreenSmem {
  union {
    struct {
      double Ts[KC][BM];
      double Rs[KC][BN];
    } d;
    struct {
      float Th[KC][BM], Tl[KC][BM];
      float Rh[KC][BN], Rl[KC][BN];
    } f;
  } op;
  int32_t srow[BM], scol[BN];
  int64_t lrow[BM], lcol[BN];
  int32_t ridx[BM][TTC_MAXD];
  int32_t cidx[BN][TTC_MAXD];
  float rowS[BM], colR[BN];
  uint64_t sk[NT / 32];
  int64_t sl[NT / 32];
  int32_t sr[NT / 32], sc[NT / 32];
  float fred[NT / 32];
  const double *acache;  // user generator: the tile's first entry in the cache
  int64_t acache_ld;
};

constexpr int TOPK_MAX = 16;
// stored-residual form: candidate slots per tile (the quarters of a fresh tile;
// a carried tile uses the first and marks the rest empty, row -2)
constexpr int STORED_SLOTS = 4;

constexpr int DEC_US = 32;  // pivot steps up to this rank stage U in shared memory
struct DecideSmem {
  double ua[RCAP], bu[RCAP], brow[RCAP];
  double hcs[RCAP], hps[RCAP];  // R(:, c*) and T(a*, :) of the pivot step
  double us[DEC_US * DEC_US];   // U before the step (z <= DEC_US)
  int32_t key[RCAP];            // pivot t's column: index sum (Hilbert) or coordinate
  int32_t lsum, rsum;           // index sums of the pivot's row part / column part
  int64_t q_nt;                 // control words of the decide item
  int32_t q_r, q_maxr, q_prow, q_pcol;
  double q_tau, q_xrms;
  double apiv;                  // A(a*, c*)
  int32_t sel[TOPK_MAX];
  uint64_t skey[TOPK_MAX];
  int64_t slin[TOPK_MAX];
  int32_t srow[TOPK_MAX], scol[TOPK_MAX];
  int32_t cnt;
  double red[NT / 32];
  uint64_t rk[NT / 32];
  int64_t rl[NT / 32];
  int32_t rr[NT / 32], rc[NT / 32];
  double delta;
  int32_t flag;
  // the eight warps' top candidates of the mixed stored decide
  uint64_t wk[NT / 32 * 8];
  int64_t wl[NT / 32 * 8];
  int32_t wr[NT / 32 * 8], wc[NT / 32 * 8];
  // keys and indices of up to 2 NT slots ranked at once (stored decide)
  uint64_t tk[2 * NT];
  int64_t tl[2 * NT];
  int32_t last;  // this CTA finishes the bond's decide
};

constexpr int SPREAD_MAXSM = 1024;
struct SpreadSmem {
  int32_t cnt[SPREAD_MAXSM];  // CTAs per SM id
  int32_t k, place, bad, nsm, not2;
};

// replays of up to 32 pivots (Alg. 4): the history triangles (row z at
// z (z - 1) / 2) and delta, shared by the CTA's replay warps; after the
// block reductions' words, which the CTA's other warps may be using meanwhile
constexpr int LANE_NZ = 32;
struct ReplaySmem {
  double red_pad[NT / 32];
  double hc[LANE_NZ * (LANE_NZ - 1) / 2], hp[LANE_NZ * (LANE_NZ - 1) / 2];
  double delta[LANE_NZ];
};

// the error's samples when the tables meet: a warp's 32 samples' table rows
// (up to 16 entries, rows padded to 17 against bank conflicts); after the
// block reduction's words
struct SampleSmem {
  double red_pad[NT / 32];
  double rows[NT / 32][32 * 17];
};

union __align__(16) PhaseSmem {
  ScreenSmem s;
  DecideSmem d;
  SpreadSmem sp;
  ReplaySmem rp;
  SampleSmem sw;
  double red[NT / 32];
};

// The descriptor of instance 0, copied into shared memory when a kernel
// starts: every phase reads its fields all the time, and from global memory
// each one is a dependent load at L2 latency.  It does not change during a
// launch (the host writes it before launching).
__shared__ InstDev s_inst0;

// This CTA's place in the SM-spread order of the grid (the CTAs sorted by
// their slot on their SM, then by SM): work dealt to places 0, 1, 2, ...
// lands on distinct SMs before any SM gets a second share.  Latency-bound
// items (pivot steps, replays) then do not queue for the FP64 pipe, which
// is shared by the whole SM.  blockIdx.x until the order is known.
__shared__ int32_t s_place;
// S when the grid holds exactly two CTAs on each of S SMs (then places p and
// p + S share an SM), else 0 (not known, or another layout)
__shared__ int32_t s_sm2;
// grid barriers this CTA has passed in the running launch
__shared__ uint32_t s_bar_epoch;

__device__ void cache_inst0(const RunArgs &ra) {
  static_assert(sizeof(InstDev) % 8 == 0, "InstDev copies as 8-byte words");
  if (threadIdx.x == 0) {
    s_place = blockIdx.x;
    s_sm2 = 0;
    s_bar_epoch = 0u;
  }
  const unsigned long long *src = reinterpret_cast<const unsigned long long *>(ra.insts[0]);
  unsigned long long *dst = reinterpret_cast<unsigned long long *>(&s_inst0);
  for (int i = threadIdx.x; i < (int)(sizeof(InstDev) / 8); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

__device__ __forceinline__ const InstDev &inst(const RunArgs &ra, int ii) {
  return ii == 0 ? s_inst0 : *ra.insts[ii];
}

// sampled screen's decide item (defined with its refinement phases below)
__device__ void decide_bond_sampled(const InstDev &in, Ctrl &cr, int b, DecideSmem &sm);

// sampled-error split (defined with the error evaluation below)
__device__ void choose_split(const InstDev &in, const int32_t *r, int &pL, int &pR);
__device__ double split_cost(const InstDev &in, const int32_t *r, int pL, int pR);

// ---------------------------------------------------------------------------
// reductions

struct KeyBest {
  uint64_t key;
  int64_t lin;
  int32_t row, col;
};

__device__ __forceinline__ void kb_take(KeyBest &a, const KeyBest &b) {
  if (b.row >= 0 && (a.row < 0 || key_better(b.key, b.lin, a.key, a.lin))) a = b;
}

// block-wide max by key; result valid in thread 0
__device__ KeyBest block_best(KeyBest v, uint64_t *sk, int64_t *sl, int32_t *sr, int32_t *sc) {
  for (int off = 16; off > 0; off >>= 1) {
    KeyBest o;
    o.key = __shfl_down_sync(0xffffffffu, v.key, off);
    o.lin = __shfl_down_sync(0xffffffffu, v.lin, off);
    o.row = __shfl_down_sync(0xffffffffu, v.row, off);
    o.col = __shfl_down_sync(0xffffffffu, v.col, off);
    kb_take(v, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) { sk[w] = v.key; sl[w] = v.lin; sr[w] = v.row; sc[w] = v.col; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < NT / 32; ++i) {
      KeyBest o{sk[i], sl[i], sr[i], sc[i]};
      kb_take(v, o);
    }
  }
  return v;
}

// deterministic block sum (fixed shuffle tree, warps summed in order)
__device__ double block_sum(double v, double *red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < NT / 32; ++i) s += red[i];
  return s;
}

// ---------------------------------------------------------------------------
// grid barrier for the persistent form: arrive, then wait for the generation
// to change; every wait gives up after wait_ns and raises the abort flag.
// Grid barrier of the persistent kernel.  The arrival counter only rises
// (the host clears it before each launch): the k-th barrier completes when
// it reaches k G, so a CTA arrives with one atomic and polls the same word.
// There is no reset or generation flip by the last arrival, whose extra
// round trips to L2 were on every barrier's critical path.  Every wait is
// bounded by wait_ns; on expiry the CTA records where, raises abort (which
// every poller checks) and returns false.
__device__ bool grid_barrier(const RunArgs &ra, int where) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    Barrier *bar = ra.bar;
    volatile unsigned int *vcount = &bar->count;
    volatile int32_t *vabort = &bar->abort;
    const unsigned int target = (s_bar_epoch + 1u) * gridDim.x;
    s_bar_epoch += 1u;
    __threadfence();  // this CTA's writes before its arrival
    const unsigned int arrived = atomicAdd(&bar->count, 1u) + 1u;
    if (arrived < target) {
      const uint64_t t0 = globaltimer_ns();
      while (*vcount < target) {
        if (*vabort) {
          ok = 0;
          break;
        }
        if (globaltimer_ns() - t0 > (uint64_t)ra.wait_ns) {
          atomicCAS(&bar->where, 0, where);
          atomicExch(&bar->abort, 1);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();  // the other CTAs' writes after the barrier
    if (*vabort) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

// ---------------------------------------------------------------------------
// tiles of the superblock of bond b.  Without a subtensor grid the rows
// (columns) are cut into BM (BN) chunks; with one, mode b (b+1) is split into
// grid[b] (grid[b+1]) balanced pieces and no tile crosses a piece.

// Balanced split of n indices into C pieces: the first rem = n mod C pieces
// hold q + 1 = n / C + 1 indices, the others q.  Tiles never cross a piece.
struct Pieces {
  int32_t q, rem, tq1, tq0, tpb;  // tiles per piece of size q+1 / q, tiles per block
};

__host__ __device__ __forceinline__ Pieces make_pieces(int32_t n, int32_t C, int32_t te) {
  Pieces P;
  P.q = n / C;
  P.rem = n - P.q * C;
  P.tq1 = (P.q + 1 + te - 1) / te;
  P.tq0 = (P.q + te - 1) / te;
  P.tpb = P.rem * P.tq1 + (C - P.rem) * P.tq0;
  return P;
}

// tile t of one block: start within the block and length
__host__ __device__ __forceinline__ void piece_tile(const Pieces &P, int32_t t, int32_t te,
                                                    int32_t &start, int32_t &len) {
  int32_t k, tin, size;
  if (t < P.rem * P.tq1) {
    k = t / P.tq1;
    tin = t - k * P.tq1;
    size = P.q + 1;
  } else {
    const int32_t u = t - P.rem * P.tq1;
    const int32_t kk = u / P.tq0;
    k = P.rem + kk;
    tin = u - kk * P.tq0;
    size = P.q;
  }
  start = k * P.q + min(k, P.rem) + tin * te;
  len = min(te, size - tin * te);
}

// Tile geometry of bond b for edge te, from the ranks r (no subtensor grid:
// rows / columns cut into te-chunks; grid: pieces of mode b / b+1 per block)
struct TileGeo {
  int32_t nrt, nct;        // row tiles, column tiles
  int32_t rows, cols;
  int32_t te;
  int32_t pr, pc;          // pieces (0 = none)
  Pieces P, Q;             // row / column pieces
};

__host__ __device__ TileGeo tile_geo_e(const InstDev &in, const Ctrl &cr, const int32_t *r, int b,
                                       int te) {
  TileGeo g;
  g.te = te;
  g.rows = (int32_t)rows_of(in, r, b);
  g.cols = (int32_t)cols_of(in, r, b);
  g.pr = cr.grid[b];
  g.pc = cr.grid[b + 1];
  const int32_t nrb = b == 0 ? 1 : r[b - 1];
  const int32_t ncb = b == in.nb - 1 ? 1 : r[b + 1];
  if (g.pr > 0) {
    g.P = make_pieces((int32_t)in.n[b], g.pr, te);
    g.nrt = nrb * g.P.tpb;
  } else {
    g.nrt = (g.rows + te - 1) / te;
  }
  if (g.pc > 0) {
    g.Q = make_pieces((int32_t)in.n[b + 1], g.pc, te);
    g.nct = ncb * g.Q.tpb;
  } else {
    g.nct = (g.cols + te - 1) / te;
  }
  return g;
}

// Tile autotuner (in write_plan_warp): 64 x 64 tiles, unless the instance's
// superblocks give under a quarter wave of them on this grid while the
// contraction is deep (rank >= 24): then 32 x 32 tiles put four times the
// CTAs to work.  At small ranks the per-tile overhead dominates and 64 x 64
// stays faster (measured on the 6D Hilbert workloads).
// the tile plan of the next screen at ranks r, computed by one warp of the
// owner CTA (lane b handles bond b)
__device__ void write_plan_warp(const InstDev &in, Ctrl &cr, const int32_t *r, int grid) {
  const int lane = threadIdx.x & 31;
  const bool act = lane < in.nb;
  TileGeo g64;
  int64_t t64 = 0;
  int kmax = 0;
  if (act) {
    g64 = tile_geo_e(in, cr, r, lane, 64);
    t64 = (int64_t)g64.nrt * g64.nct;
    kmax = r[lane];
  }
  for (int off = 16; off > 0; off >>= 1) {
    t64 += __shfl_xor_sync(0xffffffffu, t64, off);
    kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, off));
  }
  // pieces of the subtensor grid at most 32 wide on every bond: a 64-wide
  // tile would hold one piece and compute three quarters padding; 32 x 32
  // tiles give the same tiles without it (FP64 forms)
  int small = 1;
  if (act) {
    const int64_t pr = cr.grid[lane], pc = cr.grid[lane + 1];
    const int64_t sr = pr > 0 ? (in.n[lane] + pr - 1) / pr : 64;
    const int64_t sc = pc > 0 ? (in.n[lane + 1] + pc - 1) / pc : 64;
    small = sr <= 32 && sc <= 32;
  }
  const bool pieces32 = __all_sync(0xffffffffu, small) && (in.prec == P_FP64 || in.stored);
  int te = 64;
  TileGeo g = g64;
  // a tile edge set for this run (the FP64 and stored forms; the mixed
  // recompute forms keep 64-wide tiles); 32-wide tiles when the candidate
  // slots of every bond allow them
  const int fte = (in.prec == P_FP64 || in.stored) ? cr.force_te : 0;
  int fok = fte == 32 || fte == 64;
  if (fte == 32) {
    TileGeo g32;
    int ok = 1;
    if (act) {
      g32 = tile_geo_e(in, cr, r, lane, 32);
      ok = (int64_t)g32.nrt * g32.nct <= in.bond[lane].cand_cap;
    }
    fok = __all_sync(0xffffffffu, ok);
    if (fok) {
      te = 32;
      g = g32;
    }
  }
  if (fok) {
    // the edge set for the run
  } else if (pieces32) {
    te = 32;
    if (act) g = tile_geo_e(in, cr, r, lane, 32);
  } else if (!in.stored && in.prec == P_FP64 && 4 * t64 < (int64_t)grid && kmax >= 24) {
    // 32 x 32 tiles when the candidate slots of every bond allow them
    int ok = 1;
    if (act) {
      g = tile_geo_e(in, cr, r, lane, 32);
      ok = (int64_t)g.nrt * g.nct <= in.bond[lane].cand_cap;
    }
    if (__all_sync(0xffffffffu, ok)) {
      te = 32;
    } else {
      g = g64;
    }
  }
  if (act) {
    cr.plan_rows[lane] = g.rows;
    cr.plan_cols[lane] = g.cols;
    cr.plan_nrt[lane] = g.nrt;
    cr.plan_nct[lane] = g.nct;
  }
  if (lane == 0) cr.plan_te = te;
}

// geometry of bond b as planned (cheap: no tile counting)
__device__ __forceinline__ TileGeo planned_geo(const InstDev &in, const Ctrl &cr, int b) {
  TileGeo g;
  g.te = ld_cg(cr.plan_te);
  g.rows = ld_cg(cr.plan_rows[b]);
  g.cols = ld_cg(cr.plan_cols[b]);
  g.nrt = ld_cg(cr.plan_nrt[b]);
  g.nct = ld_cg(cr.plan_nct[b]);
  g.pr = cr.grid[b];
  g.pc = cr.grid[b + 1];
  if (g.pr > 0) g.P = make_pieces((int32_t)in.n[b], g.pr, g.te);
  if (g.pc > 0) g.Q = make_pieces((int32_t)in.n[b + 1], g.pc, g.te);
  return g;
}

__host__ __device__ __forceinline__ void tile_rows(const InstDev &in, const TileGeo &g, int b,
                                                   int32_t t, int64_t &r0, int &nr) {
  if (g.pr > 0) {
    const int32_t p = t / g.P.tpb;
    int32_t st, len;
    piece_tile(g.P, t - p * g.P.tpb, g.te, st, len);
    r0 = (int64_t)p * in.n[b] + st;
    nr = len;
  } else {
    r0 = (int64_t)t * g.te;
    nr = min(g.te, g.rows - t * g.te);
  }
}

__host__ __device__ __forceinline__ void tile_cols(const InstDev &in, const TileGeo &g, int b,
                                                   int32_t t, int64_t &c0, int &nc) {
  if (g.pc > 0) {
    const int32_t q = t / g.Q.tpb;
    int32_t st, len;
    piece_tile(g.Q, t - q * g.Q.tpb, g.te, st, len);
    c0 = (int64_t)q * in.n[b + 1] + st;
    nc = len;
  } else {
    c0 = (int64_t)t * g.te;
    nc = min(g.te, g.cols - t * g.te);
  }
}

// ---------------------------------------------------------------------------
// screen of one tile in FP64: A - chain(T(a,:), R(:,c)) for a 64 x 64 tile,
// 4 x 4 entries per thread, T / R staged through shared memory in 32-deep
// chunks; the accumulation order over t is the contract's serial chain.
// per-row / per-column data of a tile: linear-index parts, index sums
// (Hilbert) or the multi-indices (other generators)
__device__ void stage_meta(const InstDev &in, int b, int64_t r0, int nr, int64_t c0, int nc,
                           ScreenSmem &sm) {
  const SetDev &L = left_set(in, b);
  const SetDev &Rset = right_set(in, b);
  const int tid = threadIdx.x;
  const int64_t nb0 = in.n[b], nb1 = in.n[b + 1];
  const bool hil = in.gen == 0;
  const int wl = b, wr = in.d - b - 2;
  if (tid == 0 && in.gen == 4) {
    sm.acache = in.bond[b].A + r0 * in.bond[b].ldR + c0;
    sm.acache_ld = in.bond[b].ldR;
  }
  for (int x = tid; x < BM; x += NT) {
    if (x < nr) {
      const uint32_t a = (uint32_t)(r0 + x), p = a / (uint32_t)nb0, i = a - p * (uint32_t)nb0;
      sm.lrow[x] = L.lin[p] + i * in.stride[b];
      if (hil) {
        sm.srow[x] = L.sum[p] + (int)i;
      } else {
        for (int m = 0; m < wl; ++m) sm.ridx[x][m] = L.idx[p * wl + m];
        sm.ridx[x][wl] = (int32_t)i;
      }
    }
  }
  for (int x = tid; x < BN; x += NT) {
    if (x < nc) {
      const uint32_t c = (uint32_t)(c0 + x), q = c / (uint32_t)nb1, j = c - q * (uint32_t)nb1;
      sm.lcol[x] = j * in.stride[b + 1] + Rset.lin[q];
      if (hil) {
        sm.scol[x] = (int)j + Rset.sum[q];
      } else {
        sm.cidx[x][0] = (int32_t)j;
        for (int m = 0; m < wr; ++m) sm.cidx[x][1 + m] = Rset.idx[q * wr + m];
      }
    }
  }
}

__device__ __noinline__ double tile_entry(const InstDev &in, const ScreenSmem &sm, int wl, int wr,
                                             int rr, int cc) {
  if (in.gen == 0) return in.hilb[sm.srow[rr] + sm.scol[cc]];
  if (in.gen == 4) return sm.acache[rr * sm.acache_ld + cc];
  int32_t idx[TTC_MAXD];
  for (int m = 0; m <= wl; ++m) idx[m] = sm.ridx[rr][m];
  for (int m = 0; m <= wr; ++m) idx[wl + 1 + m] = sm.cidx[cc][m];
  return gen_full(in, idx);
}

// acc[u][v] = chain(T(r0 + ty + 16u, :), R(:, c0 + tx + 16v)) over t < K, the
// contract's serial FMA order, T / R staged through shared memory in 32-deep
// chunks (the first chunk's barrier also publishes the tile metadata)
template <int TE>
__device__ __forceinline__ void tile_chain_fp64(const BondDev &B, int K, int64_t r0, int nr,
                                                int64_t c0, int nc, double (&acc)[TE / 16][TE / 16],
                                                ScreenSmem &sm) {
  constexpr int U = TE / 16;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < U; ++v) acc[u][v] = 0.0;
  // a chunk's staging issues all its loads before the first store (one round
  // trip to L2 instead of one per loop pass)
  constexpr int PER = KC * TE / NT;
  static_assert(KC * TE % NT == 0, "staging passes");
  for (int t0 = 0; t0 < K; t0 += KC) {
    const int kc = min(KC, K - t0);
    double tl[PER], rl[PER];
#pragma unroll
    for (int m = 0; m < PER; ++m) {
      const int x = tid + NT * m, tt = x / TE, ee = x - tt * TE;
      tl[m] = (tt < kc && ee < nr) ? B.T[(int64_t)(t0 + tt) * B.ldT + r0 + ee] : 0.0;
      rl[m] = (tt < kc && ee < nc) ? B.R[(int64_t)(t0 + tt) * B.ldR + c0 + ee] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < PER; ++m) {
      const int x = tid + NT * m, tt = x / TE, ee = x - tt * TE;
      if (tt < kc) {
        sm.op.d.Ts[tt][ee] = tl[m];
        sm.op.d.Rs[tt][ee] = rl[m];
      }
    }
    __syncthreads();
    for (int tt = 0; tt < kc; ++tt) {
      double tv[U], rv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) tv[u] = sm.op.d.Ts[tt][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < U; ++v) rv[v] = sm.op.d.Rs[tt][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) acc[u][v] = __fma_rn(tv[u], rv[v], acc[u][v]);
    }
  }
}

// acc[u][v] ~ T(r0 + ty + 16u, :) R(:, c0 + tx + 16v) over t < K on the FP32
// pipe, from the (hi, lo) FP32 shadows of T and R (mixed forms of the stored
// screen).  SPLIT: float-float, th rh = p + pe exactly (pe by FMA), the cross
// terms th rl + tl rh and pe join the low word, the high word is summed by
// TwoSum and the pair renormalised every term, so the result carries about
// 44 bits; else plain FP32 products and sums (sl = 0).  The result is the
// pair (sh, sl).
template <int TE, bool SPLIT>
__device__ __forceinline__ void tile_chain_ff(const BondDev &B, int K, int64_t r0, int nr,
                                              int64_t c0, int nc, float (&sh)[TE / 16][TE / 16],
                                              float (&sl)[TE / 16][TE / 16], ScreenSmem &sm) {
  constexpr int U = TE / 16;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < U; ++v) {
      sh[u][v] = 0.f;
      sl[u][v] = 0.f;
    }
  constexpr int PER = KC * TE / NT;
  static_assert(KC * TE % NT == 0, "staging passes");
  for (int t0 = 0; t0 < K; t0 += KC) {
    const int kc = min(KC, K - t0);
    float th[PER], tl[PER], rh[PER], rl[PER];
#pragma unroll
    for (int m = 0; m < PER; ++m) {
      const int x = tid + NT * m, tt = x / TE, ee = x - tt * TE;
      const bool tv = tt < kc && ee < nr, rv = tt < kc && ee < nc;
      const int64_t ot = (int64_t)(t0 + tt) * B.ldT + r0 + ee;
      const int64_t orr = (int64_t)(t0 + tt) * B.ldR + c0 + ee;
      th[m] = tv ? B.Thi[ot] : 0.f;
      rh[m] = rv ? B.Rhi[orr] : 0.f;
      tl[m] = (SPLIT && tv) ? B.Tlo[ot] : 0.f;
      rl[m] = (SPLIT && rv) ? B.Rlo[orr] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < PER; ++m) {
      const int x = tid + NT * m, tt = x / TE, ee = x - tt * TE;
      if (tt < kc) {
        sm.op.f.Th[tt][ee] = th[m];
        sm.op.f.Rh[tt][ee] = rh[m];
        if (SPLIT) {
          sm.op.f.Tl[tt][ee] = tl[m];
          sm.op.f.Rl[tt][ee] = rl[m];
        }
      }
    }
    __syncthreads();
    for (int tt = 0; tt < kc; ++tt) {
      float a[U], al[U], b[U], bl[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        a[u] = sm.op.f.Th[tt][ty + 16 * u];
        al[u] = SPLIT ? sm.op.f.Tl[tt][ty + 16 * u] : 0.f;
      }
#pragma unroll
      for (int v = 0; v < U; ++v) {
        b[v] = sm.op.f.Rh[tt][tx + 16 * v];
        bl[v] = SPLIT ? sm.op.f.Rl[tt][tx + 16 * v] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) {
          if (SPLIT) {
            const float p = __fmul_rn(a[u], b[v]);
            const float pe = __fmaf_rn(a[u], b[v], -p);
            const float cross = __fmaf_rn(al[u], b[v], __fmaf_rn(a[u], bl[v], pe));
            const float s1 = __fadd_rn(sh[u][v], p);
            const float bb = __fsub_rn(s1, sh[u][v]);
            const float e = __fadd_rn(__fsub_rn(sh[u][v], __fsub_rn(s1, bb)), __fsub_rn(p, bb));
            const float lo = __fadd_rn(sl[u][v], __fadd_rn(e, cross));
            const float s2 = __fadd_rn(s1, lo);
            sl[u][v] = __fsub_rn(lo, __fsub_rn(s2, s1));
            sh[u][v] = s2;
          } else {
            sh[u][v] = __fmaf_rn(a[u], b[v], sh[u][v]);
          }
        }
    }
  }
}

// (ah + al) - (bh + bl) as a normalised float-float pair: TwoSum of the high
// words, the low words' difference joins the rounding error, one fast
// renormalisation (11 FP32 operations, no FP64 pipe).  The error is a few
// units of 2^-48 (|a| + |b|), below the chain's own.
__device__ __forceinline__ float2 ff_sub(float ah, float al, float bh, float bl) {
  const float s = __fsub_rn(ah, bh);
  const float v = __fsub_rn(s, ah);
  const float e = __fsub_rn(__fsub_rn(ah, __fsub_rn(s, v)), __fadd_rn(bh, v));
  const float t = __fadd_rn(e, __fsub_rn(al, bl));
  const float hi = __fadd_rn(s, t);
  return make_float2(hi, __fsub_rn(t, __fsub_rn(hi, s)));
}

template <bool HIL, int TE>
__device__ __noinline__ void screen_tile_fp64_t(const InstDev &in, int b, int K, int64_t r0, int nr,
                                                int64_t c0, int nc, Cand *out, ScreenSmem &sm) {
  constexpr int U = TE / 16;  // entries per thread and dimension
  const BondDev &B = in.bond[b];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int wl = b, wr = in.d - b - 2;
  __syncthreads();
  stage_meta(in, b, r0, nr, c0, nc, sm);
  double acc[U][U];
  tile_chain_fp64<TE>(B, K, r0, nr, c0, nc, acc, sm);
  KeyBest best{0ull, LLONG_MAX, -1, -1};
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int rr = ty + 16 * u;
    if (rr >= nr) continue;
#pragma unroll
    for (int v = 0; v < U; ++v) {
      const int cc = tx + 16 * v;
      if (cc >= nc) continue;
      const double A = HIL ? in.hilb[sm.srow[rr] + sm.scol[cc]] : tile_entry(in, sm, wl, wr, rr, cc);
      const double e = __dsub_rn(A, acc[u][v]);
      const uint64_t k = abs_key(e);
      if (best.row < 0 || k >= best.key) {
        const int64_t l = sm.lrow[rr] + sm.lcol[cc];
        if (best.row < 0 || k > best.key || l < best.lin) {
          best.key = k;
          best.lin = l;
          best.row = (int32_t)(r0 + rr);
          best.col = (int32_t)(c0 + cc);
        }
      }
    }
  }
  best = block_best(best, sm.sk, sm.sl, sm.sr, sm.sc);
  if (tid == 0) {
    out->key = best.key;
    out->lin = best.lin;
    out->row = best.row;
    out->col = best.col;
  }
}

__device__ __forceinline__ void screen_tile_fp64(const InstDev &in, int b, int K, int64_t r0,
                                                 int nr, int64_t c0, int nc, int te, Cand *out,
                                                 ScreenSmem &sm) {
  if (te == 32) {
    if (in.gen == 0)
      screen_tile_fp64_t<true, 32>(in, b, K, r0, nr, c0, nc, out, sm);
    else
      screen_tile_fp64_t<false, 32>(in, b, K, r0, nr, c0, nc, out, sm);
  } else {
    if (in.gen == 0)
      screen_tile_fp64_t<true, 64>(in, b, K, r0, nr, c0, nc, out, sm);
    else
      screen_tile_fp64_t<false, 64>(in, b, K, r0, nr, c0, nc, out, sm);
  }
}

// ---------------------------------------------------------------------------
// Stored residual values.  The FP64 form keeps E, the rank-one step's column
// ew and row erow as doubles and carries E by the FP64 FMA of the stored-form
// contract.  The mixed forms keep them as float-float pairs (hi, lo) in the
// same 8 bytes and carry E on the FP32 pipe (about 44 bits; a carried entry
// then costs no FP64 instruction); their screen keys are |hi|.
template <int MIX>
struct SV;
template <>
struct SV<0> {
  using T = double;
  static __device__ __forceinline__ T load(const double *E, int64_t i) { return E[i]; }
  static __device__ __forceinline__ void store(double *E, int64_t i, T v) { E[i] = v; }
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T step(T w, T e, T a) { return __fma_rn(w, e, a); }
  static __device__ __forceinline__ T from(double x) { return x; }
  static __device__ __forceinline__ uint64_t key(T v) { return abs_key(v); }
};
struct SVff {
  using T = float2;
  static __device__ __forceinline__ T load(const double *E, int64_t i) {
    return reinterpret_cast<const float2 *>(E)[i];
  }
  static __device__ __forceinline__ void store(double *E, int64_t i, T v) {
    reinterpret_cast<float2 *>(E)[i] = v;
  }
  static __device__ __forceinline__ T zero() { return make_float2(0.f, 0.f); }
  // a + w e: w.x e.x = p + pe exactly, the cross terms and pe join the low
  // word, TwoSum of the high words, renormalised (12 FP32 operations)
  static __device__ __forceinline__ T step(T w, T e, T a) {
    const float p = __fmul_rn(w.x, e.x);
    const float pe = __fmaf_rn(w.x, e.x, -p);
    const float cr = __fmaf_rn(w.x, e.y, __fmaf_rn(w.y, e.x, pe));
    const float s1 = __fadd_rn(a.x, p);
    const float bb = __fsub_rn(s1, a.x);
    const float er = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s1, bb)), __fsub_rn(p, bb));
    const float lo = __fadd_rn(a.y, __fadd_rn(er, cr));
    const float s2 = __fadd_rn(s1, lo);
    return make_float2(s2, __fsub_rn(lo, __fsub_rn(s2, s1)));
  }
  static __device__ __forceinline__ T from(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(__dsub_rn(x, (double)h)));
  }
  static __device__ __forceinline__ uint64_t key(T v) {
    return (uint64_t)(__float_as_uint(v.x) & 0x7FFFFFFFu);
  }
};
template <>
struct SV<1> : SVff {};
template <>
struct SV<2> : SVff {};

// value of a stored entry as a double (update phase)
__device__ __forceinline__ double sv_get(const InstDev &in, const double *E, int64_t i) {
  if (in.prec == P_FP64) return E[i];
  const float2 v = reinterpret_cast<const float2 *>(E)[i];
  return __dadd_rn((double)v.x, (double)v.y);
}
__device__ __forceinline__ void sv_put(const InstDev &in, double *E, int64_t i, double x) {
  if (in.prec == P_FP64)
    E[i] = x;
  else
    SVff::store(E, i, SVff::from(x));
}

// stored-residual screen of one tile (eq. aca_approx_E).  Entries inside the
// stored extent (row < sr and column < sc) are read from E and, when the bond
// appended a pivot in the last sweep (pend), carried through its rank-one
// step E(a,c) = E(a,c) + ew[a] erow[c] with ew[a] = -(E(a,c*) / E(a*,c*)) and
// erow = E(a*, :).  Entries outside it have just entered the superblock and
// get A - chain(T(a,:), R(:,c)) with the current factors (MIX 0: FP64 chain
// of the contract; 1 / 2: FP32 / float-float chain).  Both are written back
// to E; the tile's best |E| is kept as in the FP64 screen.
template <bool HIL, int TE, int MIX>
__device__ __noinline__ void screen_tile_stored_t(const InstDev &in, int b, int K, int64_t r0,
                                                  int nr, int64_t c0, int nc, int32_t sr,
                                                  int32_t sc, int pend, Cand *out,
                                                  ScreenSmem &sm) {
  using V = SV<MIX>;
  using VT = typename V::T;
  constexpr int U = TE / 16;
  const BondDev &B = in.bond[b];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int wl = b, wr = in.d - b - 2;
  const int64_t ld = B.ldR;
  __syncthreads();
  stage_meta(in, b, r0, nr, c0, nc, sm);
  const bool carried = r0 + nr <= sr && c0 + nc <= sc;
  VT ev[U][U];
  if (carried) {
    // streaming tile: all loads first, then the rank-one step and the stores
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int rr = ty + 16 * u;
#pragma unroll
      for (int v = 0; v < U; ++v) {
        const int cc = tx + 16 * v;
        ev[u][v] = (rr < nr && cc < nc) ? V::load(B.E, (r0 + rr) * ld + c0 + cc) : V::zero();
      }
    }
    if (pend) {
      VT wa[U], er[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        wa[u] = ty + 16 * u < nr ? V::load(B.ew, r0 + ty + 16 * u) : V::zero();
#pragma unroll
      for (int v = 0; v < U; ++v)
        er[v] = tx + 16 * v < nc ? V::load(B.erow, c0 + tx + 16 * v) : V::zero();
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int rr = ty + 16 * u;
#pragma unroll
        for (int v = 0; v < U; ++v) {
          const int cc = tx + 16 * v;
          if (rr < nr && cc < nc) {
            ev[u][v] = V::step(wa[u], er[v], ev[u][v]);
            V::store(B.E, (r0 + rr) * ld + c0 + cc, ev[u][v]);
          }
        }
      }
    }
    __syncthreads();  // publishes the tile metadata
  } else {
    // FP64: acc; mixed: the float-float pair (fh, fl), and E = A - T R is
    // formed in float-float too, so the mixed path leaves the FP64 pipe alone
    double acc[MIX == 0 ? U : 1][MIX == 0 ? U : 1];
    float fh[MIX == 0 ? 1 : U][MIX == 0 ? 1 : U], fl[MIX == 0 ? 1 : U][MIX == 0 ? 1 : U];
    if constexpr (MIX == 0)
      tile_chain_fp64<TE>(B, K, r0, nr, c0, nc, acc, sm);
    else
      tile_chain_ff<TE, MIX == 2>(B, K, r0, nr, c0, nc, fh, fl, sm);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int rr = ty + 16 * u;
      const int64_t a = r0 + rr;
      const bool arow = rr < nr && a < sr;
      const VT wa = (pend && arow) ? V::load(B.ew, a) : V::zero();
#pragma unroll
      for (int v = 0; v < U; ++v) {
        const int cc = tx + 16 * v;
        const int64_t c = c0 + cc;
        if (rr >= nr || cc >= nc) {
          ev[u][v] = V::zero();
          continue;
        }
        VT e;
        if (arow && c < sc) {
          e = V::load(B.E, a * ld + c);
          if (pend) e = V::step(wa, V::load(B.erow, c), e);
        } else if constexpr (MIX == 0) {
          const double A =
              HIL ? in.hilb[sm.srow[rr] + sm.scol[cc]] : tile_entry(in, sm, wl, wr, rr, cc);
          e = __dsub_rn(A, acc[u][v]);
        } else {
          float ah, al;
          if (HIL) {
            ah = in.hilb_hi[sm.srow[rr] + sm.scol[cc]];
            al = in.hilb_lo[sm.srow[rr] + sm.scol[cc]];
          } else {
            split2(tile_entry(in, sm, wl, wr, rr, cc), ah, al);
          }
          e = ff_sub(ah, al, fh[u][v], fl[u][v]);
        }
        V::store(B.E, a * ld + c, e);
        ev[u][v] = e;
      }
    }
  }
  KeyBest best{0ull, LLONG_MAX, -1, -1};
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int rr = ty + 16 * u;
    if (rr >= nr) continue;
#pragma unroll
    for (int v = 0; v < U; ++v) {
      const int cc = tx + 16 * v;
      if (cc >= nc) continue;
      const uint64_t k = V::key(ev[u][v]);
      if (best.row < 0 || k >= best.key) {
        const int64_t l = sm.lrow[rr] + sm.lcol[cc];
        if (best.row < 0 || k > best.key || l < best.lin) {
          best.key = k;
          best.lin = l;
          best.row = (int32_t)(r0 + rr);
          best.col = (int32_t)(c0 + cc);
        }
      }
    }
  }
  best = block_best(best, sm.sk, sm.sl, sm.sr, sm.sc);
  if (tid == 0) {
    out->key = best.key;
    out->lin = best.lin;
    out->row = best.row;
    out->col = best.col;
  }
}

template <int MIX>
__device__ __forceinline__ void screen_tile_stored_m(const InstDev &in, int b, int K, int64_t r0,
                                                     int nr, int64_t c0, int nc, int te,
                                                     int32_t sr, int32_t sc, int pend, Cand *out,
                                                     ScreenSmem &sm) {
  if (te == 32) {
    if (in.gen == 0)
      screen_tile_stored_t<true, 32, MIX>(in, b, K, r0, nr, c0, nc, sr, sc, pend, out, sm);
    else
      screen_tile_stored_t<false, 32, MIX>(in, b, K, r0, nr, c0, nc, sr, sc, pend, out, sm);
  } else {
    if (in.gen == 0)
      screen_tile_stored_t<true, 64, MIX>(in, b, K, r0, nr, c0, nc, sr, sc, pend, out, sm);
    else
      screen_tile_stored_t<false, 64, MIX>(in, b, K, r0, nr, c0, nc, sr, sc, pend, out, sm);
  }
}

// the stored screen of one tile; the mixed forms form the entries new to the
// superblock on the FP32 pipe (FP32 or float-float products), the carried
// ones stay FP64
__device__ __forceinline__ void screen_tile_stored(const InstDev &in, int b, int K, int64_t r0,
                                                   int nr, int64_t c0, int nc, int te, int32_t sr,
                                                   int32_t sc, int pend, Cand *out,
                                                   ScreenSmem &sm) {
  if (in.prec == P_FP64)
    screen_tile_stored_m<0>(in, b, K, r0, nr, c0, nc, te, sr, sc, pend, out, sm);
  else if (in.prec == P_FP32)
    screen_tile_stored_m<1>(in, b, K, r0, nr, c0, nc, te, sr, sc, pend, out, sm);
  else
    screen_tile_stored_m<2>(in, b, K, r0, nr, c0, nc, te, sr, sc, pend, out, sm);
}

// ---------------------------------------------------------------------------
// screen of one tile in FP32 (SPLIT = false) or float-float (SPLIT = true)
// from the (hi, lo) shadows of T and R.  Besides the tile's best |E| it
// bounds the FP64 residual of every entry (MCand), so that the merge can
// prove which tiles cannot hold the FP64 argmax.
//   float-float product: T R = (Th + Tl)(Rh + Rl) ~ Th Rh (exact as p + pl)
//   + (Th Rl + Tl Rh); sums (sh, sl) by TwoSum, renormalised every step.
//   bound, with S = max_a sum_t |T(a,t)|, Rm = max |R(t,c)|, A = max |A|:
//     FP32 : 2 (K + 3) u (A + S Rm),  u = 2^-24
//     split: 4 (3K + 8) u^2 (A + S Rm)
//   plus 4u |E| for the last roundings.
template <bool SPLIT, bool HIL, int TE>
__device__ __noinline__ void screen_tile_mixed_t(const InstDev &in, int b, int K, int64_t r0,
                                                 int nr, int64_t c0, int nc, MCand *out,
                                                 ScreenSmem &sm) {
  constexpr int U = TE / 16;  // entries per thread and dimension
  const BondDev &B = in.bond[b];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int wl = b, wr = in.d - b - 2;
  __syncthreads();
  stage_meta(in, b, r0, nr, c0, nc, sm);
  for (int x = tid; x < BM; x += NT) sm.rowS[x] = 0.f;
  for (int x = tid; x < BN; x += NT) sm.colR[x] = 0.f;
  float sh[U][U], sl[U][U];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < U; ++v) {
      sh[u][v] = 0.f;
      sl[u][v] = 0.f;
    }
  for (int t0 = 0; t0 < K; t0 += KC) {
    const int kc = min(KC, K - t0);
    __syncthreads();
    for (int x = tid; x < kc * TE; x += NT) {
      const int tt = x / TE, rr = x - tt * TE;
      const int64_t o = (int64_t)(t0 + tt) * B.ldT + r0 + rr;
      sm.op.f.Th[tt][rr] = rr < nr ? B.Thi[o] : 0.f;
      if (SPLIT) sm.op.f.Tl[tt][rr] = rr < nr ? B.Tlo[o] : 0.f;
    }
    for (int x = tid; x < kc * TE; x += NT) {
      const int tt = x / TE, cc = x - tt * TE;
      const int64_t o = (int64_t)(t0 + tt) * B.ldR + c0 + cc;
      sm.op.f.Rh[tt][cc] = cc < nc ? B.Rhi[o] : 0.f;
      if (SPLIT) sm.op.f.Rl[tt][cc] = cc < nc ? B.Rlo[o] : 0.f;
    }
    __syncthreads();
    if (tid < BM) {
      float acc = sm.rowS[tid];
      for (int tt = 0; tt < kc; ++tt) acc += fabsf(sm.op.f.Th[tt][tid]);
      sm.rowS[tid] = acc;
    } else if (tid < BM + BN) {
      const int c = tid - BM;
      float m = sm.colR[c];
      for (int tt = 0; tt < kc; ++tt) m = fmaxf(m, fabsf(sm.op.f.Rh[tt][c]));
      sm.colR[c] = m;
    }
    for (int tt = 0; tt < kc; ++tt) {
      float th[U], tl[U], rh[U], rl[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        th[u] = sm.op.f.Th[tt][ty + 16 * u];
        tl[u] = SPLIT ? sm.op.f.Tl[tt][ty + 16 * u] : 0.f;
      }
#pragma unroll
      for (int v = 0; v < U; ++v) {
        rh[v] = sm.op.f.Rh[tt][tx + 16 * v];
        rl[v] = SPLIT ? sm.op.f.Rl[tt][tx + 16 * v] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) {
          if (SPLIT) {
            // th rh = p + pl exactly; the cross terms join pl by FMA
            const float p = __fmul_rn(th[u], rh[v]);
            const float pc = __fmaf_rn(tl[u], rh[v], __fmaf_rn(th[u], rl[v], __fmaf_rn(th[u], rh[v], -p)));
            const float s1 = __fadd_rn(sh[u][v], p);
            const float bb = __fsub_rn(s1, sh[u][v]);
            const float e = __fadd_rn(__fsub_rn(sh[u][v], __fsub_rn(s1, bb)), __fsub_rn(p, bb));
            const float lo = __fadd_rn(sl[u][v], __fadd_rn(e, pc));
            const float s2 = __fadd_rn(s1, lo);
            sl[u][v] = __fsub_rn(lo, __fsub_rn(s2, s1));
            sh[u][v] = s2;
          } else {
            sh[u][v] = __fmaf_rn(th[u], rh[v], sh[u][v]);
          }
        }
    }
  }
  float bv = -1.f, v2 = 0.f, amax = 0.f;
  int64_t bl = LLONG_MAX;
  int32_t brow = -1, bcol = -1;
  bool bad = false;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int rr = ty + 16 * u;
    if (rr >= nr) continue;
#pragma unroll
    for (int v = 0; v < U; ++v) {
      const int cc = tx + 16 * v;
      if (cc >= nc) continue;
      float ah, al;
      if (HIL) {
        ah = in.hilb_hi[sm.srow[rr] + sm.scol[cc]];
        al = in.hilb_lo[sm.srow[rr] + sm.scol[cc]];
      } else {
        split2(tile_entry(in, sm, wl, wr, rr, cc), ah, al);
      }
      const float e = __fadd_rn(__fsub_rn(ah, sh[u][v]), __fsub_rn(al, sl[u][v]));
      const float ae = fabsf(e);
      amax = fmaxf(amax, fabsf(ah));
      if (!(ae <= FLT_MAX)) bad = true;
      const int64_t l = sm.lrow[rr] + sm.lcol[cc];
      if (ae > bv || (ae == bv && l < bl)) {
        v2 = fmaxf(v2, bv);
        bv = ae;
        bl = l;
        brow = (int32_t)(r0 + rr);
        bcol = (int32_t)(c0 + cc);
      } else {
        v2 = fmaxf(v2, ae);
      }
    }
  }
  KeyBest best{brow >= 0 ? (uint64_t)__float_as_uint(bv) : 0ull, bl, brow, bcol};
  best = block_best(best, sm.sk, sm.sl, sm.sr, sm.sc);
  __shared__ int32_t wrow, wcol;
  __shared__ float wval;
  __shared__ int wbad;
  if (tid == 0) {
    wrow = best.row;
    wcol = best.col;
    wval = __uint_as_float((unsigned)best.key);
    wbad = 0;
  }
  __syncthreads();
  if (bad) wbad = 1;
  // the tile's best among the others: every thread's second value, and the
  // thread bests that lost to the winner
  float rest = (brow == wrow && bcol == wcol) ? v2 : fmaxf(fmaxf(bv, 0.f), v2);
  float Smax = 0.f, Rmax = 0.f;
  for (int x = tid; x < nr; x += NT) Smax = fmaxf(Smax, sm.rowS[x]);
  for (int x = tid; x < nc; x += NT) Rmax = fmaxf(Rmax, sm.colR[x]);
  for (int off = 16; off > 0; off >>= 1) {
    rest = fmaxf(rest, __shfl_down_sync(0xffffffffu, rest, off));
    amax = fmaxf(amax, __shfl_down_sync(0xffffffffu, amax, off));
    Smax = fmaxf(Smax, __shfl_down_sync(0xffffffffu, Smax, off));
    Rmax = fmaxf(Rmax, __shfl_down_sync(0xffffffffu, Rmax, off));
  }
  __shared__ float wr4[NT / 32][4];
  const int w = tid >> 5;
  if ((tid & 31) == 0) {
    wr4[w][0] = rest;
    wr4[w][1] = amax;
    wr4[w][2] = Smax;
    wr4[w][3] = Rmax;
  }
  __syncthreads();
  if (tid == 0) {
    for (int i = 1; i < NT / 32; ++i) {
      rest = fmaxf(rest, wr4[i][0]);
      amax = fmaxf(amax, wr4[i][1]);
      Smax = fmaxf(Smax, wr4[i][2]);
      Rmax = fmaxf(Rmax, wr4[i][3]);
    }
    const double u = 5.9604644775390625e-8;  // 2^-24
    const double scale = (double)amax + (double)Smax * (double)Rmax;
    const double eabs = SPLIT ? 4.0 * (3.0 * K + 8.0) * u * u * scale
                              : 2.0 * (K + 3.0) * u * scale;
    out->v = wbad ? INFINITY : wval;
    out->rest = wbad ? INFINITY : rest;
    out->eabs = isfinite(eabs) ? eabs : INFINITY;
    out->lin = best.lin;
    out->row = best.row;
    out->col = best.col;
  }
}

template <bool SPLIT>
__device__ __forceinline__ void screen_tile_mixed(const InstDev &in, int b, int K, int64_t r0,
                                                  int nr, int64_t c0, int nc, int te, MCand *out,
                                                  ScreenSmem &sm) {
  if (te == 32) {
    if (in.gen == 0)
      screen_tile_mixed_t<SPLIT, true, 32>(in, b, K, r0, nr, c0, nc, out, sm);
    else
      screen_tile_mixed_t<SPLIT, false, 32>(in, b, K, r0, nr, c0, nc, out, sm);
  } else {
    if (in.gen == 0)
      screen_tile_mixed_t<SPLIT, true, 64>(in, b, K, r0, nr, c0, nc, out, sm);
    else
      screen_tile_mixed_t<SPLIT, false, 64>(in, b, K, r0, nr, c0, nc, out, sm);
  }
}

// state, screened, add[b] and r[b] of an instance, each word loaded by its
// own thread (one L2 round trip instead of a chain of them)
// control words of an instance read once per phase by the CTA (shared
// memory: per-thread copies would live in local memory, whose lines this
// kernel's large stack frame keeps out of L1)
struct CtrlSnap {
  int32_t state, screened;
  int32_t add[TTC_MAXB], r[TTC_MAXB];
  int32_t old_r[TTC_MAXB];  // r - add: the ranks at the start of the sweep
};

__device__ void snap_ctrl(const Ctrl &cr, int nb, CtrlSnap &out) {
  __syncthreads();
  const int k = threadIdx.x;
  if (k == 0)
    out.state = ld_cg(cr.state);
  else if (k == 1)
    out.screened = ld_cg(cr.screened);
  else if (k < 2 + nb)
    out.add[k - 2] = ld_cg(cr.add[k - 2]);
  else if (k < 2 + 2 * nb)
    out.r[k - 2 - nb] = ld_cg(cr.r[k - 2 - nb]);
  __syncthreads();
  if (k < nb) out.old_r[k] = out.r[k] - out.add[k];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// phase: screen.  Tiles of every (instance, bond) pair that needs a screen
// are numbered consecutively; CTA g takes tiles g, g + G, ...
// Stored-residual instances instead hand out their tiles from a counter,
// tiles new to a superblock (A - T R, r_k FMAs per entry) first and carried
// ones (one load, one FMA, one store per entry) after, so that CTAs with a
// costly tile take fewer cheap ones.  The decide phase after the screen
// clears the counter.

// carried region of bond b: row tiles < tr0 and column tiles < tc0 lie in
// the stored extent (its rows / columns are whole prefix / suffix blocks)
__host__ __device__ __forceinline__ void carried_tiles(const InstDev &in, const TileGeo &g, int b,
                                                       int32_t sr, int32_t sc, int32_t &tr0,
                                                       int32_t &tc0) {
  tr0 = g.pr > 0 ? (sr / (int32_t)in.n[b]) * g.P.tpb : sr / g.te;
  tc0 = g.pc > 0 ? (sc / (int32_t)in.n[b + 1]) * g.Q.tpb : sc / g.te;
}

// bookkeeping of a screen (one thread, from the CTA's staged geometry):
// candidate slots per bond for the merge, and the statistics.  Stored form:
// sr / sc / pend are the stored extents and pending steps, spt the slots per
// tile; recompute form: sr = sc = null.
__device__ void screen_bookkeeping(const InstDev &in, const int32_t *r, const TileGeo *geo,
                                   const int32_t *sr, const int32_t *sc, const int32_t *pend,
                                   int32_t spt) {
  Ctrl &cw = *in.ctrl;
  int64_t entries = 0, fmas = 0, fresh = 0, bytes = 0;
  for (int b = 0; b < in.nb; ++b) {
    cw.ntiles[b] = geo[b].nrt * geo[b].nct * spt;
    const int64_t e = (int64_t)geo[b].rows * geo[b].cols;
    entries += e;
    if (sr) {
      // carried entries cost one FMA when a rank-one step is pending
      const int64_t kept = (int64_t)sr[b] * sc[b];
      fresh += e - kept;
      fmas += (e - kept) * r[b] + (pend[b] ? kept : 0);
      bytes += 8 * e + (pend[b] ? 8 * kept : 0);
    } else {
      fresh += e;
      fmas += e * r[b];
    }
  }
  cw.sweeps += 1;
  cw.entries += entries;
  cw.entries_fresh += fresh;
  cw.stored_bytes += bytes;
  cw.screen_fmas += fmas;
  cw.screened = 1;
}

// A carried tile (TE = 32 or 64 wide) of bond b by one warp: lane l holds
// columns l (and l + 32); rows go in rounds of 32 (TE = 32) or 8 (TE = 64),
// every load of a round issued before its first use.  Then the pending
// rank-one step E(a,c) = fma(ew[a], erow[c], E(a,c)) and its stores, and the
// tile's best |E| (ties: lowest linear index).  The tile lies in one block
// (p, q) of the superblock, where the linear index is
// L.lin[p] + R.lin[q] + i stride_b + j stride_{b+1}: the ties need no loads.
// Eight tiles per CTA are in flight instead of one.
template <int TE, int MIX>
__device__ __noinline__ void screen_carried_warp(const InstDev &in, int b, int64_t r0, int nr,
                                                 int64_t c0, int nc, int pend, Cand *out,
                                                 int spt) {
  using V = SV<MIX>;
  using VT = typename V::T;
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int NC = TE / 32;                // columns per lane
  constexpr int RR = TE == 32 ? 32 : (MIX == 0 ? 8 : 16);  // rows per round
  const BondDev &B = in.bond[b];
  const int lane = threadIdx.x & 31;
  const int64_t ld = B.ldR;
  const int64_t nb0 = in.n[b], nb1 = in.n[b + 1];
  const int64_t p = r0 / nb0, i0 = r0 - p * nb0;
  const int64_t q = c0 / nb1, j0 = c0 - q * nb1;
  const int64_t sb = in.stride[b], sb1 = in.stride[b + 1];
  const int64_t lp = lane == 0 ? left_set(in, b).lin[p] : 0;
  const int64_t rq = lane == 1 ? right_set(in, b).lin[q] : 0;
  VT wa[NC], er[NC];
  bool cok[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    cok[k] = lane + 32 * k < nc;
    wa[k] = (pend && lane + 32 * k < nr) ? V::load(B.ew, r0 + lane + 32 * k) : V::zero();
    er[k] = (pend && cok[k]) ? V::load(B.erow, c0 + lane + 32 * k) : V::zero();
  }
  uint64_t bk = 0;
  int64_t bl = LLONG_MAX;
  int brr = -1, bcc = 0;
  // mixed forms: the rounds stay a loop; unrolled, their float-float steps
  // make a body large enough to compete for the instruction cache with the
  // fresh tiles of the SM's other CTA (the FP64 body is small)
#pragma unroll(MIX == 0 ? TE / RR : 1)
  for (int r1 = 0; r1 < TE; r1 += RR) {
    VT ev[RR][NC];
#pragma unroll
    for (int rr = 0; rr < RR; ++rr)
#pragma unroll
      for (int k = 0; k < NC; ++k)
        ev[rr][k] = (cok[k] && r1 + rr < nr) ? V::load(B.E, (r0 + r1 + rr) * ld + c0 + lane + 32 * k)
                                             : V::zero();
    if (pend) {
#pragma unroll
      for (int rr = 0; rr < RR; ++rr) {
        const int row = r1 + rr;
        VT w;
        if constexpr (MIX == 0) {
          w = __shfl_sync(FULL, wa[row >> 5], row & 31);
        } else {
          w.x = __shfl_sync(FULL, wa[row >> 5].x, row & 31);
          w.y = __shfl_sync(FULL, wa[row >> 5].y, row & 31);
        }
#pragma unroll
        for (int k = 0; k < NC; ++k)
          if (row < nr && cok[k]) {
            ev[rr][k] = V::step(w, er[k], ev[rr][k]);
            V::store(B.E, (r0 + row) * ld + c0 + lane + 32 * k, ev[rr][k]);
          }
      }
    }
    // the lane's best: rows in order, only a larger key replaces within a
    // column (the earlier row has the lower linear index); across its
    // columns the linear index decides
#pragma unroll
    for (int rr = 0; rr < RR; ++rr)
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        const int row = r1 + rr;
        if (row < nr && cok[k]) {
          const uint64_t key = V::key(ev[rr][k]);
          if (brr < 0 || key >= bk) {
            const int64_t l = (i0 + row) * sb + (j0 + lane + 32 * k) * sb1;
            if (brr < 0 || key > bk || l < bl) {
              bk = key;
              bl = l;
              brr = row;
              bcc = lane + 32 * k;
            }
          }
        }
      }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const uint64_t ok = __shfl_xor_sync(FULL, bk, off);
    const int64_t ol = __shfl_xor_sync(FULL, bl, off);
    const int orr = __shfl_xor_sync(FULL, brr, off);
    const int oc = __shfl_xor_sync(FULL, bcc, off);
    if (orr >= 0 && (brr < 0 || ok > bk || (ok == bk && ol < bl))) {
      bk = ok;
      bl = ol;
      brr = orr;
      bcc = oc;
    }
  }
  const int64_t LP = __shfl_sync(FULL, lp, 0), RQ = __shfl_sync(FULL, rq, 1);
  if (lane == 0) {
    out->key = bk;
    out->lin = LP + RQ + bl;
    out->row = (int32_t)(r0 + brr);
    out->col = (int32_t)(c0 + bcc);
    for (int k = 1; k < spt; ++k) out[k] = Cand{0ull, LLONG_MAX, -2, -2};
  }
}

__device__ __forceinline__ void carried_warp(const InstDev &in, int te, int b, int64_t r0, int nr,
                                             int64_t c0, int nc, int pend, Cand *out, int spt) {
  if (in.prec == P_FP64) {
    if (te == 32)
      screen_carried_warp<32, 0>(in, b, r0, nr, c0, nc, pend, out, spt);
    else
      screen_carried_warp<64, 0>(in, b, r0, nr, c0, nc, pend, out, spt);
  } else {
    if (te == 32)
      screen_carried_warp<32, 2>(in, b, r0, nr, c0, nc, pend, out, spt);
    else
      screen_carried_warp<64, 2>(in, b, r0, nr, c0, nc, pend, out, spt);
  }
}

// The stored screen of one instance.  Work items come from two queues:
//   A: tiles new to a superblock (fresh: A - T R, r_k FMAs per entry, FP64
//      pipe or FP32 pipe in the mixed forms), one tile (or quarter) per
//      block item;
//   B: carried tiles (one load, one FMA when a rank-one step is pending, one
//      store per entry: memory-bound).  On bonds cut into subtensor pieces a
//      carried tile lies in one block (p, q) and is screened by one warp, and
//      an item is eight such tiles, one per warp; elsewhere an item is one
//      tile screened by the whole CTA.
// The CTAs of the first half of the SM-spread order (one per SM) start on A,
// the others on B, so that every SM keeps its FP64 / FP32 pipe and its
// memory path busy at once; a CTA whose queue runs dry moves to the other.
// Place s takes the first item of its queue implicitly, later items come
// from the queue's counter, fetched when an item starts so that the atomic's
// round trip overlaps the tile.  The decide phase clears both counters.
constexpr int CW = NT / 32;  // carried warp tiles per item

__device__ void screen_stored_instance(const InstDev &in, const int32_t *r, PhaseSmem &sm) {
  const Ctrl &cr = *in.ctrl;
  int32_t *ctr[2] = {&in.ctrl->steal, &in.ctrl->steal2};
  // per-bond geometry, stored extent and item counts, staged once
  __shared__ TileGeo s_geo[TTC_MAXB];
  __shared__ int32_t s_sr[TTC_MAXB], s_sc[TTC_MAXB], s_pend[TTC_MAXB];
  __shared__ int32_t s_tr0[TTC_MAXB], s_tc0[TTC_MAXB];
  __shared__ int32_t s_warp[TTC_MAXB];  // carried tiles go to single warps
  __shared__ int32_t s_item, s_q;
  __syncthreads();
  if (threadIdx.x < in.nb) {
    const int b = threadIdx.x;
    const TileGeo g = planned_geo(in, cr, b);
    const int32_t sr = ld_cg(cr.st_rows[b]);
    const int32_t sc = ld_cg(cr.st_cols[b]);
    int32_t tr0, tc0;
    carried_tiles(in, g, b, sr, sc, tr0, tc0);
    s_geo[b] = g;
    s_sr[b] = sr;
    s_sc[b] = sc;
    s_pend[b] = ld_cg(cr.e_pend[b]);
    s_tr0[b] = tr0;
    s_tc0[b] = tc0;
    s_warp[b] = g.pr > 0 && g.pc > 0;
  }
  __syncthreads();
  // with fewer fresh tiles than CTAs, fresh tiles go out as quarters
  // (32 x 32) so that their work spreads over four times as many CTAs;
  // candidate slots are then STORED_SLOTS per tile, else one
  int32_t nf = 0, nB = 0;
  for (int b = 0; b < in.nb; ++b) {
    const int32_t nt = s_geo[b].nrt * s_geo[b].nct, nc = s_tr0[b] * s_tc0[b];
    nf += nt - nc;
    nB += s_warp[b] ? (nc + CW - 1) / CW : nc;
  }
  const bool quarters = s_geo[0].te == 64 && nf < (int32_t)gridDim.x;
  const int32_t spt = quarters ? STORED_SLOTS : 1;  // slots per tile
  const int32_t nA = spt * nf;
  const int32_t G = gridDim.x;
  const int32_t qs = ld_cg(cr.qsplit);  // eighths of the CTAs that start on A (0: half)
  const int32_t HA = nA == 0 ? 0 : nB == 0 ? G : qs > 0 ? max(1, min(G - 1, G * qs / 8))
                                                         : (G + 1) / 2;
  const int32_t N[2] = {nA, nB}, H[2] = {HA, G - HA};
  if (blockIdx.x == 0 && threadIdx.x == 0) screen_bookkeeping(in, r, s_geo, s_sr, s_sc, s_pend, spt);
  // thread 0 keeps the queue, whether it has switched, and the next item
  int q0 = s_place < HA ? 0 : 1;
  bool switched = false;
  if (threadIdx.x == 0) {
    int32_t j = q0 == 0 ? s_place : s_place - HA;
    if (j >= N[q0]) {
      switched = true;
      q0 ^= 1;
      j = H[q0] + atomicAdd(ctr[q0], 1);
    }
    s_q = q0;
    s_item = j < N[q0] ? j : -1;
  }
  int32_t nxt = 0;
  for (;;) {
    __syncthreads();
    const int qq = s_q;
    int32_t j = s_item;
    __syncthreads();
    if (j < 0) break;
    if (threadIdx.x == 0) nxt = H[qq] + atomicAdd(ctr[qq], 1);
    if (qq == 0) {
      // a fresh tile (or quarter q of it)
      const int32_t qt = j % spt;
      j /= spt;
      for (int b = 0; b < in.nb; ++b) {
        const TileGeo &g = s_geo[b];
        const int32_t tr0 = s_tr0[b], tc0 = s_tc0[b];
        const int32_t cnt = g.nrt * g.nct - tr0 * tc0;
        if (j >= cnt) {
          j -= cnt;
          continue;
        }
        int32_t tr, tc;
        if (j < tr0 * (g.nct - tc0)) {
          // new columns of the stored rows
          tr = j / (g.nct - tc0);
          tc = tc0 + (j - tr * (g.nct - tc0));
        } else {
          // new rows, every column
          const int32_t u = j - tr0 * (g.nct - tc0);
          tr = tr0 + u / g.nct;
          tc = u - (tr - tr0) * g.nct;
        }
        int64_t r0, c0;
        int nr, nc;
        tile_rows(in, g, b, tr, r0, nr);
        tile_cols(in, g, b, tc, c0, nc);
        Cand *slot = in.cand + in.bond[b].cand_base + (int64_t)(tr * g.nct + tc) * spt;
        if (quarters) {
          // quarter qt of the tile: rows / columns [32 qr, 32 qr + 32)
          const int h = g.te / 2, qr = qt >> 1, qc = qt & 1;
          const int nrq = min(h, nr - h * qr), ncq = min(h, nc - h * qc);
          if (nrq > 0 && ncq > 0)
            screen_tile_stored(in, b, r[b], r0 + h * qr, nrq, c0 + h * qc, ncq, h, s_sr[b],
                               s_sc[b], s_pend[b], slot + qt, sm.s);
          else if (threadIdx.x == 0)
            slot[qt] = Cand{0ull, LLONG_MAX, -2, -2};  // an empty quarter
        } else {
          screen_tile_stored(in, b, r[b], r0, nr, c0, nc, g.te, s_sr[b], s_sc[b], s_pend[b],
                             slot, sm.s);
        }
        break;
      }
    } else {
      // carried tiles: eight warp tiles, or one block tile
      for (int b = 0; b < in.nb; ++b) {
        const TileGeo &g = s_geo[b];
        const int32_t tc0 = s_tc0[b], nc_b = s_tr0[b] * tc0;
        const int32_t cnt = s_warp[b] ? (nc_b + CW - 1) / CW : nc_b;
        if (j >= cnt) {
          j -= cnt;
          continue;
        }
        const int32_t k = s_warp[b] ? j * CW + (int32_t)(threadIdx.x >> 5) : j;
        if (k < nc_b) {
          const int32_t tr = k / tc0, tc = k - tr * tc0;
          int64_t r0, c0;
          int nr, nc;
          tile_rows(in, g, b, tr, r0, nr);
          tile_cols(in, g, b, tc, c0, nc);
          Cand *slot = in.cand + in.bond[b].cand_base + (int64_t)(tr * g.nct + tc) * spt;
          if (!s_warp[b]) {
            screen_tile_stored(in, b, r[b], r0, nr, c0, nc, g.te, s_sr[b], s_sc[b], s_pend[b],
                               slot, sm.s);
            if (threadIdx.x == 0)
              for (int x = 1; x < spt; ++x) slot[x] = Cand{0ull, LLONG_MAX, -2, -2};
          } else {
            carried_warp(in, g.te, b, r0, nr, c0, nc, s_pend[b], slot, spt);
          }
        }
        break;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (nxt >= N[qq]) {
        nxt = -1;
        if (!switched) {
          switched = true;
          q0 = qq ^ 1;
          const int32_t t = H[q0] + atomicAdd(ctr[q0], 1);
          nxt = t < N[q0] ? t : -1;
        }
      } else {
        q0 = qq;
      }
      s_q = q0;
      s_item = nxt;
    }
  }
}

// ---------------------------------------------------------------------------
// Alg. 1 with a random sample set L (recompute form, FP64).  Per screen t
// and bond b, samples j < nl are the superblock entries
//   a = floor(x rows / 2^64), c = floor(x' cols / 2^64),
//   x = SplitMix64(seed) output 2i, x' = output 2i+1, i = (t nb + b) nl + j;
// their argmax (lowest linear index on ties) is refined by whole-column and
// whole-row scans (the while loop of Alg. 1) in the refinement phases.

// column-major linear index of superblock entry (a, c) of bond b
__device__ __forceinline__ int64_t entry_lin(const InstDev &in, int b, int64_t a, int64_t c) {
  const int64_t nb0 = in.n[b], nb1 = in.n[b + 1];
  const int64_t p = a / nb0, i = a - p * nb0;
  const int64_t q = c / nb1, j = c - q * nb1;
  return left_set(in, b).lin[p] + i * in.stride[b] + j * in.stride[b + 1] +
         right_set(in, b).lin[q];
}

// E(a,c) = A(a,c) - chain(T(a,:), R(:,c)) with K terms: the contract's residual
__device__ __forceinline__ double residual_at(const InstDev &in, int b, int K, int64_t a,
                                              int64_t c) {
  const BondDev &B = in.bond[b];
  return __dsub_rn(sb_entry(in, b, a, c), chain(B.T + a, B.ldT, B.R + c, B.ldR, K));
}

__device__ __forceinline__ void take_key(KeyBest &best, double e, int64_t lin, int64_t a,
                                         int64_t c) {
  const uint64_t k = abs_key(e);
  if (best.row < 0 || k > best.key || (k == best.key && lin < best.lin)) {
    best.key = k;
    best.lin = lin;
    best.row = (int32_t)a;
    best.col = (int32_t)c;
  }
}

// the CTA's best of its share of the samples of every bond, into the bond's
// slot blockIdx.x (thread x of the grid takes samples x, x + G NT, ...)
__device__ void screen_sampled_instance(const InstDev &in, const int32_t *r, int64_t t,
                                        PhaseSmem &sm) {
  const int64_t NTOT = (int64_t)gridDim.x * NT;
  const int64_t gt = (int64_t)blockIdx.x * NT + threadIdx.x;
  for (int b = 0; b < in.nb; ++b) {
    const int64_t rows = rows_of(in, r, b), cols = cols_of(in, r, b);
    KeyBest best{0ull, LLONG_MAX, -1, -1};
    for (int64_t j = gt; j < in.nl; j += NTOT) {
      const uint64_t i = (uint64_t)((t * in.nb + b) * in.nl + j);
      const int64_t a = (int64_t)__umul64hi(splitmix64_at(in.lseed, 2 * i), (uint64_t)rows);
      const int64_t c = (int64_t)__umul64hi(splitmix64_at(in.lseed, 2 * i + 1), (uint64_t)cols);
      take_key(best, residual_at(in, b, r[b], a, c), entry_lin(in, b, a, c), a, c);
    }
    best = block_best(best, sm.s.sk, sm.s.sl, sm.s.sr, sm.s.sc);
    if (threadIdx.x == 0) {
      Cand *slot = in.cand + in.bond[b].cand_base + blockIdx.x;
      *slot = best.row >= 0 ? Cand{best.key, best.lin, best.row, best.col}
                            : Cand{0ull, LLONG_MAX, -2, -2};
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Ctrl &cw = *in.ctrl;
    int64_t fmas = 0;
    for (int b = 0; b < in.nb; ++b) {
      cw.ntiles[b] = gridDim.x;
      fmas += in.nl * r[b];
    }
    cw.sweeps += 1;
    cw.entries += in.nl * in.nb;
    cw.entries_fresh += in.nl * in.nb;
    cw.screen_fmas += fmas;
    cw.screened = 1;
  }
}

__device__ void phase_screen(const RunArgs &ra, PhaseSmem &sm) {
  __shared__ CtrlSnap snap;
  const int32_t G = gridDim.x;
  int64_t base = 0;
  int32_t boff = 0;  // base mod G
  for (int ii = 0; ii < ra.count; ++ii) {
    const InstDev &in = inst(ra, ii);
    const Ctrl &cr = *in.ctrl;
    snap_ctrl(cr, in.nb, snap);
    if (blockIdx.x == 0 && threadIdx.x == 0)
      in.ctrl->dkind = snap.state == ST_SCREEN ? DK_BONDS : snap.state == ST_VERIFY ? DK_VERIFY
                                                                                   : DK_NONE;
    if (snap.state != ST_SCREEN) continue;
    const int32_t *r = snap.r;
    if (in.stored) {
      screen_stored_instance(in, r, sm);
      continue;
    }
    if (in.nl > 0) {
      // the screen counter is advanced by the decide phase, never here
      screen_sampled_instance(in, r, ld_cg(cr.screen_t), sm);
      continue;
    }
    // every bond's tile geometry, one bond per thread
    __shared__ TileGeo s_pg[TTC_MAXB];
    __syncthreads();
    if (threadIdx.x < in.nb) s_pg[threadIdx.x] = planned_geo(in, cr, threadIdx.x);
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0)
      screen_bookkeeping(in, r, s_pg, nullptr, nullptr, nullptr, 1);
    for (int b = 0; b < in.nb; ++b) {
      const TileGeo &g = s_pg[b];
      const int32_t nt = g.nrt * g.nct;
      for (int32_t lt = ((int32_t)blockIdx.x - boff + G) % G; lt < nt; lt += G) {
        const int32_t tr = lt / g.nct, tc = lt - tr * g.nct;
        int64_t r0, c0;
        int nr, nc;
        tile_rows(in, g, b, tr, r0, nr);
        tile_cols(in, g, b, tc, c0, nc);
        if (in.prec == P_SPLIT)
          screen_tile_mixed<true>(in, b, r[b], r0, nr, c0, nc, g.te,
                                  in.mcand + in.bond[b].cand_base + lt, sm.s);
        else if (in.prec == P_FP32)
          screen_tile_mixed<false>(in, b, r[b], r0, nr, c0, nc, g.te,
                                   in.mcand + in.bond[b].cand_base + lt, sm.s);
        else
          screen_tile_fp64(in, b, r[b], r0, nr, c0, nc, g.te, in.cand + in.bond[b].cand_base + lt,
                           sm.s);
      }
      base += nt;
      boff = (int32_t)((boff + nt) % G);
    }
  }
}

// ---------------------------------------------------------------------------
// decide: append the pivot (a*, c*) to bond b (block-wide).  I_{<=k} gets
// (alpha*, i*), J_{>k} gets (j*, beta*) (eq. nestedpivots); the history of
// step z keeps c_z = R(:, c*), T(a*, :) and delta; U = P^{-1} is bordered
// by [[U + d U a b U, -d U a], [-d b U, d]] (Sec. 3.1.1).
__device__ bool append_pivot(const InstDev &in, Ctrl &cr, int b, int64_t as, int64_t cs, int z,
                             DecideSmem &sm) {
  const BondDev &B = in.bond[b];
  const int cap = B.cap;
  const int tid = threadIdx.x;
  const int64_t nb0 = in.n[b], nb1 = in.n[b + 1];
  const int64_t p = as / nb0, i = as - p * nb0;
  const int64_t q = cs / nb1, j = cs - q * nb1;
  const SetDev &L = left_set(in, b);
  const SetDev &Rset = right_set(in, b);
  const bool hil = in.gen == 0;
  const bool ustage = z <= DEC_US;
  // one round of independent loads: warp 1 appends the index sets (a lane
  // per index), threads t < z gather the history (R(t, c*), T(a*, t)) and
  // the pivot columns' index sums (Hilbert) or coordinates, the rest stage U
  if (tid >= 32 && tid < 64) {
    const int lane = tid - 32;
    const int wl = b, wj = in.d - 1 - b;
    if (lane < wl) B.I.idx[(int64_t)z * (wl + 1) + lane] = L.idx[p * wl + lane];
    if (lane == wl) B.I.idx[(int64_t)z * (wl + 1) + wl] = (int32_t)i;
    if (lane == 0) B.J.idx[(int64_t)z * wj] = (int32_t)j;
    if (lane >= 1 && lane < wj) B.J.idx[(int64_t)z * wj + lane] = Rset.idx[q * (wj - 1) + lane - 1];
    if (lane == 16) B.I.lin[z] = L.lin[p] + i * in.stride[b];
    if (lane == 17) B.I.sum[z] = L.sum[p] + (int32_t)i;
    if (lane == 18) B.J.lin[z] = j * in.stride[b + 1] + Rset.lin[q];
    if (lane == 19) B.J.sum[z] = (int32_t)j + Rset.sum[q];
    if (lane == 20) {
      B.prow[z] = (int32_t)as;
      B.pcol[z] = (int32_t)cs;
    }
  }
  double *hc = B.hc + (int64_t)z * cap;
  double *hp = B.hpiv + (int64_t)z * cap;
  for (int t = tid; t < z; t += NT) {
    const double c = B.R[(int64_t)t * B.ldR + cs], v = B.T[(int64_t)t * B.ldT + as];
    sm.key[t] = hil ? B.J.sum[t] : B.pcol[t];
    hc[t] = c;
    hp[t] = v;
    sm.hcs[t] = c;
    sm.hps[t] = v;
  }
  if (tid == NT - 1) sm.lsum = L.sum[p] + (int32_t)i;
  if (tid == NT - 2) sm.rsum = Rset.sum[q] + (int32_t)j;
  if (ustage)
    for (int x = tid; x < z * z; x += NT) {
      const int t = x / z, u = x - t * z;
      sm.us[x] = B.U[(int64_t)t * cap + u];
    }
  __syncthreads();
  // the pivot row's entries A(a*, c_t) and A(a*, c*)
  for (int t = tid; t < z; t += NT)
    sm.brow[t] = hil ? in.hilb[sm.lsum + sm.key[t]] : sb_entry(in, b, as, sm.key[t]);
  if (tid == NT - 1) sm.apiv = hil ? in.hilb[sm.lsum + sm.rsum] : sb_entry(in, b, as, cs);
  __syncthreads();
  if (tid == 0) {
    const double piv = __dsub_rn(sm.apiv, chain(sm.hps, 1, sm.hcs, 1, z));
    const double delta = 1.0 / piv;
    sm.delta = delta;
    // 1: a usable pivot; 0: the residual formed afresh at the pivot is zero
    // (or its reciprocal overflows), so the screened value was rounding
    // noise and the bond takes no pivot; -1: not finite
    sm.flag = isfinite(delta) ? 1 : isfinite(piv) ? 0 : -1;
    B.delta[z] = delta;
  }
  __syncthreads();
  if (sm.flag != 1) return false;
  const double delta = sm.delta;
  double *U = B.U;
  const double *Ur = ustage ? sm.us : U;
  const int64_t ldu = ustage ? z : cap;
  // U a and b U side by side: lanes [0, z) take the rows, [z, 2z) the columns
  for (int x = tid; x < 2 * z; x += NT) {
    if (x < z)
      sm.ua[x] = chain(Ur + (int64_t)x * ldu, 1, sm.hcs, 1, z);
    else
      sm.bu[x - z] = chain(sm.brow, 1, Ur + (x - z), ldu, z);
  }
  __syncthreads();
  for (int x = tid; x < z * z; x += NT) {
    const int t = x / z, u = x - t * z;
    const double du = __dmul_rn(delta, sm.ua[t]);
    U[(int64_t)t * cap + u] = __fma_rn(du, sm.bu[u], Ur[(int64_t)t * ldu + u]);
  }
  for (int t = tid; t < z; t += NT) {
    U[(int64_t)t * cap + z] = -__dmul_rn(delta, sm.ua[t]);
    U[(int64_t)z * cap + t] = -__dmul_rn(delta, sm.bu[t]);
  }
  if (tid == 0) U[(int64_t)z * cap + z] = delta;
  __syncthreads();
  return true;
}

// FP64 residual of superblock entry (a, c) with the contract's chain
__device__ double residual64(const InstDev &in, const Ctrl &cr, int b, int64_t a, int64_t c) {
  if (a < 0 || c < 0) return __longlong_as_double(0x7FF8000000000000ll);  // no entry: NaN
  const BondDev &B = in.bond[b];
  double acc = 0.0;
  const int K = ld_cg(cr.r[b]);
  for (int t = 0; t < K; ++t)
    acc = __fma_rn(B.T[(int64_t)t * B.ldT + a], B.R[(int64_t)t * B.ldR + c], acc);
  return __dsub_rn(sb_entry(in, b, a, c), acc);
}

__device__ void fail_instance(Ctrl &cr, int32_t status) {
  if (threadIdx.x == 0) {
    cr.status = status;
    cr.state = ST_DONE;
  }
}

// stored-residual form: the rank-one step of eq. aca_approx_E for pivot
// (a*, c*) of bond b is applied by the next screen to the stored extent:
//   ew[a] = -(E(a,c*) / E(a*,c*)) (exactly -1 at a*), erow[c] = E(a*,c);
// the decide phase only marks it pending, the update phase (every CTA, as
// thread items) fills ew and erow from E, which the screen left unchanged
__device__ void stored_step(Ctrl &cr, int b) {
  if (threadIdx.x == 0) cr.e_pend[b] = 1;
}

// stop test and pivot append for bond b on its merged best (block-wide): add
// the pivot while the best |E| exceeds tau * rms(X) and the cap allows.  The
// bond's own rank is the only rank this touches, so bonds decide in parallel.
// The values come from the caller (every thread holds the same ones).
__device__ void finalize_bond_v(const InstDev &in, Ctrl &cr, int b, DecideSmem &sm, uint64_t key,
                                int32_t row, int32_t col, int32_t rb, double tau, double xrms,
                                int32_t maxr) {
  __syncthreads();
  if (key > KEY_INF || row < 0) {
    fail_instance(cr, 4);  // TTC_ERR_NONFINITE
    if (threadIdx.x == 0) cr.add[b] = 0;
    __syncthreads();
    return;
  }
  const double v = __longlong_as_double((long long)key);
  const bool add = v > tau * xrms && v > 0.0 && rb < maxr;
  bool ok = true;
  if (add) ok = append_pivot(in, cr, b, row, col, rb, sm);
  if (add && ok && in.stored) stored_step(cr, b);
  if (add && !ok && sm.flag < 0) fail_instance(cr, 4);
  __syncthreads();
  if (threadIdx.x == 0) {
    cr.add[b] = (add && ok) ? 1 : 0;
    cr.r[b] = rb + ((add && ok) ? 1 : 0);
  }
  __syncthreads();
}

// the same with the best and the words read from the control block
__device__ void finalize_bond(const InstDev &in, Ctrl &cr, int b, DecideSmem &sm) {
  const uint64_t key = ld_cg(cr.best_key[b]);
  const int32_t row = ld_cg(cr.best_row[b]), col = ld_cg(cr.best_col[b]);
  finalize_bond_v(in, cr, b, sm, key, row, col, ld_cg(cr.r[b]), ld_cg(cr.tau), ld_cg(cr.xrms),
                  ld_cg(cr.maxr[b]));
}

// FP64 decide item of bond b: the control words it needs in one round of
// parallel loads, the merge of the tile candidates (the Allgather of Alg. 3),
// then the stop test on the merged best as it stands
__device__ void decide_bond_fp64(const InstDev &in, Ctrl &cr, int b, DecideSmem &sm) {
  const int tid = threadIdx.x;
  if (tid == 0) sm.q_nt = ld_cg(cr.ntiles[b]);
  if (tid == 1) sm.q_r = ld_cg(cr.r[b]);
  if (tid == 2) sm.q_tau = ld_cg(cr.tau);
  if (tid == 3) sm.q_xrms = ld_cg(cr.xrms);
  if (tid == 4) sm.q_maxr = ld_cg(cr.maxr[b]);
  if (tid == 5 && in.stored) sm.q_prow = ld_cg(cr.plan_rows[b]);
  if (tid == 6 && in.stored) sm.q_pcol = ld_cg(cr.plan_cols[b]);
  __syncthreads();
  if (in.stored && tid == 0) {
    // the screen just stored every entry of the superblock and applied the
    // pending rank-one step
    cr.st_rows[b] = sm.q_prow;
    cr.st_cols[b] = sm.q_pcol;
    cr.e_pend[b] = 0;
    if (b == 0) cr.steal = cr.steal2 = 0;  // item counters of the next screen
  }
  const int64_t nt = sm.q_nt;
  KeyBest best{0ull, LLONG_MAX, -1, -1};
  const Cand *cand = in.cand + in.bond[b].cand_base;
  int bad = 0;
  // four slots' loads in flight before their compares
  int64_t t = tid;
  for (; t + 3 * NT < nt; t += 4 * NT) {
    KeyBest o[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const Cand &c = cand[t + u * NT];
      o[u] = KeyBest{c.key, c.lin, c.row, c.col};
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      bad += o[u].row == -1;  // -2 marks a slot left empty on purpose
      kb_take(best, o[u]);
    }
  }
  for (; t < nt; t += NT) {
    KeyBest o{cand[t].key, cand[t].lin, cand[t].row, cand[t].col};
    bad += o.row == -1;
    kb_take(best, o);
  }
  if (bad) atomicAdd((unsigned long long *)&cr.unscreened, (unsigned long long)bad);
  best = block_best(best, sm.rk, sm.rl, sm.rr, sm.rc);
  if (tid == 0) {
    cr.best_key[b] = best.key;
    cr.best_lin[b] = best.lin;
    cr.best_row[b] = best.row;
    cr.best_col[b] = best.col;
    sm.rk[0] = best.key;
    sm.rr[0] = best.row;
    sm.rc[0] = best.col;
  }
  __syncthreads();
  finalize_bond_v(in, cr, b, sm, sm.rk[0], sm.rr[0], sm.rc[0], sm.q_r, sm.q_tau, sm.q_xrms,
                  sm.q_maxr);
}

constexpr int RS_K = 8;  // candidates re-scored per bond in the mixed stored form

// The k best (k <= RS_K) of the lanes' sorted lists loc[0..L-1]: k rounds of
// a butterfly argmax of the list heads, the winning lane popping its head;
// lane j < k returns the j-th (the others an empty candidate).
template <int L>
__device__ KeyBest warp_topk(KeyBest (&loc)[L], int k) {
  const int lane = threadIdx.x & 31;
  KeyBest mine{0ull, LLONG_MAX, -1, -1};
  for (int j = 0; j < k; ++j) {
    KeyBest w = loc[0];
    for (int off = 16; off > 0; off >>= 1) {
      KeyBest o;
      o.key = __shfl_xor_sync(0xffffffffu, w.key, off);
      o.lin = __shfl_xor_sync(0xffffffffu, w.lin, off);
      o.row = __shfl_xor_sync(0xffffffffu, w.row, off);
      o.col = __shfl_xor_sync(0xffffffffu, w.col, off);
      if (o.row >= 0 && (w.row < 0 || key_better(o.key, o.lin, w.key, w.lin))) w = o;
    }
    if (lane == j) mine = w;
    if (w.row >= 0 && loc[0].row == w.row && loc[0].col == w.col) {
#pragma unroll
      for (int q = 0; q + 1 < L; ++q) loc[q] = loc[q + 1];
      loc[L - 1] = KeyBest{0ull, LLONG_MAX, -1, -1};
    }
  }
  return mine;
}

// a candidate slot read through L2 (other SMs wrote it in this launch)
__device__ __forceinline__ Cand ld_cand(const Cand *p) {
  Cand c;
  c.key = __ldcg(&p->key);
  c.lin = __ldcg(&p->lin);
  const int2 rc = __ldcg(reinterpret_cast<const int2 *>(&p->row));
  c.row = rc.x;
  c.col = rc.y;
  return c;
}

// The k best (k <= RS_K; key, then lowest linear index) of slots [t0, t1)
// into sm.skey / slin / srow / scol [0, k), missing ones with row -1;
// block-wide.  Up to 2 NT slots: every slot's rank is the number of better
// slots (the slots are distinct entries).  More: every thread keeps its own
// k best in one pass, each warp merges its lanes' lists, one warp the warps'.
__device__ void topk_of_slots(const Cand *src, int64_t t0, int64_t t1, int k, DecideSmem &sm,
                              int &bad) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t m = t1 - t0;
  if (tid < RS_K) sm.srow[tid] = -1;
  if (m <= 2 * NT) {
    Cand c[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t i = tid + u * NT;
      c[u] = i < m ? ld_cand(src + t0 + i) : Cand{0ull, LLONG_MAX, -2, -2};
      bad += c[u].row == -1;
      const bool v = c[u].row >= 0;
      sm.tk[i] = v ? c[u].key : 0ull;
      sm.tl[i] = v ? c[u].lin : LLONG_MAX;  // never better than a real slot
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (c[u].row < 0) continue;
      int rank = 0;
      for (int j = 0; j < (int)m; ++j) rank += key_better(sm.tk[j], sm.tl[j], c[u].key, c[u].lin);
      if (rank < k) {
        sm.skey[rank] = c[u].key;
        sm.slin[rank] = c[u].lin;
        sm.srow[rank] = c[u].row;
        sm.scol[rank] = c[u].col;
      }
    }
    __syncthreads();
    return;
  }
  KeyBest loc[RS_K];
#pragma unroll
  for (int j = 0; j < RS_K; ++j) loc[j] = KeyBest{0ull, LLONG_MAX, -1, -1};
  for (int64_t t = t0 + tid; t < t1; t += NT) {
    const Cand c = ld_cand(src + t);
    bad += c.row == -1;
    if (c.row < 0) continue;
    // most slots lose to the list's last entry: one comparison
    if (k == RS_K && loc[RS_K - 1].row >= 0 &&
        !key_better(c.key, c.lin, loc[RS_K - 1].key, loc[RS_K - 1].lin))
      continue;
    KeyBest o{c.key, c.lin, c.row, c.col};
    // insertion into the sorted list loc[0..k-1]
#pragma unroll
    for (int j = 0; j < RS_K; ++j) {
      if (j >= k) break;
      if (loc[j].row < 0 || key_better(o.key, o.lin, loc[j].key, loc[j].lin)) {
        const KeyBest tmp = loc[j];
        loc[j] = o;
        o = tmp;
        if (o.row < 0) break;
      }
    }
  }
  const KeyBest wb = warp_topk<RS_K>(loc, k);
  __syncthreads();  // the srow marks above are written before warp 0's results
  if (lane < RS_K) {
    sm.wk[warp * RS_K + lane] = wb.key;
    sm.wl[warp * RS_K + lane] = wb.lin;
    sm.wr[warp * RS_K + lane] = wb.row;
    sm.wc[warp * RS_K + lane] = wb.col;
  }
  __syncthreads();
  if (warp == 0) {
    KeyBest l2[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = lane + 32 * h;
      l2[h] = i < NT / 32 * RS_K ? KeyBest{sm.wk[i], sm.wl[i], sm.wr[i], sm.wc[i]}
                                 : KeyBest{0ull, LLONG_MAX, -1, -1};
    }
    if (l2[1].row >= 0 && (l2[0].row < 0 || key_better(l2[1].key, l2[1].lin, l2[0].key, l2[0].lin))) {
      const KeyBest tmp = l2[0];
      l2[0] = l2[1];
      l2[1] = tmp;
    }
    const KeyBest g = warp_topk<2>(l2, k);
    if (lane < k) {
      sm.skey[lane] = g.key;
      sm.slin[lane] = g.lin;
      sm.srow[lane] = g.row;
      sm.scol[lane] = g.col;
    }
  }
  __syncthreads();
}

// Mixed stored form, decide item (bond b, part of P): the part takes the k
// best of its share of the tile slots by stored |E| (k = topk, at most RS_K;
// entries new to the superblock formed on the FP32 pipe) into the bond's
// partial results, the Allgather of Alg. 3.  The last part to finish takes
// the k best of the partials, re-scores them in FP64 as A - chain(T(a,:),
// R(:,c)) with the current factors, and takes the best FP64 value (same tie
// rule) to the stop test and the pivot step.
__device__ __noinline__ void decide_bond_rescore(const InstDev &in, Ctrl &cr, int b, int part,
                                                 int P, DecideSmem &sm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = max(1, min(in.topk, RS_K));
  if (tid == 0) sm.q_nt = ld_cg(cr.ntiles[b]);
  if (tid == 1) sm.q_r = ld_cg(cr.r[b]);
  if (tid == 2) sm.q_tau = ld_cg(cr.tau);
  if (tid == 3) sm.q_xrms = ld_cg(cr.xrms);
  if (tid == 4) sm.q_maxr = ld_cg(cr.maxr[b]);
  if (tid == 5) sm.q_prow = ld_cg(cr.plan_rows[b]);
  if (tid == 6) sm.q_pcol = ld_cg(cr.plan_cols[b]);
  __syncthreads();
  const int64_t nt = sm.q_nt, L = (nt + P - 1) / P;
  const int64_t t0 = min(nt, (int64_t)part * L), t1 = min(nt, t0 + L);
  const Cand *cand = in.cand + in.bond[b].cand_base;
  Cand *pb = in.refine_cand + in.bond[b].cand_base;  // the parts' results, [P][k]
  int bad = 0;
  topk_of_slots(cand, t0, t1, k, sm, bad);
  if (P > 1) {
    if (tid < k)
      pb[part * k + tid] = sm.srow[tid] >= 0
                               ? Cand{sm.skey[tid], sm.slin[tid], sm.srow[tid], sm.scol[tid]}
                               : Cand{0ull, LLONG_MAX, -2, -2};
    // the last of the P parts to arrive finishes the bond
    __syncthreads();
    if (tid == 0) {
      __threadfence();  // the part's results before its arrival
      sm.last = atomicAdd(&cr.dcount[b], 1) == P - 1;
      if (sm.last) {
        cr.dcount[b] = 0;
        __threadfence();  // the other parts' results after theirs
      }
    }
    __syncthreads();
    if (!sm.last) {
      if (bad) atomicAdd((unsigned long long *)&cr.unscreened, (unsigned long long)bad);
      return;
    }
    topk_of_slots(pb, 0, (int64_t)P * k, k, sm, bad);
  }
  if (tid == 0) {
    // the screen just stored every entry of the superblock and applied the
    // pending rank-one step
    cr.st_rows[b] = sm.q_prow;
    cr.st_cols[b] = sm.q_pcol;
    cr.e_pend[b] = 0;
    if (b == 0) cr.steal = cr.steal2 = 0;  // item counters of the next screen
  }
  if (bad) atomicAdd((unsigned long long *)&cr.unscreened, (unsigned long long)bad);
  // FP64 re-score of the k candidates, a lane each of warp 0 (the chains run
  // side by side instead of queueing warps on the SM's FP64 units)
  if (warp == 0 && lane < k && sm.srow[lane] >= 0)
    sm.skey[lane] = abs_key(residual_at(in, b, sm.q_r, sm.srow[lane], sm.scol[lane]));
  __syncthreads();
  if (tid == 0) {
    KeyBest best{0ull, LLONG_MAX, -1, -1};
    for (int j = 0; j < k; ++j) {
      KeyBest o{sm.skey[j], sm.slin[j], sm.srow[j], sm.scol[j]};
      kb_take(best, o);
    }
    cr.best_key[b] = best.key;
    cr.best_lin[b] = best.lin;
    cr.best_row[b] = best.row;
    cr.best_col[b] = best.col;
    atomicAdd((unsigned long long *)&cr.tiles_refined, (unsigned long long)min((int64_t)k, nt));
    sm.rk[0] = best.key;
    sm.rr[0] = best.row;
    sm.rc[0] = best.col;
  }
  __syncthreads();
  finalize_bond_v(in, cr, b, sm, sm.rk[0], sm.rr[0], sm.rc[0], sm.q_r, sm.q_tau, sm.q_xrms,
                  sm.q_maxr);
}

// mixed forms, part 1 for bond b: re-score the top-k tile bests in FP64,
// then queue for the FP64 refinement every tile whose bound reaches the best
// exact value (when that exceeds the threshold theta: the tile could hold the
// FP64 argmax, or an equal residual with a lower index) or exceeds theta
// (otherwise: the tile could hold an entry that must become a pivot).
__device__ void merge_bond_mixed(const InstDev &in, Ctrl &cr, int b, DecideSmem &sm) {
  __syncthreads();
  if (threadIdx.x == 0) sm.flag = 0;
  __syncthreads();
  const int64_t nt = ld_cg(cr.ntiles[b]);
  const MCand *mc = in.mcand + in.bond[b].cand_base;
  int32_t *list = in.refine_list + 2 * in.bond[b].cand_base;
  const int k = (int)min((int64_t)min(in.topk, TOPK_MAX), nt);
  // one pass: every thread keeps its k best tiles, the block merges them
  KeyBest loc[TOPK_MAX];
  for (int j = 0; j < k; ++j) loc[j] = KeyBest{0ull, LLONG_MAX, -1, -1};
  int bad = 0, badtile = 0;
  for (int64_t t = threadIdx.x; t < nt; t += NT) {
    const float v = mc[t].v;
    if (mc[t].row < 0) {
      // never written (NaN sentinel): count, do not use; written without an
      // entry (every residual of the tile non-finite): the instance fails
      if (!(v == v)) ++bad; else ++badtile;
      continue;
    }
    KeyBest o{(v == v) ? (uint64_t)__float_as_uint(v) : 0xFFFFFFFFull, mc[t].lin, 0, (int32_t)t};
    for (int j = 0; j < k; ++j) {
      if (loc[j].row < 0 || key_better(o.key, o.lin, loc[j].key, loc[j].lin)) {
        const KeyBest tmp = loc[j];
        loc[j] = o;
        o = tmp;
        if (o.row < 0) break;
      }
    }
  }
  if (bad) atomicAdd((unsigned long long *)&cr.unscreened, (unsigned long long)bad);
  if (badtile) atomicExch(&sm.flag, 1);
  for (int j = 0; j < k; ++j) {
    // the block's j-th best: the best head among the threads' lists
    KeyBest head = loc[0];
    KeyBest win = block_best(head, sm.rk, sm.rl, sm.rr, sm.rc);
    if (threadIdx.x == 0) sm.sel[j] = win.row >= 0 ? win.col : -1;
    __syncthreads();
    if (loc[0].row >= 0 && loc[0].col == sm.sel[j]) {
      for (int q = 0; q + 1 < k; ++q) loc[q] = loc[q + 1];
      loc[k - 1] = KeyBest{0ull, LLONG_MAX, -1, -1};
    }
    __syncthreads();
  }
  if (sm.flag) {
    // a tile without a finite residual: the FP64 screen would report it
    fail_instance(cr, 4);  // TTC_ERR_NONFINITE
    if (threadIdx.x == 0) {
      cr.best_key[b] = KEY_INF + 1;
      cr.best_row[b] = -1;
      cr.nrefine_bond[b] = 0;
      cr.pending[b] = 1;
    }
    __syncthreads();
    return;
  }
  if (threadIdx.x < k) {
    const int32_t t = sm.sel[threadIdx.x];
    if (t >= 0) {
      const MCand &c = mc[t];
      sm.skey[threadIdx.x] = abs_key(residual64(in, cr, b, c.row, c.col));
      sm.slin[threadIdx.x] = c.lin;
      sm.srow[threadIdx.x] = c.row;
      sm.scol[threadIdx.x] = c.col;
    } else {
      sm.skey[threadIdx.x] = 0ull;
      sm.slin[threadIdx.x] = LLONG_MAX;
      sm.srow[threadIdx.x] = -1;
      sm.scol[threadIdx.x] = -1;
    }
  }
  if (threadIdx.x == 0) sm.cnt = 0;
  __syncthreads();
  KeyBest vb{0ull, LLONG_MAX, -1, -1};
  for (int j = 0; j < k; ++j) {
    KeyBest o{sm.skey[j], sm.slin[j], sm.srow[j], sm.scol[j]};
    kb_take(vb, o);
  }
  const double vstar = __longlong_as_double((long long)(vb.key > KEY_INF ? KEY_INF : vb.key));
  const double theta = ld_cg(cr.tau) * ld_cg(cr.xrms);
  const bool strict = !(vstar > theta);
  const double thr = strict ? theta : vstar;
  const double g = 1.0 + 4.0 * 5.9604644775390625e-8;
  for (int64_t t = threadIdx.x; t < nt; t += NT) {
    const MCand &c = mc[t];
    bool taken = false;
    for (int q = 0; q < k; ++q) taken |= sm.sel[q] == (int32_t)t;
    if (c.row < 0 && !(c.v == c.v)) continue;  // never written (counted above)
    const double top = taken ? (double)c.rest : fmax((double)c.v, (double)c.rest);
    const double U = top * g + c.eabs;
    if (!(U == U) || (strict ? U > thr : U >= thr)) {
      const int slot = atomicAdd(&sm.cnt, 1);
      list[2 * slot] = b;
      list[2 * slot + 1] = (int32_t)t;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    cr.best_key[b] = vb.key;
    cr.best_lin[b] = vb.lin;
    cr.best_row[b] = vb.row;
    cr.best_col[b] = vb.col;
    cr.nrefine_bond[b] = sm.cnt;
    cr.pending[b] = 1;
    atomicAdd((unsigned long long *)&cr.tiles_refined, (unsigned long long)sm.cnt);
  }
  __syncthreads();
}

// sampled-error verification of an instance whose bonds all stopped (Sec. 5)
__device__ void verify_instance(const InstDev &in, Ctrl &cr, DecideSmem &sm) {
  double part = 0.0;
  for (int c = threadIdx.x; c < (int)gridDim.x; c += NT) part += in.err_part[c];
  const double num = block_sum(part, sm.red);
  if (threadIdx.x == 0) {
    cr.screened = 0;
    const double err = sqrt(num / ld_cg(cr.den));
    cr.err = err;
    int pL, pR;
    int32_t rr[TTC_MAXD];
    for (int b = 0; b < in.nb; ++b) rr[b] = ld_cg(cr.r[b]);
    choose_split(in, rr, pL, pR);
    cr.error_fmas += (int64_t)split_cost(in, rr, pL, pR);
    for (int b = 0; b < in.nb; ++b) cr.add[b] = 0;
    sm.flag = 0;
    if (!isfinite(err)) {
      cr.status = 4;
      cr.state = ST_DONE;
    } else if (cr.eps == 0.0 || err <= cr.eps) {
      cr.status = 0;
      cr.state = ST_DONE;
    } else {
      sm.flag = 1;
    }
  }
  __syncthreads();
  // tau /= 10 until a bond adds, the caps are hit or the refinements run out
  while (sm.flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
      bool capped = true;
      for (int b = 0; b < in.nb; ++b)
        if (ld_cg(cr.r[b]) < ld_cg(cr.maxr[b])) capped = false;
      if (capped || ld_cg(cr.refinements) >= ld_cg(cr.max_refine)) {
        cr.status = 7;  // TTC_NOT_CONVERGED
        cr.state = ST_DONE;
        sm.flag = 0;
      } else {
        cr.tau = ld_cg(cr.tau) / 10.0;
        cr.refinements = ld_cg(cr.refinements) + 1;
        cr.state = ST_SCREEN;
        // the mixed recompute forms certified their bests only against the
        // old threshold: they screen again; the FP64 and stored forms keep
        // FP64 values of their bests
        // (a sampled screen draws new samples, as its reference does)
        sm.flag = ((in.prec == P_FP64 || in.stored) && in.nl == 0) ? 1 : 0;
      }
    }
    __syncthreads();
    if (!sm.flag) return;
    // FP64: the cached bests are exact, decide again at the new threshold
    int nadd = 0;
    for (int b = 0; b < in.nb; ++b) {
      finalize_bond(in, cr, b, sm);
      nadd += cr.add[b];
    }
    if (nadd > 0 || cr.state == ST_DONE) return;
  }
}

// decide work items.  Every instance contributes nb + 1 items, numbered
// alike by every CTA whatever the instance's state: item 0 the verification
// (instance, -1), items 1..nb the bonds; place g takes items g, g + G, ...
// Each item checks its own eligibility against the decide kind the screen
// phase fixed.  The numbering must not depend on words that items rewrite
// during the phase (state, screened, pending): a CTA that read them late
// would number the items differently, and one bond would be decided twice.
// item kinds of for_decide_items
enum ItemMode { IM_DECIDE = 0, IM_PENDING = 1, IM_ROOK = 2, IM_FINALIZE = 3 };

// CTAs that share one bond's decide: the mixed stored form of a single
// instance merges its tile slots' k best in DPARTS parts (the last part to
// finish re-scores, takes the stop test and the pivot step); everything else
// in one part (the FP64 best of the slots is one short pass)
constexpr int DPARTS = 32;
__device__ __forceinline__ int decide_parts(const RunArgs &ra, const InstDev &in, int mode) {
  return (mode == IM_DECIDE && ra.count == 1 && in.stored && in.nl == 0 && in.prec != P_FP64)
             ? DPARTS
             : 1;
}

template <class F>
__device__ void for_decide_items(const RunArgs &ra, int mode, F &&f) {
  __shared__ int s_take;
  const int64_t G = gridDim.x;
  int64_t first = 0;
  for (int ii = 0; ii < ra.count; ++ii) {
    const InstDev &in = inst(ra, ii);
    const Ctrl &cr = *in.ctrl;
    const int P = decide_parts(ra, in, mode);
    const int64_t end = first + (int64_t)in.nb * P + 1;
    for (int64_t x = first + ((s_place - first) % G + G) % G; x < end; x += G) {
      const int slot = x == first ? -1 : (int)((x - first - 1) / P);
      const int part = x == first ? 0 : (int)((x - first - 1) % P);
      // one thread decides and the CTA follows: the words it reads can be
      // rewritten by other CTAs' items during the phase (a failing bond ends
      // the instance), and every thread of the CTA must take the same branch
      __syncthreads();
      if (threadIdx.x == 0) {
        const int kind = ld_cg(cr.dkind);
        bool take;
        if (slot < 0) {
          take = mode == IM_DECIDE && kind == DK_VERIFY;
        } else {
          take = kind == DK_BONDS && ld_cg(cr.state) != ST_DONE;
          if (mode == IM_PENDING) take = take && ld_cg(cr.pending[slot]);
          if (mode == IM_ROOK) take = take && in.nl > 0 && ld_cg(cr.rook_stage[slot]) != 0;
          if (mode == IM_FINALIZE) take = take && in.nl > 0;
        }
        s_take = take ? 1 : 0;
      }
      __syncthreads();
      if (s_take) f(ii, slot, part, P);
    }
    first = end;
  }
}

__device__ void phase_decide(const RunArgs &ra, PhaseSmem &sm) {
  for_decide_items(ra, IM_DECIDE, [&](int ii, int b, int part, int P) {
    const InstDev &in = inst(ra, ii);
    Ctrl &cr = *in.ctrl;
    if (b < 0) {
      verify_instance(in, cr, sm.d);
    } else if (in.nl > 0) {
      decide_bond_sampled(in, cr, b, sm.d);
    } else if (in.prec == P_FP64) {
      decide_bond_fp64(in, cr, b, sm.d);
    } else if (in.stored) {
      decide_bond_rescore(in, cr, b, part, P, sm.d);
    } else {
      merge_bond_mixed(in, cr, b, sm.d);
    }
  });
}

// mixed forms, part 2: the FP64 results of the refined tiles join the
// re-scored candidates; the best is the FP64 argmax of the screen.
__device__ void phase_decide2(const RunArgs &ra, PhaseSmem &sm) {
  for_decide_items(ra, IM_PENDING, [&](int ii, int b, int, int) {
    const InstDev &in = inst(ra, ii);
    Ctrl &cr = *in.ctrl;
    DecideSmem &d = sm.d;
    const int32_t cnt = ld_cg(cr.nrefine_bond[b]);
    const Cand *rc = in.refine_cand + in.bond[b].cand_base;
    KeyBest best{ld_cg(cr.best_key[b]), ld_cg(cr.best_lin[b]), ld_cg(cr.best_row[b]),
                 ld_cg(cr.best_col[b])};
    int bad = 0;
    for (int32_t t = threadIdx.x; t < cnt; t += NT) {
      KeyBest o{rc[t].key, rc[t].lin, rc[t].row, rc[t].col};
      bad += o.row < 0;
      kb_take(best, o);
    }
    if (bad) atomicAdd((unsigned long long *)&cr.unscreened, (unsigned long long)bad);
    best = block_best(best, d.rk, d.rl, d.rr, d.rc);
    if (threadIdx.x == 0) {
      cr.best_key[b] = best.key;
      cr.best_lin[b] = best.lin;
      cr.best_row[b] = best.row;
      cr.best_col[b] = best.col;
    }
    __syncthreads();
    finalize_bond(in, cr, b, d);
  });
}

// merge of the G candidate slots of bond b (block-wide; the best is valid
// in every thread)
__device__ KeyBest merge_slots(const InstDev &in, Ctrl &cr, int b, int64_t nt, DecideSmem &sm) {
  const Cand *cand = in.cand + in.bond[b].cand_base;
  KeyBest best{0ull, LLONG_MAX, -1, -1};
  int bad = 0;
  for (int64_t t = threadIdx.x; t < nt; t += NT) {
    KeyBest o{cand[t].key, cand[t].lin, cand[t].row, cand[t].col};
    bad += o.row == -1;
    kb_take(best, o);
  }
  if (bad) atomicAdd((unsigned long long *)&cr.unscreened, (unsigned long long)bad);
  best = block_best(best, sm.rk, sm.rl, sm.rr, sm.rc);
  __syncthreads();
  if (threadIdx.x == 0) {
    sm.rk[0] = best.key;
    sm.rl[0] = best.lin;
    sm.rr[0] = best.row;
    sm.rc[0] = best.col;
  }
  __syncthreads();
  return KeyBest{sm.rk[0], sm.rl[0], sm.rr[0], sm.rc[0]};
}

// sampled screen, decide item of bond b: the argmax over the samples becomes
// the pivot candidate, and its refinement starts (column step first)
__device__ void decide_bond_sampled(const InstDev &in, Ctrl &cr, int b, DecideSmem &sm) {
  const KeyBest best = merge_slots(in, cr, b, gridDim.x, sm);
  if (threadIdx.x == 0) {
    cr.best_key[b] = best.key;
    cr.best_lin[b] = best.lin;
    cr.best_row[b] = best.row;
    cr.best_col[b] = best.col;
    const bool go = in.max_rook > 0 && best.row >= 0 && best.key <= KEY_INF;
    cr.rook_stage[b] = go ? 1 : 0;
    cr.rook_round[b] = 0;
    cr.rook_moved[b] = 0;
    if (b == 0) cr.screen_t = ld_cg(cr.screen_t) + 1;
  }
  __syncthreads();
}

// some bond of a sampled instance is in a refinement step
__device__ bool any_rook(const RunArgs &ra) {
  __shared__ int hit;
  __syncthreads();
  if (threadIdx.x == 0) {
    hit = 0;
    for (int ii = 0; ii < ra.count; ++ii) {
      const InstDev &in = inst(ra, ii);
      if (in.nl == 0) continue;
      const Ctrl &cr = *in.ctrl;
      if (ld_cg(cr.state) == ST_DONE || ld_cg(cr.dkind) != DK_BONDS) continue;
      for (int b = 0; b < in.nb; ++b)
        if (ld_cg(cr.rook_stage[b])) hit = 1;
    }
  }
  __syncthreads();
  return hit != 0;
}

// refinement scan: the pivot's column (step 1) or row (step 2) of every bond
// in a refinement step, spread over the grid; each CTA's best of its share
// goes to its slot
__device__ void phase_rook_scan(const RunArgs &ra, PhaseSmem &sm) {
  __shared__ CtrlSnap snap;
  __shared__ int32_t s_stage[TTC_MAXB], s_row[TTC_MAXB], s_col[TTC_MAXB];
  const int64_t NTOT = (int64_t)gridDim.x * NT;
  const int64_t gt = (int64_t)blockIdx.x * NT + threadIdx.x;
  for (int ii = 0; ii < ra.count; ++ii) {
    const InstDev &in = inst(ra, ii);
    if (in.nl == 0) continue;
    const Ctrl &cr = *in.ctrl;
    snap_ctrl(cr, in.nb, snap);
    if (snap.state == ST_DONE || ld_cg(cr.dkind) != DK_BONDS) continue;
    if (threadIdx.x < in.nb) {
      s_stage[threadIdx.x] = ld_cg(cr.rook_stage[threadIdx.x]);
      s_row[threadIdx.x] = ld_cg(cr.best_row[threadIdx.x]);
      s_col[threadIdx.x] = ld_cg(cr.best_col[threadIdx.x]);
    }
    __syncthreads();
    const int32_t *r = snap.r;  // the sweep-start ranks (no pivot added yet)
    for (int b = 0; b < in.nb; ++b) {
      const int st = s_stage[b];
      if (!st) continue;
      const int64_t rows = rows_of(in, r, b), cols = cols_of(in, r, b);
      KeyBest best{0ull, LLONG_MAX, -1, -1};
      if (st == 1) {
        const int64_t c = s_col[b];
        for (int64_t a = gt; a < rows; a += NTOT)
          take_key(best, residual_at(in, b, r[b], a, c), entry_lin(in, b, a, c), a, c);
      } else {
        const int64_t a = s_row[b];
        for (int64_t c = gt; c < cols; c += NTOT)
          take_key(best, residual_at(in, b, r[b], a, c), entry_lin(in, b, a, c), a, c);
      }
      best = block_best(best, sm.s.sk, sm.s.sl, sm.s.sr, sm.s.sc);
      if (threadIdx.x == 0) {
        Cand *slot = in.cand + in.bond[b].cand_base + blockIdx.x;
        *slot = best.row >= 0 ? Cand{best.key, best.lin, best.row, best.col}
                              : Cand{0ull, LLONG_MAX, -2, -2};
      }
    }
  }
}

// refinement decide: the pivot moves to a strictly larger |E| of its column
// (step 1) or row (step 2); a round is step 1 then step 2, and the
// refinement ends after a round that moved nothing or after max_rook rounds
__device__ void phase_rook_decide(const RunArgs &ra, PhaseSmem &sm) {
  for_decide_items(ra, IM_ROOK, [&](int ii, int b, int, int) {
    const InstDev &in = inst(ra, ii);
    Ctrl &cr = *in.ctrl;
    const KeyBest line = merge_slots(in, cr, b, gridDim.x, sm.d);
    if (threadIdx.x == 0) {
      const int st = ld_cg(cr.rook_stage[b]);
      const uint64_t cur = ld_cg(cr.best_key[b]);
      int moved = ld_cg(cr.rook_moved[b]);
      // ranks written by other CTAs' items: read through L2, not this SM's L1
      const int32_t r_old = ld_cg(cr.r[b]);
      const int64_t rows = (b == 0 ? 1 : ld_cg(cr.r[b - 1])) * in.n[b];
      const int64_t cols = in.n[b + 1] * (b == in.nb - 1 ? 1 : ld_cg(cr.r[b + 1]));
      // several CTAs decide bonds of one instance at once: atomic counts
      const unsigned long long cnt = (unsigned long long)(st == 1 ? rows : cols);
      atomicAdd((unsigned long long *)&cr.entries, cnt);
      atomicAdd((unsigned long long *)&cr.entries_fresh, cnt);
      atomicAdd((unsigned long long *)&cr.screen_fmas, cnt * (unsigned long long)r_old);
      if (line.row >= 0 && line.key > cur) {
        cr.best_key[b] = line.key;
        cr.best_lin[b] = line.lin;
        if (st == 1)
          cr.best_row[b] = line.row;
        else
          cr.best_col[b] = line.col;
        moved = 1;
      }
      if (line.key > KEY_INF) cr.best_key[b] = line.key;  // a non-finite residual ends the bond
      if (st == 1) {
        cr.rook_stage[b] = 2;
        cr.rook_moved[b] = moved;
      } else {
        const int round = ld_cg(cr.rook_round[b]) + 1;
        cr.rook_round[b] = round;
        const bool again = moved && round < in.max_rook && ld_cg(cr.best_key[b]) <= KEY_INF;
        cr.rook_stage[b] = again ? 1 : 0;
        cr.rook_moved[b] = 0;
      }
    }
    __syncthreads();
  });
}

// sampled screen: the stop test and the pivot append of every bond, on the
// refined pivots
__device__ void phase_finalize(const RunArgs &ra, PhaseSmem &sm) {
  for_decide_items(ra, IM_FINALIZE, [&](int ii, int b, int, int) {
    const InstDev &in = inst(ra, ii);
    finalize_bond(in, *in.ctrl, b, sm.d);
  });
}

// ---------------------------------------------------------------------------
// update: items of one instance, in this order per bond b
//   C: replay rows of the new prefix (Alg. 4)                 n_b items
//   A: eq. aca_approx_T_sub on the sweep-start rows           rows_old items
//   B: new row z of R on the sweep-start columns              cols_old items
//   D: new columns of R for the new suffix                    r_new * n_{b+1}
// stores into T / R keep the FP32 (hi, lo) shadows of the mixed forms
__device__ __forceinline__ void putT(const InstDev &in, const BondDev &B, int64_t o, double v) {
  B.T[o] = v;
  if (in.prec != P_FP64) {
    float hi, lo;
    split2(v, hi, lo);
    B.Thi[o] = hi;
    B.Tlo[o] = lo;
  }
}
__device__ __forceinline__ void putR(const InstDev &in, const BondDev &B, int64_t o, double v) {
  B.R[o] = v;
  if (in.prec != P_FP64) {
    float hi, lo;
    split2(v, hi, lo);
    B.Rhi[o] = hi;
    B.Rlo[o] = lo;
  }
}

// A(a, c_z) for z < nz: superblock row a of bond b against the columns of
// its first nz pivots, all issued before any is used (the replay and the row
// update need them inside serial chains).  Hilbert: the entry is the table
// value at the row's index sum plus the pivot's J_{>k} index sum.
__device__ __forceinline__ void pivot_col_entries(const InstDev &in, int b, int64_t a, int z0,
                                                  int nz, double *ent) {
  const BondDev &B = in.bond[b];
  if (in.gen == 0) {
    const int64_t nb0 = in.n[b];
    const int64_t p = a / nb0, i = a - p * nb0;
    const int32_t rs = left_set(in, b).sum[p] + (int32_t)i;
    for (int z = z0; z < nz; ++z) ent[z - z0] = in.hilb[rs + B.J.sum[z]];
  } else {
    for (int z = z0; z < nz; ++z) ent[z - z0] = sb_entry(in, b, a, B.pcol[z]);
  }
}

// Alg. 4 for row a of bond b (eq. aca_approx_T_sub for pivots 0..nz-1 in
// insertion order) by one warp: lane u keeps T(a, 32k + u), k < K, in
// registers.  Step z runs the contract's chain over t < z on every lane from
// broadcasts (the serial order is the contract's; the chain's FP64 latency
// is the cost), then each lane updates its own entries - one instruction
// per 32 entries.  A row per warp issues one FP64 instruction per chain
// element; an SMSP's FP64 unit takes one warp instruction per ~64 cycles,
// the latency of the chain itself.  History row z (hc, hpiv, delta) comes
// from the triangles staged in shared memory (ST: row z at z (z - 1) / 2)
// or from the bond's arrays (row z at z * cap), the next row loading
// during this step when PF.
__device__ void stage_history(const BondDev &B, int nz, int nw, ReplaySmem &rs);

template <int K, bool PF>
__device__ __noinline__ void replay_row_warp(const InstDev &in, int b, int64_t a, int nz,
                                             ReplaySmem *st, bool valid, int nw) {
  const BondDev &B = in.bond[b];
  const int lane = threadIdx.x & 31;
  const int64_t cap = B.cap;
  constexpr unsigned FULL = 0xffffffffu;
  const double *hcb = st ? st->hc : B.hc;
  const double *hpb = st ? st->hp : B.hpiv;
  const double *dlb = st ? st->delta : B.delta;
  auto off = [&](int z) -> int64_t { return st ? (int64_t)z * (z - 1) / 2 : (int64_t)z * cap; };
  double tr[K], en[K], hc[K], hp[K], hcn[K], hpn[K];
  if (in.gen == 0) {
    const int64_t nb0 = in.n[b];
    const int64_t p = a / nb0, i = a - p * nb0;
    const int32_t rs = left_set(in, b).sum[p] + (int32_t)i;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int t = 32 * k + lane;
      en[k] = t < nz ? in.hilb[rs + B.J.sum[t]] : 0.0;
    }
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int t = 32 * k + lane;
      en[k] = t < nz ? sb_entry(in, b, a, B.pcol[t]) : 0.0;
    }
  }
  // the staging's round trip overlaps the entries'; every replay warp of
  // the CTA takes part in it, rows past n_b included
  if (st) stage_history(B, nz, nw, *st);
  if (!valid) return;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    tr[k] = 0.0;
    hcn[k] = 0.0;
    hpn[k] = 0.0;
  }
  double dn = nz > 0 ? dlb[0] : 0.0;
  for (int z = 0; z < nz; ++z) {
    const double dz = dn;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int t = 32 * k + lane;
      if (PF) {
        hc[k] = hcn[k];
        hp[k] = hpn[k];
      } else {
        hc[k] = t < z ? hcb[off(z) + t] : 0.0;
        hp[k] = t < z ? hpb[off(z) + t] : 0.0;
      }
    }
    if (z + 1 < nz) {
      dn = dlb[z + 1];
      if (PF) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int t = 32 * k + lane;
          hcn[k] = t < z + 1 ? hcb[off(z + 1) + t] : 0.0;
          hpn[k] = t < z + 1 ? hpb[off(z + 1) + t] : 0.0;
        }
      }
    }
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (32 * k >= z) break;
      const int lim = min(32, z - 32 * k);
      for (int u = 0; u < lim; ++u)
        acc = __fma_rn(__shfl_sync(FULL, tr[k], u), __shfl_sync(FULL, hc[k], u), acc);
    }
    double ez = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (k == (z >> 5)) ez = __shfl_sync(FULL, en[k], z & 31);
    const double w = __dmul_rn(dz, __dsub_rn(acc, ez));
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int t = 32 * k + lane;
      if (t < z)
        tr[k] = __fma_rn(w, hp[k], tr[k]);
      else if (t == z)
        tr[k] = -w;
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int t = 32 * k + lane;
    if (t < nz) putT(in, B, (int64_t)t * B.ldT + a, tr[k]);
  }
}

// history of bond b (nz <= 32 pivots) into the triangles of shared memory by
// the nw replay warps of the CTA (named barrier 1: the other warps are busy
// elsewhere); every load is issued before the first store
__device__ void stage_history(const BondDev &B, int nz, int nw, ReplaySmem &rs) {
  constexpr int TRI = LANE_NZ * (LANE_NZ - 1) / 2;
  constexpr int PER = (TRI + 31) / 32;
  const int nthr = nw * 32;
  const int64_t cap = B.cap;
  const int tri = nz * (nz - 1) / 2;
  double vc[PER], vp[PER];
#pragma unroll
  for (int m = 0; m < PER; ++m) {
    const int k = threadIdx.x + nthr * m;
    vc[m] = vp[m] = 0.0;
    if (k < tri) {
      int z = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)k)) * 0.5f);
      while (z * (z - 1) / 2 > k) --z;
      while ((z + 1) * z / 2 <= k) ++z;
      const int64_t o = (int64_t)z * cap + (k - z * (z - 1) / 2);
      vc[m] = B.hc[o];
      vp[m] = B.hpiv[o];
    }
  }
  const double dl = (int)threadIdx.x < nz ? B.delta[threadIdx.x] : 0.0;
  asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory");  // earlier readers are done
#pragma unroll
  for (int m = 0; m < PER; ++m) {
    const int k = threadIdx.x + nthr * m;
    if (k < tri) {
      rs.hc[k] = vc[m];
      rs.hp[k] = vp[m];
    }
  }
  if ((int)threadIdx.x < nz) rs.delta[threadIdx.x] = dl;
  asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory");
}

// Alg. 4 replay of up to 32 rows of bond b at once, a row per lane: lane l
// rebuilds T(a0 + l, 0..nz-1) from the pivot history (R(:, c_z) and T(a_z, :)
// of every step z, delta_z) by the steps of update_row, the same FMAs in the
// same order, its row in local memory.  A chain instruction then serves 32
// rows: the FP64 unit, shared by the SM's warps at two FMAs per clock (an
// instruction costs it 16 cycles whatever lanes are active), takes 1/32 of
// the issue of a warp per row.  st: the history staged in shared memory;
// nz <= LANE_NZ.
__device__ __noinline__ void replay_rows_lane(const InstDev &in, int b, int64_t a0, int nrows,
                                              int nz, const ReplaySmem *st) {
  const BondDev &B = in.bond[b];
  const int lane = threadIdx.x & 31;
  const int64_t a = a0 + min(lane, nrows - 1);
  const double *hcb = st->hc, *hpb = st->hp, *dlb = st->delta;
  double tr[LANE_NZ], en[LANE_NZ];  // nz <= LANE_NZ (the staged histories)
  // the row's entries at the pivot columns, gathered before the steps
  if (in.gen == 0) {
    const int64_t nb0 = in.n[b];
    const int64_t p = a / nb0, i = a - p * nb0;
    const int32_t rs = left_set(in, b).sum[p] + (int32_t)i;
    for (int z = 0; z < nz; ++z) en[z] = in.hilb[rs + B.J.sum[z]];
  } else {
    for (int z = 0; z < nz; ++z) en[z] = sb_entry(in, b, a, B.pcol[z]);
  }
  for (int z = 0; z < nz; ++z) {
    const int o = z * (z - 1) / 2;  // row z of the staged triangles
    const double *hc = hcb + o, *hp = hpb + o;
    const double ez = en[z];
    const double dz = dlb[z];
    double acc = 0.0;
    int t = 0;
    for (; t + 4 <= z; t += 4) {
      double x[4], y[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        x[k] = tr[t + k];
        y[k] = hc[t + k];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) acc = __fma_rn(x[k], y[k], acc);
    }
    for (; t < z; ++t) acc = __fma_rn(tr[t], hc[t], acc);
    const double w = __dmul_rn(dz, __dsub_rn(acc, ez));
    for (t = 0; t < z; ++t) tr[t] = __fma_rn(w, hp[t], tr[t]);
    tr[z] = -w;
  }
  if (lane < nrows)
    for (int t = 0; t < nz; ++t) putT(in, B, (int64_t)t * B.ldT + a, tr[t]);
}

// the replays of the n_b rows that the new prefix of bond b-1 adds to bond b:
// chunks of W <= 8 rows, a row per warp (warps 0..W-1; W <= 4 keeps one per
// SMSP, the smallest W that gives every row a warp is taken), chunk
// g to place (cbase + g) mod G, so that the first chunks land on distinct
// SMs and the dependent FP64 chains run at their latency
__device__ int32_t replay_chunks(const InstDev &in, int b, int64_t p, int nz, int32_t &cbase,
                                 int W, ReplaySmem &rs) {
  const int64_t nit = in.n[b];
  const int32_t G = gridDim.x;
  const int32_t nch = (int32_t)((nit + W - 1) / W);
  const int warp = threadIdx.x >> 5;
  if (warp < W) {
    // places and cbase are in [0, G)
    for (int32_t ch = (s_place - cbase + G) % G; ch < nch; ch += G) {
      const int64_t i = (int64_t)ch * W + warp;
      if (nz <= LANE_NZ) {
        replay_row_warp<1, true>(in, b, p * nit + min(i, nit - 1), nz, &rs, i < nit, W);
      } else if (i < nit) {
        const int64_t a = p * nit + i;
        if (nz <= 64)
          replay_row_warp<2, true>(in, b, a, nz, nullptr, true, W);
        else if (nz <= 128)
          replay_row_warp<4, true>(in, b, a, nz, nullptr, true, W);
        else
          replay_row_warp<8, false>(in, b, a, nz, nullptr, true, W);
      }
    }
  }
  cbase = (int32_t)(((int64_t)cbase + nch) % G);
  return nch;
}

__device__ void update_row(const InstDev &in, int b, int64_t a, int z) {
  const BondDev &B = in.bond[b];
  const int cap = B.cap;
  const double *hc = B.hc + (int64_t)z * cap;
  const double *hp = B.hpiv + (int64_t)z * cap;
  double *T = B.T + a;
  const int64_t ld = B.ldT;
  double ent;
  pivot_col_entries(in, b, a, z, z + 1, &ent);
  const double s = __dsub_rn(chain(T, ld, hc, 1, z), ent);
  const double w = __dmul_rn(B.delta[z], s);
  for (int t = 0; t < z; ++t) putT(in, B, a + t * ld, __fma_rn(w, hp[t], T[t * ld]));
  putT(in, B, a + (int64_t)z * ld, -w);
}

// first item >= base that thread gt of NTOT takes when items are dealt
// round-robin (32-bit arithmetic while the counts allow)
__device__ __forceinline__ int64_t first_item(int64_t base, int64_t gt, int64_t NTOT) {
  if (base < ((int64_t)1 << 31) && NTOT < ((int64_t)1 << 31)) {
    const int32_t n = (int32_t)NTOT;
    return base + (((int32_t)gt - (int32_t)base % n) % n + n) % n;
  }
  return base + ((gt - base) % NTOT + NTOT) % NTOT;
}

// ---------------------------------------------------------------------------
// sampled error (Sec. 5).  X~(i) = G_1(i_1) ... G_d(i_d), cores read from T
// (core m < d: element (p, i, u) = T_m[u][p n_m + i]) and R (last core).
// The leading pL and trailing pR cores are contracted once for every index
// combination of their modes (tables tabL, tabR), so a sample pays only the
// middle cores and one dot product.  (pL, pR) minimise
//   NL * s_{pL-1} s_pL + NR * s_{d-pR} s_{d-pR+1} + ns * (middle + s_{d-pR})
// within the table capacities; every CTA evaluates the same choice.

// core size s_m (s_0 = s_d = 1, s_m = r_{m-1})
__device__ __forceinline__ int64_t core_s(const InstDev &in, const int32_t *r, int m) {
  return (m == 0 || m == in.d) ? 1 : r[m - 1];
}

// FMAs of the error evaluation with tables of pL / pR modes (the last table
// level dominates; the chunked build adds its lower levels once per chunk)
// (in FP32: a cost estimate, identical on every thread; FP64 operations are
// long-latency on this GPU and every thread evaluates the choice)
__device__ double split_cost(const InstDev &in, const int32_t *r, int pL, int pR) {
  const int d = in.d;
  float NL = 1.f, NR = 1.f;
  for (int m = 0; m < pL; ++m) NL *= (float)in.n[m];
  for (int m = d - pR; m < d; ++m) NR *= (float)in.n[m];
  const float tl = pL >= 2 ? NL * (float)core_s(in, r, pL - 1) * (float)core_s(in, r, pL) : 0.f;
  const float tr =
      pR >= 2 ? NR * (float)core_s(in, r, d - pR) * (float)core_s(in, r, d - pR + 1) : 0.f;
  float mid = (float)core_s(in, r, d - pR);
  for (int m = pL; m < d - pR; ++m) mid += (float)core_s(in, r, m) * (float)core_s(in, r, m + 1);
  return (double)(tl + tr + (float)in.nsamples * mid);
}

__device__ void choose_split(const InstDev &in, const int32_t *r, int &pL, int &pR) {
  const int d = in.d;
  double best = 1e300;
  pL = 1;
  pR = 1;
  float NL = 1.f;
  for (int a = 1; a < d; ++a) {
    NL *= (float)in.n[a - 1];
    if (a >= 2 && NL * (float)core_s(in, r, a) > (float)in.tabL_cap) break;
    float NR = 1.f;
    for (int c = 1; a + c <= d; ++c) {
      NR *= (float)in.n[d - c];
      if (c >= 2 && NR * (float)core_s(in, r, d - c) > (float)in.tabR_cap) break;
      const double cost = split_cost(in, r, a, c);
      if (cost < best) {
        best = cost;
        pL = a;
        pR = c;
      }
    }
  }
}

// v (length s_m) <- v G_m(i) for a middle core 1 <= m <= d-2
// dst[t] = src[t * s] for t < n, eight loads in flight (a plain copy loop
// waits for each load before it issues the next)
__device__ __forceinline__ void copy8(double *dst, const double *src, int64_t s, int n) {
  int t = 0;
  for (; t + 8 <= n; t += 8) {
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = src[(int64_t)(t + k) * s];
#pragma unroll
    for (int k = 0; k < 8; ++k) dst[t + k] = x[k];
  }
  for (; t < n; ++t) dst[t] = src[(int64_t)t * s];
}

// out[o] = sum_p x[p] * col_o[p * s] for o < n, col_o = base + o * so: four
// outputs at a time, each its own serial FMA chain in p (so the FP64 pipe
// has four independent chains to overlap instead of one)
__device__ __forceinline__ void contract4(const double *x, int len, const double *base, int64_t so,
                                          int64_t s, double *out, int n) {
  int o = 0;
  for (; o + 4 <= n; o += 4) {
    const double *c0 = base + (int64_t)o * so, *c1 = c0 + so, *c2 = c1 + so, *c3 = c2 + so;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int p = 0;
    for (; p + 4 <= len; p += 4) {
      // 20 loads in flight, then the 16 FMAs in chain order
      double xv[4], v0[4], v1[4], v2[4], v3[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int64_t q = (int64_t)(p + k) * s;
        xv[k] = x[p + k];
        v0[k] = c0[q];
        v1[k] = c1[q];
        v2[k] = c2[q];
        v3[k] = c3[q];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        a0 = __fma_rn(xv[k], v0[k], a0);
        a1 = __fma_rn(xv[k], v1[k], a1);
        a2 = __fma_rn(xv[k], v2[k], a2);
        a3 = __fma_rn(xv[k], v3[k], a3);
      }
    }
    for (; p < len; ++p) {
      const double xp = x[p];
      const int64_t q = (int64_t)p * s;
      a0 = __fma_rn(xp, c0[q], a0);
      a1 = __fma_rn(xp, c1[q], a1);
      a2 = __fma_rn(xp, c2[q], a2);
      a3 = __fma_rn(xp, c3[q], a3);
    }
    out[o] = a0;
    out[o + 1] = a1;
    out[o + 2] = a2;
    out[o + 3] = a3;
  }
  for (; o < n; ++o) {
    const double *c = base + (int64_t)o * so;
    double a = 0.0;
    for (int p = 0; p < len; ++p) a = __fma_rn(x[p], c[(int64_t)p * s], a);
    out[o] = a;
  }
}

// v (length s_m) <- v G_m(i) for a middle core 1 <= m <= d-2
__device__ __forceinline__ int mul_core(const InstDev &in, const int32_t *r, int m, int64_t i,
                                        double *v, double *w) {
  const BondDev &B = in.bond[m];
  const int rl = (int)core_s(in, r, m), rr = (int)core_s(in, r, m + 1);
  contract4(v, rl, B.T + i, B.ldT, in.n[m], w, rr);
  for (int u = 0; u < rr; ++u) v[u] = w[u];
  return rr;
}

// w (length s_{m+1}) <- G_m(i) w for a core 1 <= m <= d-2 (right to left)
__device__ __forceinline__ int mul_core_right(const InstDev &in, const int32_t *r, int m,
                                              int64_t i, double *w, double *t) {
  const BondDev &B = in.bond[m];
  const int rl = (int)core_s(in, r, m), rr = (int)core_s(in, r, m + 1);
  contract4(w, rr, B.T + i, in.n[m], B.ldT, t, rl);
  for (int p = 0; p < rl; ++p) w[p] = t[p];
  return rl;
}

constexpr int TAB_CHUNK = 8;  // last-mode indices per table work item

// tables of the verifying instances: a work item is a prefix of pL-1 modes
// (suffix of pR-1 modes) and a chunk of TAB_CHUNK values of the next mode
__device__ void phase_tables(const RunArgs &ra) {
  // items are dealt a warp's worth per CTA in turn (lane l of warp w of CTA
  // c is number (w G + c) 32 + l): when there are fewer items than threads
  // every SM still gets an equal share of this FP64-bound phase, and the
  // lanes of a warp keep neighbouring items (the same core rows)
  const int64_t NTOT = (int64_t)gridDim.x * blockDim.x;
  const int64_t gt = ((int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32 + (threadIdx.x & 31);
  __shared__ CtrlSnap snap;
  int64_t base = 0;
  for (int ii = 0; ii < ra.count; ++ii) {
    const InstDev &in = inst(ra, ii);
    const Ctrl &cr = *in.ctrl;
    snap_ctrl(cr, in.nb, snap);
    if (snap.state == ST_DONE) continue;
    if (!snap.screened) continue;
    const int32_t *r = snap.r;
    int nadd = 0;
    for (int b = 0; b < in.nb; ++b) nadd += snap.add[b];
    if (nadd) continue;
    int pL, pR;
    choose_split(in, r, pL, pR);
    const int d = in.d;
    double v[RCAP], w[RCAP];
    if (pL >= 2) {
      int64_t np = 1;
      for (int m = 0; m < pL - 1; ++m) np *= in.n[m];
      const int64_t nl = in.n[pL - 1], nch = (nl + TAB_CHUNK - 1) / TAB_CHUNK;
      const int64_t sl = core_s(in, r, pL);
      const int64_t items = np * nch;
      for (int64_t x = first_item(base, gt, NTOT); x < base + items; x += NTOT) {
        const int64_t pre = (x - base) / nch, ch = (x - base) - pre * nch;
        int64_t l = pre;
        int32_t idx[TTC_MAXD];
        for (int m = 0; m < pL - 1; ++m) {
          idx[m] = (int32_t)(l % in.n[m]);
          l /= in.n[m];
        }
        const BondDev &B0 = in.bond[0];
        int len = (int)core_s(in, r, 1);
        copy8(v, B0.T + idx[0], B0.ldT, len);
        for (int m = 1; m < pL - 1; ++m) len = mul_core(in, r, m, idx[m], v, w);
        // last mode of the prefix: core pL-1 (a middle core, pL-1 <= d-2)
        const BondDev &B = in.bond[pL - 1];
        for (int64_t i = ch * TAB_CHUNK; i < min(nl, (ch + 1) * TAB_CHUNK); ++i)
          contract4(v, len, B.T + i, B.ldT, nl, in.tabL + (pre + i * np) * sl, (int)sl);
      }
      base += items;
    }
    if (pR >= 2) {
      int64_t np = 1;
      for (int m = d - pR + 1; m < d; ++m) np *= in.n[m];
      const int mf = d - pR;  // first mode of the suffix
      const int64_t nf = in.n[mf], nch = (nf + TAB_CHUNK - 1) / TAB_CHUNK;
      const int64_t sr = core_s(in, r, mf);
      const int64_t items = np * nch;
      for (int64_t x = first_item(base, gt, NTOT); x < base + items; x += NTOT) {
        const int64_t suf = (x - base) / nch, ch = (x - base) - suf * nch;
        int64_t l = suf;
        int32_t idx[TTC_MAXD];
        for (int m = mf + 1; m < d; ++m) {
          idx[m] = (int32_t)(l % in.n[m]);
          l /= in.n[m];
        }
        const BondDev &BL = in.bond[d - 2];
        int len = (int)core_s(in, r, d - 1);
        copy8(w, BL.R + idx[d - 1], BL.ldR, len);
        for (int m = d - 2; m > mf; --m) len = mul_core_right(in, r, m, idx[m], w, v);
        const BondDev &B = in.bond[mf];
        for (int64_t i = ch * TAB_CHUNK; i < min(nf, (ch + 1) * TAB_CHUNK); ++i)
          contract4(w, len, B.T + i, nf, B.ldT, in.tabR + (i + nf * suf) * sr, (int)sr);
      }
      base += items;
    }
  }
}

// error of one sample: X(i) - X~(i), using the tables of (pL, pR)
__device__ double sample_residual(const InstDev &in, const int32_t *r, int pL, int pR, int64_t k) {
  const double xk = in.xs[k];
  double v[RCAP], w[RCAP];
  const int d = in.d;
  int len;
  const double *src;   // the prefix vector in memory (stride sv)
  int64_t sv;
  if (pL >= 2) {
    int64_t e = 0, st = 1;
    for (int m = 0; m < pL; ++m) {
      e += sample_coord(in, k, m) * st;
      st *= in.n[m];
    }
    len = (int)core_s(in, r, pL);
    src = in.tabL + e * len;
    sv = 1;
  } else {
    const BondDev &B0 = in.bond[0];
    len = (int)core_s(in, r, 1);
    src = B0.T + sample_coord(in, k, 0);
    sv = B0.ldT;
  }
  if (pL + pR < d) {
    // middle cores: the vector goes to local memory
    copy8(v, src, sv, len);
    for (int m = pL; m < d - pR; ++m) len = mul_core(in, r, m, sample_coord(in, k, m), v, w);
    src = v;
    sv = 1;
  }
  double xt;
  if (pR >= 2) {
    int64_t e = 0, st = 1;
    for (int m = d - pR; m < d; ++m) {
      e += sample_coord(in, k, m) * st;
      st *= in.n[m];
    }
    const double *y = in.tabR + e * len;
    if (len <= 16) {
      // both rows in flight at once (a round trip to L2 each otherwise per
      // eight entries), then the contract's chain
      double xv[16], yv[16];
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        xv[t] = t < len ? src[t * sv] : 0.0;
        yv[t] = t < len ? y[t] : 0.0;
      }
      double acc = 0.0;
#pragma unroll
      for (int t = 0; t < 16; ++t)
        if (t < len) acc = __fma_rn(xv[t], yv[t], acc);
      xt = acc;
    } else {
      xt = chain(src, sv, y, 1, len);
    }
  } else {
    const BondDev &BL = in.bond[d - 2];
    xt = chain(src, sv, BL.R + sample_coord(in, k, d - 1), BL.ldR, len);
  }
  return __dsub_rn(xk, xt);
}


// The error's samples when the prefix and suffix tables meet (pL + pR = d,
// rows of len <= 16): lane l of a warp takes the l-th of 32 consecutive
// samples, as in the thread dealing of the plain loop.  The warp loads the
// 32 samples' rows together, two rows per instruction, into shared memory,
// and each lane then runs the contract's chain on its own two rows.  The
// operations and their order per thread are those of sample_residual.
__device__ __noinline__ double samples_joined(const InstDev &in, int pL, int pR, int len,
                                              int64_t base, int64_t ns, int64_t gs, int64_t NTOT,
                                              SampleSmem &sw) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, half = lane >> 4, el = lane & 15;
  double *buf = sw.rows[threadIdx.x >> 5];
  const int d = in.d;
  double part = 0.0;
  for (int64_t x = first_item(base, gs, NTOT);; x += NTOT) {
    const int valid = x < base + ns;
    if (!__any_sync(FULL, valid)) break;
    const int64_t k = valid ? x - base : 0;
    const double xk = valid ? in.xs[k] : 0.0;
    int64_t eL = 0, eR = 0, st = 1;
    for (int m = 0; m < pL; ++m) {
      eL += sample_coord(in, k, m) * st;
      st *= in.n[m];
    }
    st = 1;
    for (int m = d - pR; m < d; ++m) {
      eR += sample_coord(in, k, m) * st;
      st *= in.n[m];
    }
    double xv[16], yv[16];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const double *tab = side == 0 ? in.tabL : in.tabR;
      const int64_t e = side == 0 ? eL : eR;
      double v[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int sr = 2 * q + half;
        const int64_t es = __shfl_sync(FULL, e, sr);
        const int vs = __shfl_sync(FULL, valid, sr);
        v[q] = (vs && el < len) ? tab[es * len + el] : 0.0;
      }
      __syncwarp();  // the previous rows are read
#pragma unroll
      for (int q = 0; q < 16; ++q) buf[(2 * q + half) * 17 + el] = v[q];
      __syncwarp();
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        if (side == 0)
          xv[t] = buf[lane * 17 + t];
        else
          yv[t] = buf[lane * 17 + t];
      }
    }
    double acc = 0.0;
#pragma unroll
    for (int t = 0; t < 16; ++t)
      if (t < len) acc = __fma_rn(xv[t], yv[t], acc);
    if (valid) {
      const double e = __dsub_rn(xk, acc);
      part = __fma_rn(e, e, part);
    }
  }
  return part;
}

__device__ void phase_update(const RunArgs &ra, PhaseSmem &sm) {
  __shared__ CtrlSnap snap;
  const int64_t NTOT = (int64_t)gridDim.x * NT;
  // items that each write their own outputs are dealt over the places; the
  // error's samples by blockIdx, so that the partial sums (and their
  // rounding) do not depend on where the CTAs run
  const int64_t gt = (int64_t)s_place * NT + threadIdx.x;
  const int64_t gs = (int64_t)blockIdx.x * NT + threadIdx.x;
  int64_t base = 0;
  for (int ii = 0; ii < ra.count; ++ii) {
    const InstDev &in = inst(ra, ii);
    const Ctrl &cr = *in.ctrl;
    // the work follows from the decisions (every CTA reads the same flags;
    // the state word is rewritten by the owner CTA during this phase)
    snap_ctrl(cr, in.nb, snap);
    const int st = snap.state;
    if (st == ST_DONE) continue;
    const int32_t *ro = snap.old_r, *rn = snap.r, *ad = snap.add;
    int nadd = 0;
    for (int b = 0; b < in.nb; ++b) nadd += ad[b];
    const bool screened = snap.screened != 0;
    if (blockIdx.x == ii % gridDim.x && threadIdx.x < 32) {
      if (nadd == 0 && screened && threadIdx.x == 0) in.ctrl->state = ST_VERIFY;
      if (nadd > 0) write_plan_warp(in, *in.ctrl, rn, gridDim.x);  // next screen's tiles
    }
    if (nadd > 0) {
      // the replays are the longest items.  One instance on a grid of two
      // CTAs per SM: the replays go a row per lane to warps 0..RW-1 of the
      // first places (distinct SMs, at most a quarter of them), whose SMs
      // take no other item, so that their dependent FP64 chains do not
      // queue behind other warps' FP64 work on the SM's shared unit; the
      // thread-dealt items go to the other places.  Otherwise a row per
      // warp, and the thread-dealt items start on the place after the last
      // replay chunk.
      const int32_t S = s_sm2;
      int64_t lch = 0;
      for (int b = 1; b < in.nb; ++b)
        if (ad[b - 1]) lch += (in.n[b] + 31) / 32;
      const int32_t RW = (int32_t)min((int64_t)4, (lch + (S / 4) - 1) / max(1, S / 4));
      const int32_t nsr = RW > 0 ? (int32_t)((lch + RW - 1) / RW) : 0;  // replay SMs
      bool small = true;  // every replayed history fits the staging (rank <= LANE_NZ)
      for (int b = 1; b < in.nb; ++b)
        if (ad[b - 1] && rn[b] > LANE_NZ) small = false;
      const bool iso = ra.count == 1 && S > 0 && (int32_t)gridDim.x == 2 * S && lch > 0 &&
                       RW == 1 && nsr <= S / 4 && 2 * nsr < (int32_t)gridDim.x && small;
      int64_t gti = gt, NTI = NTOT;
      bool idle = false;  // a thread of a replay SM: no thread-dealt item
      if (iso) {
        const int32_t pl = s_place;
        const bool rsm = pl < nsr || (pl >= S && pl < S + nsr);
        idle = rsm;
        if (pl < nsr && (threadIdx.x >> 5) == 0) {
          // replay chunk g = pl of this SM (bonds in order), by warp 0 from
          // the history staged in shared memory
          const int64_t g = pl;
          int64_t first = 0;
          for (int b = 1; b < in.nb && g >= first; ++b) {
            if (!ad[b - 1]) continue;
            const int64_t nc = (in.n[b] + 31) / 32;
            if (g < first + nc) {
              const int64_t i0 = (g - first) * 32;
              stage_history(in.bond[b], rn[b], 1, sm.rp);
              replay_rows_lane(in, b, (int64_t)ro[b - 1] * in.n[b] + i0,
                               (int)min((int64_t)32, in.n[b] - i0), rn[b], &sm.rp);
            }
            first += nc;
          }
        }
        // item threads: the places of the other SMs, renumbered from 0
        NTI = (int64_t)(gridDim.x - 2 * nsr) * NT;
        gti = rsm ? 0 : (int64_t)(pl < S ? pl - nsr : pl - 2 * nsr) * NT + threadIdx.x;
      } else {
        int32_t cbase = (int32_t)((base / NT) % gridDim.x);
        int64_t nchunks = 0, rrows = 0;
        for (int b = 1; b < in.nb; ++b)
          if (ad[b - 1]) rrows += in.n[b];
        const int W = (int)min((int64_t)(NT / 32), max((int64_t)1, (rrows + gridDim.x - 1) / gridDim.x));
        for (int b = 1; b < in.nb; ++b) {
          if (!ad[b - 1]) continue;
          nchunks += replay_chunks(in, b, ro[b - 1], rn[b], cbase, W, sm.rp);
        }
        base += nchunks * NT;
      }
      auto item0 = [&](int64_t bs) -> int64_t {
        return idle ? LLONG_MAX : first_item(bs, gti, NTI);
      };
      for (int b = 0; b < in.nb; ++b) {
        const BondDev &B = in.bond[b];
        // a thread with no item of this bond skips it whole: no load of the
        // pivot's coordinates or entries reaches its path
        {
          const int64_t rc = ad[b] ? rows_of(in, ro, b) + cols_of(in, ro, b) : 0;
          const int64_t tot = (in.stored ? 2 : 1) * rc +
                              (b < in.nb - 1 && ad[b + 1] ? (int64_t)rn[b] * in.n[b + 1] : 0);
          if (item0(base) >= base + tot) {
            base += tot;
            continue;
          }
        }
        if (ad[b] && in.stored) {
          // the pending rank-one step of the stored residual (from the
          // sweep-start superblock, which E still holds)
          const int64_t rows = rows_of(in, ro, b), cols = cols_of(in, ro, b);
          const int64_t ld = B.ldR, as = B.prow[ro[b]], cs = B.pcol[ro[b]];
          for (int64_t x = item0(base); x < base + rows; x += NTI)
            sv_put(in, B.ew, x - base,
                   -(sv_get(in, B.E, (x - base) * ld + cs) / sv_get(in, B.E, as * ld + cs)));
          base += rows;
          for (int64_t x = item0(base); x < base + cols; x += NTI)
            B.erow[x - base] = B.E[as * ld + (x - base)];  // the same 8 bytes in either form
          base += cols;
        }
        if (ad[b]) {
          const int z = ro[b];
          const int64_t rows = rows_of(in, ro, b), cols = cols_of(in, ro, b);
          for (int64_t x = item0(base); x < base + rows; x += NTI)
            update_row(in, b, x - base, z);
          base += rows;
          for (int64_t x = item0(base); x < base + cols; x += NTI)
            putR(in, B, (int64_t)z * B.ldR + (x - base), sb_entry(in, b, B.prow[z], x - base));
          base += cols;
        }
        if (b < in.nb - 1 && ad[b + 1]) {
          const int64_t nb1 = in.n[b + 1];
          const int64_t q = ro[b + 1];
          const int64_t nit = (int64_t)rn[b] * nb1;
          for (int64_t x = item0(base); x < base + nit; x += NTI) {
            const int64_t l = x - base, t = l / nb1, jj = l - t * nb1;
            const int64_t c = q * nb1 + jj;
            putR(in, B, t * B.ldR + c, sb_entry(in, b, B.prow[t], c));
          }
          base += nit;
        }
      }
    } else if (screened) {
      double part = 0.0;
      const int64_t ns = in.nsamples;
      int pL, pR;
      choose_split(in, rn, pL, pR);
      const int jl = pL >= 2 && pR >= 2 && pL + pR == in.d ? (int)core_s(in, rn, pL) : 0;
      if (jl > 0 && jl <= 16) {
        part = samples_joined(in, pL, pR, jl, base, ns, gs, NTOT, sm.sw);
      } else {
        for (int64_t x = first_item(base, gs, NTOT); x < base + ns; x += NTOT) {
          const double e = sample_residual(in, rn, pL, pR, x - base);
          part = __fma_rn(e, e, part);
        }
      }
      base += ns;
      const double s = block_sum(part, sm.red);
      if (threadIdx.x == 0) in.err_part[blockIdx.x] = s;
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// init.  The start pivot is Alg. 1 line 1 with a zero approximation: the
// argmax of |X| over the error's random samples and the origin (ties: lowest
// linear index).  Every bond takes it as its first pivot (ranks 1).
//   init1 (all CTAs): X at the samples, partial sums of X^2, per-CTA argmax
//   init2 (owner CTA): reduce; pivot sets, delta_0, U = [delta_0]
//   init3 (all CTAs): T(:,0) and R(0,:) of every bond
__device__ void phase_init1(const RunArgs &ra, PhaseSmem &sm) {
  const int64_t NTOT = (int64_t)gridDim.x * NT;
  const int64_t gt = (int64_t)blockIdx.x * NT + threadIdx.x;
  int64_t base = 0;
  for (int ii = 0; ii < ra.count; ++ii) {
    const InstDev &in = inst(ra, ii);
    double part = 0.0;
    KeyBest best{0ull, LLONG_MAX, -1, -1};
    const int64_t ns = in.nsamples;
    for (int64_t x = first_item(base, gt, NTOT); x < base + ns; x += NTOT) {
      int32_t idx[TTC_MAXD];
      sample_index(in, x - base, idx);
      // user generator: the samples' values were filled by the callback
      const double v = in.gen == 4 ? in.xs[x - base] : gen_full(in, idx);
      in.xs[x - base] = v;
      part = __fma_rn(v, v, part);
      const uint64_t k = abs_key(v);
      if (best.row < 0 || k >= best.key) {
        int64_t l = 0;
        for (int m = 0; m < in.d; ++m) l += (int64_t)idx[m] * in.stride[m];
        if (best.row < 0 || k > best.key || l < best.lin) {
          best.key = k;
          best.lin = l;
          best.row = 0;
          best.col = (int32_t)(x - base);
        }
      }
    }
    base += ns;
    const double s = block_sum(part, sm.red);
    __shared__ uint64_t sk[NT / 32];
    __shared__ int64_t sl[NT / 32];
    __shared__ int32_t sr[NT / 32], sc[NT / 32];
    best = block_best(best, sk, sl, sr, sc);
    if (threadIdx.x == 0) {
      in.err_part[blockIdx.x] = s;
      in.start_part[blockIdx.x].key = best.key;
      in.start_part[blockIdx.x].lin = best.lin;
      in.start_part[blockIdx.x].row = best.row;
      in.start_part[blockIdx.x].col = best.col;  // the sample's number
    }
    __syncthreads();
  }
}

__device__ void phase_init2(const RunArgs &ra, PhaseSmem &sm) {
  for (int ii = blockIdx.x; ii < ra.count; ii += gridDim.x) {
    const InstDev &in = inst(ra, ii);
    Ctrl &cr = *in.ctrl;
    double part = 0.0;
    KeyBest best{0ull, LLONG_MAX, -1, -1};
    for (int c = threadIdx.x; c < (int)gridDim.x; c += NT) {
      part += in.err_part[c];
      const Cand &cd = in.start_part[c];
      KeyBest o{cd.key, cd.lin, cd.row, cd.col};
      kb_take(best, o);
    }
    const double den = block_sum(part, sm.d.red);
    best = block_best(best, sm.d.rk, sm.d.rl, sm.d.rr, sm.d.rc);
    if (threadIdx.x == 0) {
      cr.den = den;
      cr.xrms = sqrt(den / (double)in.nsamples);
      int32_t zero[TTC_MAXD] = {0};
      // user generator: the origin's value follows the samples in xs
      const double x0 = in.gen == 4 ? in.xs[in.nsamples] : gen_full(in, zero);
      KeyBest o{abs_key(x0), 0, 0, (int32_t)in.nsamples};
      kb_take(best, o);
      int32_t st[TTC_MAXD];
      int64_t l = best.lin;
      for (int m = 0; m < in.d; ++m) {
        st[m] = (int32_t)(l % in.n[m]);
        l /= in.n[m];
      }
      const double xs0 = in.gen == 4 ? in.xs[best.col] : gen_full(in, st);
      if (!isfinite(den) || !isfinite(xs0)) {
        cr.status = 4;
        cr.state = ST_DONE;
      } else if (xs0 == 0.0) {
        cr.status = 3;
        cr.state = ST_DONE;
      }
      for (int b = 0; b < in.nb && cr.state != ST_DONE; ++b) {
        const BondDev &B = in.bond[b];
        int64_t ll = 0;
        int32_t ss = 0;
        for (int m = 0; m <= b; ++m) {
          B.I.idx[m] = st[m];
          ll += (int64_t)st[m] * in.stride[m];
          ss += st[m];
        }
        B.I.lin[0] = ll;
        B.I.sum[0] = ss;
        ll = 0;
        ss = 0;
        for (int m = b + 1; m < in.d; ++m) {
          B.J.idx[m - b - 1] = st[m];
          ll += (int64_t)st[m] * in.stride[m];
          ss += st[m];
        }
        B.J.lin[0] = ll;
        B.J.sum[0] = ss;
        B.prow[0] = st[b];
        B.pcol[0] = st[b + 1];
        cr.r[b] = 1;
        cr.r_old[b] = 1;
        cr.add[b] = 0;
      }
      if (cr.state != ST_DONE) {
        // the pivot entry of every superblock is X(start)
        const double delta = 1.0 / __dsub_rn(xs0, 0.0);
        if (!isfinite(delta)) {
          cr.status = 4;
          cr.state = ST_DONE;
        }
        for (int b = 0; b < in.nb; ++b) {
          in.bond[b].delta[0] = delta;
          in.bond[b].U[0] = delta;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < 32 && cr.state != ST_DONE) write_plan_warp(in, cr, cr.r, gridDim.x);
    __syncthreads();
  }
}

__device__ void phase_init3(const RunArgs &ra, PhaseSmem &sm) {
  const int64_t NTOT = (int64_t)gridDim.x * NT;
  const int64_t gt = (int64_t)blockIdx.x * NT + threadIdx.x;
  int64_t base = 0;
  for (int ii = 0; ii < ra.count; ++ii) {
    const InstDev &in = inst(ra, ii);
    const Ctrl &cr = *in.ctrl;
    if (ld_cg(cr.state) == ST_DONE) continue;
    for (int b = 0; b < in.nb; ++b) {
      const BondDev &B = in.bond[b];
      const int64_t rows = in.n[b], cols = in.n[b + 1];
      const double delta = B.delta[0];
      const int64_t a0 = B.prow[0], c0 = B.pcol[0];
      for (int64_t x = first_item(base, gt, NTOT); x < base + rows; x += NTOT) {
        const int64_t a = x - base;
        const double s = __dsub_rn(0.0, sb_entry(in, b, a, c0));
        putT(in, B, a, -__dmul_rn(delta, s));
      }
      base += rows;
      for (int64_t x = first_item(base, gt, NTOT); x < base + cols; x += NTOT)
        putR(in, B, x - base, sb_entry(in, b, a0, x - base));
      base += cols;
    }
  }
}

// refine (mixed forms): FP64 screen of the queued tiles
__device__ void phase_refine(const RunArgs &ra, PhaseSmem &sm) {
  const int64_t G = gridDim.x;
  int64_t base = 0;
  for (int ii = 0; ii < ra.count; ++ii) {
    const InstDev &in = inst(ra, ii);
    const Ctrl &cr = *in.ctrl;
    if (ld_cg(cr.state) == ST_DONE) continue;
    if (!ld_cg(cr.screened)) continue;
    int32_t r[TTC_MAXD];
    for (int b = 0; b < in.nb; ++b) r[b] = ld_cg(cr.r[b]);
    for (int b = 0; b < in.nb; ++b) {
      if (!ld_cg(cr.pending[b])) continue;
      const int64_t cnt = ld_cg(cr.nrefine_bond[b]);
      const int32_t *list = in.refine_list + 2 * in.bond[b].cand_base;
      Cand *out = in.refine_cand + in.bond[b].cand_base;
      const TileGeo g = planned_geo(in, cr, b);
      for (int64_t t = base + ((blockIdx.x - base) % G + G) % G; t < base + cnt; t += G) {
        const int64_t li = t - base;
        const int32_t tile = list[2 * li + 1];
        const int32_t tr = tile / g.nct, tc = tile - tr * g.nct;
        int64_t r0, c0;
        int nr, nc;
        tile_rows(in, g, b, tr, r0, nr);
        tile_cols(in, g, b, tc, c0, nc);
        screen_tile_fp64(in, b, r[b], r0, nr, c0, nc, g.te, out + li, sm.s);
      }
      base += cnt;
    }
  }
}

__device__ bool all_done(const RunArgs &ra) {
  __shared__ int done;
  __syncthreads();
  if (threadIdx.x == 0) {
    done = 1;
    for (int ii = 0; ii < ra.count; ++ii)
      if (ld_cg(inst(ra, ii).ctrl->state) != ST_DONE) done = 0;
  }
  __syncthreads();
  return done != 0;
}

// ---------------------------------------------------------------------------
// kernels

extern __shared__ __align__(16) unsigned char dyn_smem[];



// CTA 0 accounts the time between barrier exits to the phase that ran
struct PhaseClock {
  uint64_t t;
  __device__ void start() {
    if (blockIdx.x == 0 && threadIdx.x == 0) t = globaltimer_ns();
  }
  __device__ void lap(const RunArgs &ra, int slot) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      const uint64_t now = globaltimer_ns();
      ra.bar->phase_ns[slot] += now - t;
      t = now;
    }
  }
};

// some instance evaluates its sampled error in the coming update phase
__device__ bool any_verify(const RunArgs &ra) {
  __shared__ int hit;
  __syncthreads();
  if (threadIdx.x == 0) {
    hit = 0;
    for (int ii = 0; ii < ra.count; ++ii) {
      const Ctrl &cr = *inst(ra, ii).ctrl;
      if (ld_cg(cr.state) == ST_DONE) continue;
      if (!ld_cg(cr.screened)) continue;
      int nadd = 0;
      for (int b = 0; b < inst(ra, ii).nb; ++b) nadd += ld_cg(cr.add[b]);
      if (nadd == 0) hit = 1;
    }
  }
  __syncthreads();
  return hit != 0;
}

__device__ __forceinline__ int32_t sm_id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return (int32_t)r;
}

// s_place from the table of SM ids (written by every CTA before a grid
// barrier): with cnt[s] CTAs on SM s and this CTA the k-th on its SM sm,
//   place = sum_s min(cnt[s], k) + #{s < sm : cnt[s] > k},
// its rank when the CTAs are sorted by (k, SM) - a bijection onto [0, G).
// Ids outside the table keep the identity order.
__device__ void spread_order(const RunArgs &ra, PhaseSmem &sm) {
  SpreadSmem &sp = sm.sp;
  const int G = gridDim.x, me = sm_id();
  for (int s = threadIdx.x; s < SPREAD_MAXSM; s += NT) sp.cnt[s] = 0;
  if (threadIdx.x == 0) {
    sp.k = 0;
    sp.place = 0;
    sp.bad = me >= SPREAD_MAXSM;
    sp.nsm = 0;
    sp.not2 = 0;
  }
  __syncthreads();
  int k = 0;
  for (int j = threadIdx.x; j < G; j += NT) {
    const int s = ld_cg(ra.smid[j]);
    if (s >= 0 && s < SPREAD_MAXSM)
      atomicAdd(&sp.cnt[s], 1);
    else
      sp.bad = 1;
    k += (j < (int)blockIdx.x && s == me);
  }
  if (k) atomicAdd(&sp.k, k);
  __syncthreads();
  const int kk = sp.k;
  int part = 0, used = 0, odd = 0;
  for (int s = threadIdx.x; s < SPREAD_MAXSM; s += NT) {
    const int c = sp.cnt[s];
    part += min(c, kk) + (s < me && c > kk);
    used += c > 0;
    odd += c != 0 && c != 2;
  }
  if (part) atomicAdd(&sp.place, part);
  if (used) atomicAdd(&sp.nsm, used);
  if (odd) atomicAdd(&sp.not2, odd);
  __syncthreads();
  if (threadIdx.x == 0) {
    s_place = sp.bad ? (int32_t)blockIdx.x : sp.place;
    s_sm2 = (sp.bad || sp.not2) ? 0 : sp.nsm;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(NT, 2) k_persistent(RunArgs ra) {
  PhaseSmem &sm = *reinterpret_cast<PhaseSmem *>(dyn_smem);
  cache_inst0(ra);
  PhaseClock clk;
  clk.start();
  if (threadIdx.x == 0) ra.smid[blockIdx.x] = sm_id();
  phase_init1(ra, sm);
  if (!grid_barrier(ra, 1)) return;
  spread_order(ra, sm);
  phase_init2(ra, sm);
  if (!grid_barrier(ra, 2)) return;
  phase_init3(ra, sm);
  if (!grid_barrier(ra, 6)) return;
  clk.lap(ra, T_INIT);
  for (int it = 0;; ++it) {
    if (all_done(ra)) break;
    if (it >= ra.max_iters) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&ra.bar->overrun, 1);
      break;
    }
    phase_screen(ra, sm);
    if (!grid_barrier(ra, 3)) return;
    clk.lap(ra, T_SCREEN);
    phase_decide(ra, sm);
    if (!grid_barrier(ra, 4)) return;
    clk.lap(ra, T_DECIDE);
    if (ra.sampled) {
      // the refinement of Alg. 1: a scan and a decide per step, then the
      // stop tests on the refined pivots
      for (int k = 0; k < 2 * ra.max_rook && any_rook(ra); ++k) {
        phase_rook_scan(ra, sm);
        if (!grid_barrier(ra, 10)) return;
        phase_rook_decide(ra, sm);
        if (!grid_barrier(ra, 11)) return;
      }
      clk.lap(ra, T_SCREEN);
      phase_finalize(ra, sm);
      if (!grid_barrier(ra, 12)) return;
      clk.lap(ra, T_DECIDE);
    }
    if (ra.mixed) {
      phase_refine(ra, sm);
      if (!grid_barrier(ra, 7)) return;
      clk.lap(ra, T_REFINE);
      phase_decide2(ra, sm);
      if (!grid_barrier(ra, 8)) return;
      clk.lap(ra, T_DECIDE);
    }
    const bool verify = any_verify(ra);
    if (verify) {
      phase_tables(ra);
      if (!grid_barrier(ra, 9)) return;
    }
    phase_update(ra, sm);
    if (!grid_barrier(ra, 5)) return;
    clk.lap(ra, verify ? T_VERIFY : T_UPDATE);
  }
}

__global__ void __launch_bounds__(NT, 2) k_init1(RunArgs ra) {
  cache_inst0(ra);
  phase_init1(ra, *reinterpret_cast<PhaseSmem *>(dyn_smem));
}
__global__ void __launch_bounds__(NT, 2) k_init2(RunArgs ra) {
  cache_inst0(ra);
  phase_init2(ra, *reinterpret_cast<PhaseSmem *>(dyn_smem));
}
__global__ void __launch_bounds__(NT, 2) k_init3(RunArgs ra) {
  cache_inst0(ra);
  phase_init3(ra, *reinterpret_cast<PhaseSmem *>(dyn_smem));
}
__global__ void __launch_bounds__(NT, 2) k_screen(RunArgs ra) {
  cache_inst0(ra);
  phase_screen(ra, *reinterpret_cast<PhaseSmem *>(dyn_smem));
}
__global__ void __launch_bounds__(NT, 2) k_decide(RunArgs ra) {
  cache_inst0(ra);
  phase_decide(ra, *reinterpret_cast<PhaseSmem *>(dyn_smem));
}
__global__ void __launch_bounds__(NT, 2) k_refine(RunArgs ra) {
  cache_inst0(ra);
  phase_refine(ra, *reinterpret_cast<PhaseSmem *>(dyn_smem));
}
__global__ void __launch_bounds__(NT, 2) k_decide2(RunArgs ra) {
  cache_inst0(ra);
  phase_decide2(ra, *reinterpret_cast<PhaseSmem *>(dyn_smem));
}
__global__ void __launch_bounds__(NT, 2) k_rook_scan(RunArgs ra) {
  cache_inst0(ra);
  phase_rook_scan(ra, *reinterpret_cast<PhaseSmem *>(dyn_smem));
}
__global__ void __launch_bounds__(NT, 2) k_rook_decide(RunArgs ra) {
  cache_inst0(ra);
  phase_rook_decide(ra, *reinterpret_cast<PhaseSmem *>(dyn_smem));
}
__global__ void __launch_bounds__(NT, 2) k_finalize(RunArgs ra) {
  cache_inst0(ra);
  phase_finalize(ra, *reinterpret_cast<PhaseSmem *>(dyn_smem));
}
__global__ void __launch_bounds__(NT, 2) k_tables(RunArgs ra) {
  cache_inst0(ra);
  phase_tables(ra);
}
__global__ void __launch_bounds__(NT, 2) k_update(RunArgs ra) {
  cache_inst0(ra);
  phase_update(ra, *reinterpret_cast<PhaseSmem *>(dyn_smem));
}

// cores: G_k = reshape(T_k, [s_{k-1}, n_k, s_k]) (eq. corereshape) written
// row-major from the t-major T; the last core is R of the last bond.
__global__ void k_core(const InstDev *inp, int m, double *dst) {
  const InstDev &in = *inp;
  const Ctrl &cr = *in.ctrl;
  const int d = in.d;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t NTOT = (int64_t)gridDim.x * blockDim.x;
  if (m < d - 1) {
    const BondDev &B = in.bond[m];
    const int rr = cr.r[m];
    const int64_t rows = (int64_t)(m == 0 ? 1 : cr.r[m - 1]) * in.n[m];
    for (int64_t x = gt; x < rows * rr; x += NTOT) {
      const int64_t a = x / rr, t = x - a * rr;
      dst[x] = B.T[t * B.ldT + a];
    }
  } else {
    const BondDev &B = in.bond[d - 2];
    const int rl = cr.r[d - 2];
    const int64_t nn = in.n[d - 1];
    for (int64_t x = gt; x < rl * nn; x += NTOT) {
      const int64_t t = x / nn, j = x - t * nn;
      dst[x] = B.R[t * B.ldR + j];
    }
  }
}

// ---------------------------------------------------------------------------
// host-side launch helpers (declared in ttc_launch.h)

size_t phase_smem_bytes() { return sizeof(PhaseSmem); }

static int64_t host_piece_tiles(int64_t n, int32_t C, int64_t T) {
  const int64_t q = n / C, rem = n - q * C;  // the balanced split of make_pieces
  return rem * ((q + 1 + T - 1) / T) + (C - rem) * ((q + T - 1) / T);
}

int64_t host_tiles(int64_t n_b, int64_t n_b1, int64_t rl, int64_t rr, int32_t pr, int32_t pc) {
  const int64_t nrt = pr > 0 ? rl * host_piece_tiles(n_b, pr, BM) : (rl * n_b + BM - 1) / BM;
  const int64_t nct = pc > 0 ? rr * host_piece_tiles(n_b1, pc, BN) : (n_b1 * rr + BN - 1) / BN;
  return nrt * nct;
}

// Host replay of the screens' tile arithmetic for bond b at ranks r: the
// kernels' own tile_geo_e / tile_rows / tile_cols / carried_tiles, run on
// the host.  Counts the violations: a tile that is empty, wider than te or
// outside the superblock; a tile that crosses a piece of the subtensor grid
// (the pieces recomputed here from the balanced split); a superblock row or
// column that the tiles cover other than exactly once; with r_stored (the
// ranks the stored residual was written at), a carried tile outside the
// stored extent.
int64_t host_check_bond_tiles(int d, const int64_t *n, const int32_t *r, const int32_t *r_stored,
                              const int32_t *grid, int b, int te, int64_t *ntiles) {
  std::unique_ptr<InstDev> in(new InstDev());
  std::unique_ptr<Ctrl> cr(new Ctrl());
  in->d = d;
  in->nb = d - 1;
  for (int m = 0; m < d; ++m) {
    in->n[m] = n[m];
    cr->grid[m] = grid ? grid[m] : 0;
  }
  const TileGeo g = tile_geo_e(*in, *cr, r, b, te);
  int64_t bad = 0;
  auto side = [&](int64_t len, int64_t nm, int32_t pieces, int32_t count, bool rows) {
    std::vector<int32_t> cov((size_t)len, 0);
    for (int32_t t = 0; t < count; ++t) {
      int64_t s0;
      int nl;
      if (rows)
        tile_rows(*in, g, b, t, s0, nl);
      else
        tile_cols(*in, g, b, t, s0, nl);
      if (nl < 1 || nl > te || s0 < 0 || s0 + nl > len) {
        ++bad;
        continue;
      }
      if (pieces > 0) {
        const int64_t i0 = s0 % nm, q = nm / pieces, rem = nm % pieces;
        int64_t k = 0;
        while (k + 1 < pieces && (k + 1) * q + std::min<int64_t>(k + 1, rem) <= i0) ++k;
        const int64_t st = k * q + std::min<int64_t>(k, rem), sz = q + (k < rem ? 1 : 0);
        if ((s0 + nl - 1) / nm != s0 / nm || i0 + nl > st + sz) ++bad;
      }
      for (int64_t x = s0; x < s0 + nl; ++x) ++cov[(size_t)x];
    }
    for (int64_t x = 0; x < len; ++x) bad += cov[(size_t)x] != 1;
  };
  side(g.rows, n[b], g.pr, g.nrt, true);
  side(g.cols, n[b + 1], g.pc, g.nct, false);
  if (r_stored) {
    // stored form: the carried rectangle (row tiles < tr0, column tiles <
    // tc0) lies inside the stored extent at the ranks the residual was last
    // written with, so the carried warp tiles read only carried entries
    const int32_t sr = (int32_t)rows_of(*in, r_stored, b), sc = (int32_t)cols_of(*in, r_stored, b);
    int32_t tr0, tc0;
    carried_tiles(*in, g, b, sr, sc, tr0, tc0);
    if (tr0 < 0 || tr0 > g.nrt || tc0 < 0 || tc0 > g.nct) ++bad;
    for (int32_t t = 0; t < std::min(tr0, g.nrt); ++t) {
      int64_t s0;
      int nl;
      tile_rows(*in, g, b, t, s0, nl);
      if (s0 + nl > sr) ++bad;
    }
    for (int32_t t = 0; t < std::min(tc0, g.nct); ++t) {
      int64_t s0;
      int nl;
      tile_cols(*in, g, b, t, s0, nl);
      if (s0 + nl > sc) ++bad;
    }
  }
  if (ntiles) *ntiles = (int64_t)g.nrt * g.nct;
  return bad;
}

cudaError_t persistent_occupancy(int *blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(PhaseSmem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_persistent, NT,
                                                       sizeof(PhaseSmem));
}

cudaError_t launch_persistent(const RunArgs &ra, int grid, cudaStream_t s) {
  void *args[] = {(void *)&ra};
  return cudaLaunchCooperativeKernel((const void *)k_persistent, dim3(grid), dim3(NT), args,
                                     sizeof(PhaseSmem), s);
}

static cudaError_t prep(const void *f) {
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(PhaseSmem));
}

cudaError_t launch_phase(int phase, const RunArgs &ra, int grid, cudaStream_t s) {
  const void *f = nullptr;
  switch (phase) {
    case PH_INIT1: f = (const void *)k_init1; break;
    case PH_INIT2: f = (const void *)k_init2; break;
    case PH_INIT3: f = (const void *)k_init3; break;
    case PH_SCREEN: f = (const void *)k_screen; break;
    case PH_DECIDE: f = (const void *)k_decide; break;
    case PH_UPDATE: f = (const void *)k_update; break;
    case PH_REFINE: f = (const void *)k_refine; break;
    case PH_DECIDE2: f = (const void *)k_decide2; break;
    case PH_TABLES: f = (const void *)k_tables; break;
    case PH_ROOK_SCAN: f = (const void *)k_rook_scan; break;
    case PH_ROOK_DECIDE: f = (const void *)k_rook_decide; break;
    case PH_FINALIZE: f = (const void *)k_finalize; break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = prep(f);
  if (e != cudaSuccess) return e;
  void *args[] = {(void *)&ra};
  return cudaLaunchKernel(f, dim3(grid), dim3(NT), args, sizeof(PhaseSmem), s);
}

// ---------------------------------------------------------------------------
// Core construction from the pivot sets alone (Alg. 5, second loop; Sec.
// 3.2.2 and eq. corereshape): the history of Alg. 4 is rebuilt for every
// bond, then every superblock row of T_k is replayed from it, sliced over the
// grid (a row per warp), and the last bond's R is formed from the entries.
// By the arithmetic contract every value equals the one the sweeps kept.

// history of bond blockIdx.x (one CTA per bond), step by step: before step
// t every pivot row a_z (z >= t) holds T(a_z, :t); step t takes its column
// c_t = R(:t, c_t) = A(a_u, c_t), its snapshot T(a_t, :t) and delta_t, then
// applies itself to the later pivot rows (a thread per row)
__global__ void __launch_bounds__(NT) k_rebuild_history(const InstDev *inp, double *scratch) {
  const InstDev &in = *inp;
  const int b = blockIdx.x;
  if (b >= in.nb) return;
  const BondDev &B = in.bond[b];
  const int r = in.ctrl->r[b];
  const int64_t cap = B.cap;
  double *Tp = scratch + (int64_t)b * RCAP * RCAP;  // [z][u]: T(a_z, u) of pivot row z
  __shared__ double s_hc[RCAP], s_hp[RCAP];
  __shared__ double s_delta;
  __shared__ int s_ok;
  for (int x = threadIdx.x; x < r * r; x += NT) Tp[x] = 0.0;
  __syncthreads();
  for (int t = 0; t < r; ++t) {
    // c_t restricted to the earlier pivots, and row a_t's snapshot
    for (int u = threadIdx.x; u < t; u += NT) {
      const double c = sb_entry(in, b, B.prow[u], B.pcol[t]);
      s_hc[u] = c;
      s_hp[u] = Tp[(int64_t)t * RCAP + u];
      B.hc[(int64_t)t * cap + u] = c;
      B.hpiv[(int64_t)t * cap + u] = s_hp[u];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const double piv = __dsub_rn(sb_entry(in, b, B.prow[t], B.pcol[t]), chain(s_hp, 1, s_hc, 1, t));
      s_delta = 1.0 / piv;
      s_ok = isfinite(s_delta) ? 1 : 0;
      B.delta[t] = s_delta;
    }
    __syncthreads();
    if (!s_ok) return;  // no such pivot was taken (the sweeps check the same value)
    const double dt = s_delta;
    // step t on the later pivot rows z > t
    for (int z = t + 1 + threadIdx.x; z < r; z += NT) {
      double *Tz = Tp + (int64_t)z * RCAP;
      const double sv = __dsub_rn(chain(Tz, 1, s_hc, 1, t), sb_entry(in, b, B.prow[z], B.pcol[t]));
      const double w = __dmul_rn(dt, sv);
      for (int u = 0; u < t; ++u) Tz[u] = __fma_rn(w, s_hp[u], Tz[u]);
      Tz[t] = -w;
    }
    __syncthreads();
  }
}

// every superblock row of every bond replayed through its whole history
// (Alg. 4), a row per warp, rows dealt over the grid; then R of the last
// bond (its core) from the entries
__global__ void __launch_bounds__(NT, 2) k_rebuild_rows(const InstDev *inp) {
  const InstDev &in = *inp;
  const int64_t nwarps = (int64_t)gridDim.x * (NT / 32);
  const int64_t gw = (int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
  int64_t base = 0;
  for (int b = 0; b < in.nb; ++b) {
    const int r = in.ctrl->r[b];
    const int64_t rows = (int64_t)(b == 0 ? 1 : in.ctrl->r[b - 1]) * in.n[b];
    for (int64_t a = ((gw - base) % nwarps + nwarps) % nwarps; a < rows; a += nwarps) {
      if (r <= 32)
        replay_row_warp<1, true>(in, b, a, r, nullptr, true, 1);
      else if (r <= 64)
        replay_row_warp<2, true>(in, b, a, r, nullptr, true, 1);
      else if (r <= 128)
        replay_row_warp<4, true>(in, b, a, r, nullptr, true, 1);
      else
        replay_row_warp<8, false>(in, b, a, r, nullptr, true, 1);
    }
    base += rows;
  }
  const int bl = in.nb - 1;
  const BondDev &B = in.bond[bl];
  const int r = in.ctrl->r[bl];
  const int64_t nn = in.n[in.d - 1];
  const int64_t gt = (int64_t)blockIdx.x * NT + threadIdx.x, NTOT = (int64_t)gridDim.x * NT;
  for (int64_t x = gt; x < r * nn; x += NTOT) {
    const int64_t t = x / nn, c = x - t * nn;
    putR(in, B, t * B.ldR + c, sb_entry(in, bl, B.prow[t], c));
  }
}

cudaError_t launch_rebuild_cores(const InstDev *d_inst, int nb, double *scratch, int grid,
                                 cudaStream_t s) {
  k_rebuild_history<<<nb, NT, 0, s>>>(d_inst, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_rebuild_rows<<<grid, NT, 0, s>>>(d_inst);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// user generator: the entries that enter the superblocks after a decision.
// For bond b with old / new ranks the superblock grows from ro x co to
// rn x cn (rows, columns); its new entries are, in this order,
//   rows ro..rn-1 x columns 0..cn-1, then rows 0..ro-1 x columns co..cn-1.
// k_user_count sums them per bond (first: every entry of the rank-one
// superblocks); k_user_gather writes their multi-indices, k_user_scatter
// puts the callback's values into the cache at (a, c).

__device__ void user_extent(const InstDev &in, const Ctrl &cr, int b, int first, int64_t &ro,
                            int64_t &co, int64_t &rn, int64_t &cn) {
  const int32_t *r = cr.r, *ad = cr.add;
  const int64_t pl = b == 0 ? 1 : r[b - 1], ql = b == in.nb - 1 ? 1 : r[b + 1];
  const int64_t pa = b == 0 ? 0 : ad[b - 1], qa = b == in.nb - 1 ? 0 : ad[b + 1];
  rn = pl * in.n[b];
  cn = in.n[b + 1] * ql;
  ro = first ? 0 : (pl - pa) * in.n[b];
  co = first ? 0 : in.n[b + 1] * (ql - qa);
}

__global__ void k_user_count(const InstDev *inp, int first, int64_t *counts) {
  const InstDev &in = *inp;
  const Ctrl &cr = *in.ctrl;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t tot = 0;
  for (int b = 0; b < in.nb; ++b) {
    counts[b] = tot;
    int64_t ro, co, rn, cn;
    user_extent(in, cr, b, first, ro, co, rn, cn);
    if (cr.state != ST_DONE) tot += rn * cn - ro * co;
  }
  counts[in.nb] = tot;
}

// entry x of the new entries of bond b -> superblock (a, c)
__device__ __forceinline__ void user_entry(int64_t x, int64_t ro, int64_t co, int64_t rn,
                                           int64_t cn, int64_t &a, int64_t &c) {
  const int64_t top = (rn - ro) * cn;
  if (x < top) {
    a = ro + x / cn;
    c = x - (a - ro) * cn;
  } else {
    const int64_t y = x - top, w = cn - co;
    a = y / w;
    c = co + (y - a * w);
  }
}

__global__ void k_user_gather(const InstDev *inp, int first, const int64_t *counts, int32_t *idx) {
  const InstDev &in = *inp;
  const Ctrl &cr = *in.ctrl;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t NTOT = (int64_t)gridDim.x * blockDim.x;
  for (int b = 0; b < in.nb; ++b) {
    int64_t ro, co, rn, cn;
    user_extent(in, cr, b, first, ro, co, rn, cn);
    const int64_t base = counts[b], cnt = counts[b + 1] - base;
    const SetDev &L = left_set(in, b), &Rs = right_set(in, b);
    const int wl = b, wr = in.d - b - 2;
    for (int64_t x = gt; x < cnt; x += NTOT) {
      int64_t a, c;
      user_entry(x, ro, co, rn, cn, a, c);
      const int64_t p = a / in.n[b], i = a - p * in.n[b];
      const int64_t q = c / in.n[b + 1], j = c - q * in.n[b + 1];
      int32_t *o = idx + (base + x) * in.d;
      for (int m = 0; m < wl; ++m) o[m] = L.idx[p * wl + m];
      o[b] = (int32_t)i;
      o[b + 1] = (int32_t)j;
      for (int m = 0; m < wr; ++m) o[b + 2 + m] = Rs.idx[q * wr + m];
    }
  }
}

__global__ void k_user_scatter(const InstDev *inp, int first, const int64_t *counts,
                               const double *vals) {
  const InstDev &in = *inp;
  const Ctrl &cr = *in.ctrl;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t NTOT = (int64_t)gridDim.x * blockDim.x;
  for (int b = 0; b < in.nb; ++b) {
    int64_t ro, co, rn, cn;
    user_extent(in, cr, b, first, ro, co, rn, cn);
    const int64_t base = counts[b], cnt = counts[b + 1] - base;
    const BondDev &B = in.bond[b];
    for (int64_t x = gt; x < cnt; x += NTOT) {
      int64_t a, c;
      user_entry(x, ro, co, rn, cn, a, c);
      B.A[a * B.ldR + c] = vals[base + x];
    }
  }
}

// the error samples' multi-indices, then the origin's
__global__ void k_user_samples(const InstDev *inp, int32_t *idx) {
  const InstDev &in = *inp;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t NTOT = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = gt; k <= in.nsamples; k += NTOT) {
    int32_t *o = idx + k * in.d;
    if (k == in.nsamples) {
      for (int m = 0; m < in.d; ++m) o[m] = 0;
    } else {
      for (int m = 0; m < in.d; ++m) o[m] = sample_coord(in, k, m);
    }
  }
}

cudaError_t launch_user_count(const InstDev *d_inst, int first, int64_t *counts, cudaStream_t s) {
  k_user_count<<<1, 32, 0, s>>>(d_inst, first, counts);
  return cudaGetLastError();
}
cudaError_t launch_user_gather(const InstDev *d_inst, int first, const int64_t *counts,
                               int32_t *idx, cudaStream_t s) {
  k_user_gather<<<152 * 4, 256, 0, s>>>(d_inst, first, counts, idx);
  return cudaGetLastError();
}
cudaError_t launch_user_scatter(const InstDev *d_inst, int first, const int64_t *counts,
                                const double *vals, cudaStream_t s) {
  k_user_scatter<<<152 * 4, 256, 0, s>>>(d_inst, first, counts, vals);
  return cudaGetLastError();
}
cudaError_t launch_user_samples(const InstDev *d_inst, int32_t *idx, cudaStream_t s) {
  k_user_samples<<<152 * 4, 256, 0, s>>>(d_inst, idx);
  return cudaGetLastError();
}

// Maxwellian tables of an instance (create time)
__global__ void k_maxwellian_tables(const InstDev *inp, double *coef, double *nh, double *cosx) {
  const InstDev &in = *inp;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t NTOT = (int64_t)gridDim.x * blockDim.x;
  if (in.gen == 3) {
    for (int m = 0; m < in.d; ++m)
      for (int64_t i = gt; i < in.n[m]; i += NTOT)
        maxwellian_xv_table_entry(in, m, i, coef + in.mx_off[m] + i, nh + in.mx_off[m] + i);
    return;
  }
  int64_t ncombo = 1;
  for (int m = 0; m < in.dx; ++m) ncombo *= in.n[m];
  for (int64_t c = gt; c < ncombo; c += NTOT) maxwellian_table_entry(in, c, coef + c, nh + c);
  const double two_pi = 6.283185307179586476925286766559;
  for (int m = 0; m < in.dx; ++m)
    for (int64_t i = gt; i < in.n[m]; i += NTOT)
      cosx[in.mx_off[m] + i] = cos(__dmul_rn(two_pi, (double)i) / (double)in.n[m]);
}

cudaError_t launch_maxwellian_tables(const InstDev *d_inst, double *coef, double *nh, double *cosx) {
  k_maxwellian_tables<<<152 * 4, 256>>>(d_inst, coef, nh, cosx);
  return cudaGetLastError();
}

cudaError_t launch_core(const InstDev *d_inst, int m, double *dst, cudaStream_t s) {
  k_core<<<152, 256, 0, s>>>(d_inst, m, dst);
  return cudaGetLastError();
}


}  // namespace ttc
