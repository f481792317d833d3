/*
 * ttc_oracle.c -- CPU FP64 oracle for the adaptive TT cross (arXiv 2407.11290).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product library.
 *
 * Plain loops, binary64, explicit fma(), compiled without FP contraction.
 * Every step names the passage of the paper it follows; the arithmetic
 * contract is written out in ttc_oracle.h.
 *
 * Index conventions (0-based; the paper counts from 1):
 *   modes m = 0..d-1, bonds b = 0..d-2 (the paper's k = b+1).
 *   I[b] = I_{<=k}: r_b multi-indices over modes 0..b.
 *   J[b] = J_{>k} : r_b multi-indices over modes b+1..d-1.
 *   Superblock of bond b (Alg. 2): rows (alpha in I[b-1], i_b) -> a = p*n_b + i,
 *   columns (i_{b+1}, beta in J[b+1]) -> c = q*n_{b+1} + j.
 *   T_b = C_b U_b has one row per superblock row, R_b = X(I[b], superblock cols).
 */
#include "ttc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

struct orc_state {
  int d;
  int64_t n[ORC_MAXD];
  int64_t stride[ORC_MAXD]; /* prod_{l<m} n_l: column-major linear index */
  int kind;
  int32_t rho[ORC_MAXD + 1];
  int64_t core_off[ORC_MAXD + 1];
  double *tt; /* copied TT cores */
  int32_t dx, dv;
  double a_rho, a_u, a_T, vmin, vmax;
  int nthreads;

  int32_t maxr[ORC_MAXD];
  int32_t r[ORC_MAXD];
  int64_t rows_cap[ORC_MAXD], cols_cap[ORC_MAXD];
  int32_t *I[ORC_MAXD]; /* [cap][b+1] */
  int32_t *J[ORC_MAXD]; /* [cap][d-1-b] */
  int32_t *prow[ORC_MAXD], *pcol[ORC_MAXD];
  double *T[ORC_MAXD];  /* [rows_cap][cap] */
  double *R[ORC_MAXD];  /* [cap][cols_cap] */
  double *U[ORC_MAXD];  /* [cap][cap] */
  double *hdelta[ORC_MAXD];
  double *hpiv[ORC_MAXD]; /* [cap][cap]: row z = T(a_z, 0..z-1) before step z */
  double *hc[ORC_MAXD];   /* [cap][cap]: row z = A(a_t, c_z), t < z */
  /* stored-residual form (eq. aca_approx_E): E[b] [rows_cap][cols_cap], valid
     on rows < st_rows[b] and columns < st_cols[b] */
  int stored;
  double *E[ORC_MAXD];
  int64_t st_rows[ORC_MAXD], st_cols[ORC_MAXD];
  /* Alg. 1 with a random sample set (recompute form): nl samples per bond
     and screen, SplitMix64 seeded with lseed, at most max_rook rounds of
     the row / column refinement; nl = 0 screens the whole superblock */
  int64_t nl;
  uint64_t lseed;
  int max_rook;
  int64_t screens;        /* screens since the start (the sample counter) */
  int64_t last_screened;  /* entries evaluated by the last screen */
  int64_t rook_moves;     /* refinement steps that moved a pivot */
  int initialized;
};

static uint64_t splitmix64_at(uint64_t seed, uint64_t k);

/* ------------------------------------------------------------------------- */
/* The arithmetic contract's dot product: a serial FMA chain from +0.        */
static double chain(const double *x, int64_t sx, const double *y, int64_t sy,
                    int K) {
  double acc = 0.0;
  for (int t = 0; t < K; ++t) acc = fma(x[t * sx], y[t * sy], acc);
  return acc;
}

/* ------------------------------------------------------------------------- */
/* Tensor entries (Sec. 5: the tensor is a function of its indices).         */

/* Hilbert tensor, eq. HilbertTensor shifted to 0-based indices. */
static double hilbert(const orc_state *s, const int32_t *idx) {
  int64_t sum = 1;
  for (int m = 0; m < s->d; ++m) sum += idx[m];
  return 1.0 / (double)sum;
}

/* A TT given by its cores (Sec. 2.2): left-to-right product of the slices. */
static double tt_entry(const orc_state *s, const int32_t *idx) {
  double v[256], w[256];
  int rl = s->rho[1];
  const double *G0 = s->tt + s->core_off[0];
  for (int t = 0; t < rl; ++t) v[t] = G0[(int64_t)idx[0] * rl + t];
  for (int m = 1; m < s->d; ++m) {
    int ra = s->rho[m], rb = s->rho[m + 1];
    const double *G = s->tt + s->core_off[m];
    for (int q = 0; q < rb; ++q)
      w[q] = chain(v, 1, G + (int64_t)idx[m] * rb + q, s->n[m] * rb, ra);
    for (int q = 0; q < rb; ++q) v[q] = w[q];
  }
  return v[0];
}

/* Maxwellian f(x,v) = rho(x) (2 pi T(x))^{-dv/2} exp(-|v-u(x)|^2 / (2 T(x))) */
static double maxwellian(const orc_state *s, const int32_t *idx) {
  const double two_pi = 6.283185307179586476925286766559;
  double x[ORC_MAXD], prod_sin = 1.0, sum_x = 0.0;
  for (int m = 0; m < s->dx; ++m) {
    x[m] = two_pi * (double)idx[m] / (double)s->n[m];
    prod_sin *= sin(x[m]);
    sum_x += x[m];
  }
  double rho = 1.0 + s->a_rho * prod_sin;
  double T = 1.0 + s->a_T * cos(sum_x);
  double q = 0.0;
  for (int j = 0; j < s->dv; ++j) {
    int m = s->dx + j;
    double v = s->vmin + (s->vmax - s->vmin) * (double)idx[m] / (double)(s->n[m] - 1);
    double u = s->a_u * cos(x[(j + 1) % s->dx]);
    double dvu = v - u;
    q += dvu * dvu;
  }
  return rho / pow(two_pi * T, 0.5 * (double)s->dv) * exp(-q / (2.0 * T));
}

/* The 2d2v / 3d3v distribution of Sec. 5.2 (eq. 2d2vFunction and its 3d3v
   extension), modes interleaved (x, v_x, y, v_y[, z, v_z]):
     f = sum_q rho(s_q) / (2 sqrt(2 pi T(s_q)))
         * [exp(-sum_q b_q^-) + exp(-sum_q b_q^+)],  b_q^± = (v_q ± a_u)^2 / (2 T(s_q)),
   rho(s) = 1 + a_rho sin(2 pi s), T(s) = 1/2 + a_T sin(2 pi s), positions
   s = -1/2 + i / (n - 1), velocities v = vmin + (vmax - vmin) i / (n - 1). */
static double maxwellian_xv(const orc_state *s, const int32_t *idx) {
  const double two_pi = 6.283185307179586476925286766559;
  double rs = 0.0, bm = 0.0, bp = 0.0;
  for (int q = 0; q < s->dx; ++q) {
    double sv = -0.5 + (double)idx[2 * q] / (double)(s->n[2 * q] - 1);
    double sn = sin(two_pi * sv);
    double rho = 1.0 + s->a_rho * sn;
    double T = 0.5 + s->a_T * sn;
    double v = s->vmin + (s->vmax - s->vmin) * (double)idx[2 * q + 1] / (double)(s->n[2 * q + 1] - 1);
    double dm = v - s->a_u, dp = v + s->a_u;
    rs = rs + rho / (2.0 * sqrt(two_pi * T));
    bm = bm + (dm * dm) * (1.0 / (2.0 * T));
    bp = bp + (dp * dp) * (1.0 / (2.0 * T));
  }
  return rs * (exp(-bm) + exp(-bp));
}

double orc_entry(const orc_state *s, const int32_t *idx) {
  switch (s->kind) {
    case ORC_GEN_HILBERT: return hilbert(s, idx);
    case ORC_GEN_TT: return tt_entry(s, idx);
    case ORC_GEN_MAXWELLIAN_XV: return maxwellian_xv(s, idx);
    default: return maxwellian(s, idx);
  }
}

static int64_t lin_index(const orc_state *s, const int32_t *idx) {
  int64_t l = 0;
  for (int m = 0; m < s->d; ++m) l += (int64_t)idx[m] * s->stride[m];
  return l;
}

/* ------------------------------------------------------------------------- */
/* Superblock geometry (Alg. 2 line 2).                                      */
static int64_t rows_of(const orc_state *s, int b) {
  return (b == 0 ? 1 : s->r[b - 1]) * s->n[b];
}
static int64_t cols_of(const orc_state *s, int b) {
  return s->n[b + 1] * (b == s->d - 2 ? 1 : s->r[b + 1]);
}

/* Full multi-index of superblock entry (a, c) of bond b. */
static void sb_index(const orc_state *s, int b, int64_t a, int64_t c,
                     int32_t *idx) {
  int64_t p = a / s->n[b], i = a % s->n[b];
  int64_t q = c / s->n[b + 1], j = c % s->n[b + 1];
  if (b > 0) memcpy(idx, s->I[b - 1] + p * b, sizeof(int32_t) * b);
  idx[b] = (int32_t)i;
  idx[b + 1] = (int32_t)j;
  int nb = s->d - b - 2; /* modes b+2..d-1 */
  if (nb > 0) memcpy(idx + b + 2, s->J[b + 1] + q * nb, sizeof(int32_t) * nb);
}

static double sb_entry(const orc_state *s, int b, int64_t a, int64_t c) {
  int32_t idx[ORC_MAXD];
  sb_index(s, b, a, c, idx);
  return orc_entry(s, idx);
}

/* ------------------------------------------------------------------------- */
orc_state *orc_create(int d, const int64_t *n, const orc_gen *g,
                      const int32_t *maxr, int nthreads) {
  if (d < 2 || d > ORC_MAXD || !n || !g || !maxr) return NULL;
  orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
  if (!s) return NULL;
  s->d = d;
  s->kind = g->kind;
  s->nthreads = nthreads < 1 ? 1 : nthreads;
  int64_t st = 1;
  for (int m = 0; m < d; ++m) {
    if (n[m] < 1) { free(s); return NULL; }
    s->n[m] = n[m];
    s->stride[m] = st;
    st *= n[m];
  }
  if (g->kind == ORC_GEN_TT) {
    int64_t tot = 0;
    for (int m = 0; m <= d; ++m) s->rho[m] = g->tt_ranks[m];
    if (s->rho[0] != 1 || s->rho[d] != 1) { free(s); return NULL; }
    for (int m = 0; m < d; ++m) {
      if (s->rho[m + 1] > 256) { free(s); return NULL; }
      s->core_off[m] = tot;
      tot += (int64_t)s->rho[m] * n[m] * s->rho[m + 1];
    }
    s->tt = (double *)malloc(sizeof(double) * tot);
    memcpy(s->tt, g->tt_cores, sizeof(double) * tot);
  } else if (g->kind == ORC_GEN_MAXWELLIAN) {
    s->dx = g->dx; s->dv = g->dv;
    s->a_rho = g->a_rho; s->a_u = g->a_u; s->a_T = g->a_T;
    s->vmin = g->vmin; s->vmax = g->vmax;
    if (s->dx < 1 || s->dv < 1 || s->dx + s->dv != d) { free(s); return NULL; }
  } else if (g->kind == ORC_GEN_MAXWELLIAN_XV) {
    s->dx = g->dx; s->dv = g->dv;
    s->a_rho = g->a_rho; s->a_u = g->a_u; s->a_T = g->a_T;
    s->vmin = g->vmin; s->vmax = g->vmax;
    if (s->dx < 1 || s->dv != s->dx || 2 * s->dx != d) { free(s); return NULL; }
    for (int m = 0; m < d; ++m) if (n[m] < 2) { free(s); return NULL; }
  } else if (g->kind != ORC_GEN_HILBERT) {
    free(s);
    return NULL;
  }
  for (int b = 0; b < d - 1; ++b) {
    int cap = maxr[b] < 1 ? 1 : maxr[b];
    if (cap > 1024) { free(s->tt); free(s); return NULL; }
    s->maxr[b] = cap;
  }
  for (int b = 0; b < d - 1; ++b) {
    int64_t cap = s->maxr[b];
    int64_t capL = b == 0 ? 1 : s->maxr[b - 1];
    int64_t capR = b == d - 2 ? 1 : s->maxr[b + 1];
    s->rows_cap[b] = capL * n[b];
    s->cols_cap[b] = n[b + 1] * capR;
    s->I[b] = (int32_t *)calloc(cap * (b + 1), sizeof(int32_t));
    s->J[b] = (int32_t *)calloc(cap * (d - 1 - b), sizeof(int32_t));
    s->prow[b] = (int32_t *)calloc(cap, sizeof(int32_t));
    s->pcol[b] = (int32_t *)calloc(cap, sizeof(int32_t));
    s->T[b] = (double *)calloc(s->rows_cap[b] * cap, sizeof(double));
    s->R[b] = (double *)calloc(cap * s->cols_cap[b], sizeof(double));
    s->U[b] = (double *)calloc(cap * cap, sizeof(double));
    s->hdelta[b] = (double *)calloc(cap, sizeof(double));
    s->hpiv[b] = (double *)calloc(cap * cap, sizeof(double));
    s->hc[b] = (double *)calloc(cap * cap, sizeof(double));
    if (!s->I[b] || !s->J[b] || !s->T[b] || !s->R[b] || !s->U[b] ||
        !s->hpiv[b] || !s->hc[b]) {
      orc_destroy(s);
      return NULL;
    }
  }
  return s;
}

void orc_destroy(orc_state *s) {
  if (!s) return;
  for (int b = 0; b < ORC_MAXD; ++b) {
    free(s->I[b]); free(s->J[b]); free(s->prow[b]); free(s->pcol[b]);
    free(s->T[b]); free(s->R[b]); free(s->U[b]);
    free(s->hdelta[b]); free(s->hpiv[b]); free(s->hc[b]);
    free(s->E[b]);
  }
  free(s->tt);
  free(s);
}

int orc_set_stored(orc_state *s, int on) {
  if (!on) { s->stored = 0; return ORC_OK; }
  for (int b = 0; b < s->d - 1; ++b) {
    if (s->E[b]) continue;
    s->E[b] = (double *)calloc((size_t)(s->rows_cap[b] * s->cols_cap[b]), sizeof(double));
    if (!s->E[b]) return ORC_ERR_OOM;
  }
  s->stored = 1;
  for (int b = 0; b < s->d - 1; ++b) s->st_rows[b] = s->st_cols[b] = 0;
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Alg. 4 for one row: rebuild T(a,:) from the pivot history of bond b by
   applying eq. aca_approx_T_sub once per pivot, in insertion order.         */
static void replay_row(const orc_state *s, int b, int64_t a, int nz) {
  int64_t cap = s->maxr[b];
  double *Ta = s->T[b] + a * cap;
  for (int z = 0; z < nz; ++z) {
    const double *cz = s->hc[b] + z * cap;
    const double *Tp = s->hpiv[b] + z * cap;
    double sv = chain(Ta, 1, cz, 1, z) - sb_entry(s, b, a, s->pcol[b][z]);
    double w = s->hdelta[b][z] * sv;
    for (int t = 0; t < z; ++t) Ta[t] = fma(w, Tp[t], Ta[t]);
    Ta[z] = -w;
  }
}

/* ------------------------------------------------------------------------- */
/* Start: every bond takes the same first pivot, the multi-index `start`, so
   all ranks are 1.  Step z = 0 of eq. aca_approx_T with an empty T gives
   T(:,0) = A(:,c_0) / A(a_0,c_0) in the form delta*A.                      */
int orc_init_at(orc_state *s, const int32_t *start) {
  int d = s->d;
  for (int m = 0; m < d; ++m)
    if (start[m] < 0 || start[m] >= s->n[m]) return ORC_ERR_INVALID_ARG;
  double x0 = orc_entry(s, start);
  if (x0 == 0.0) return ORC_ERR_ZERO_START;
  if (!isfinite(x0)) return ORC_ERR_NONFINITE;
  for (int b = 0; b < d - 1; ++b) {
    memcpy(s->I[b], start, sizeof(int32_t) * (b + 1));
    memcpy(s->J[b], start + b + 1, sizeof(int32_t) * (d - 1 - b));
    s->r[b] = 1;
    /* row (p = 0, i_b), column (i_{b+1}, q = 0) of the superblock */
    s->prow[b][0] = start[b];
    s->pcol[b][0] = start[b + 1];
  }
  for (int b = 0; b < d - 1; ++b) {
    int64_t rows = rows_of(s, b), cols = cols_of(s, b);
    int64_t a0 = s->prow[b][0], c0 = s->pcol[b][0];
    for (int64_t c = 0; c < cols; ++c) s->R[b][c] = sb_entry(s, b, a0, c);
    double piv = sb_entry(s, b, a0, c0) - 0.0;
    double delta = 1.0 / piv;
    if (!isfinite(delta)) return ORC_ERR_NONFINITE;
    s->hdelta[b][0] = delta;
    s->U[b][0] = delta;
    for (int64_t a = 0; a < rows; ++a) replay_row(s, b, a, 1);
    s->st_rows[b] = s->st_cols[b] = 0; /* nothing stored yet */
  }
  s->screens = 0;
  s->rook_moves = 0;
  s->initialized = 1;
  return ORC_OK;
}

int orc_set_sampled(orc_state *s, int64_t nl, uint64_t seed, int max_rook) {
  if (nl < 0 || max_rook < 0) return ORC_ERR_INVALID_ARG;
  s->nl = nl;
  s->lseed = seed;
  s->max_rook = max_rook;
  return ORC_OK;
}

int orc_init(orc_state *s) {
  int32_t zero[ORC_MAXD] = {0};
  return orc_init_at(s, zero);
}

/* ------------------------------------------------------------------------- */
/* Alg. 1 line 1 with L = the whole superblock: argmax |A - T R|.            */
typedef struct {
  double v;
  int64_t lin;
  int64_t a, c;
  double maxabs;
  int bad;
} best_t;

static int better(double v, int64_t lin, const best_t *b) {
  return v > b->v || (v == b->v && lin < b->lin);
}

static best_t screen_rows(const orc_state *s, int b, int64_t a0, int64_t a1) {
  best_t bt;
  bt.v = -1.0; bt.lin = INT64_MAX; bt.a = -1; bt.c = -1; bt.maxabs = 0.0; bt.bad = 0;
  int64_t cols = cols_of(s, b);
  int64_t cap = s->maxr[b];
  int K = s->r[b];
  int32_t idx[ORC_MAXD];
  for (int64_t a = a0; a < a1; ++a) {
    const double *Ta = s->T[b] + a * cap;
    double *Ea = s->stored ? s->E[b] + a * s->cols_cap[b] : NULL;
    for (int64_t c = 0; c < cols; ++c) {
      sb_index(s, b, a, c, idx);
      double e;
      if (Ea && a < s->st_rows[b] && c < s->st_cols[b]) {
        /* stored form: the residual kept from the last screen, already
           carried through the rank-one steps since (eq. aca_approx_E) */
        e = Ea[c];
      } else {
        /* an entry seen for the first time: E = A - T R */
        double A = orc_entry(s, idx);
        e = A - chain(Ta, 1, s->R[b] + c, s->cols_cap[b], K);
        if (Ea) Ea[c] = e;
        if (fabs(A) > bt.maxabs) bt.maxabs = fabs(A);
      }
      if (!isfinite(e)) { bt.bad = 1; continue; }
      double v = fabs(e);
      int64_t lin = lin_index(s, idx);
      if (better(v, lin, &bt)) { bt.v = v; bt.lin = lin; bt.a = a; bt.c = c; }
    }
  }
  return bt;
}

/* Residual E(a,c) = A - chain(T(a,:), R(:,c)) of one superblock entry as
   best_t candidate bookkeeping: keeps (|E|, lin) under the tie rule. */
static void take_entry(const orc_state *s, int b, int64_t a, int64_t c, best_t *bt) {
  int32_t idx[ORC_MAXD];
  sb_index(s, b, a, c, idx);
  double A = orc_entry(s, idx);
  double e = A - chain(s->T[b] + a * s->maxr[b], 1, s->R[b] + c, s->cols_cap[b], s->r[b]);
  if (!isfinite(e)) { bt->bad = 1; return; }
  double v = fabs(e);
  int64_t lin = lin_index(s, idx);
  if (better(v, lin, bt)) { bt->v = v; bt->lin = lin; bt->a = a; bt->c = c; }
}

/* Alg. 1 on the superblock of bond b with a random sample set L:
     - L = nl entries (a, c) drawn with replacement, sample j of bond b in
       screen t from SplitMix64 outputs 2k and 2k+1, k = (t (d-1) + b) nl + j,
       a = floor(x rows / 2^64), c = floor(x' cols / 2^64);
     - (a*, c*) = argmax over L of |E| (ties: lowest linear index);
     - refinement (the while loop of Alg. 1): a* moves to the argmax of column
       c*, then c* to the argmax of row a*, each only to a strictly larger
       |E|; repeated until a round moves neither (the pivot then dominates
       its row and column) or max_rook rounds have run.                     */
static best_t sampled_screen(orc_state *s, int b) {
  const int64_t rows = rows_of(s, b), cols = cols_of(s, b);
  const int64_t t = s->screens;
  best_t parts[256];
  int nt = s->nthreads > 256 ? 256 : s->nthreads;
  if (nt > s->nl) nt = s->nl < 1 ? 1 : (int)s->nl;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nt) schedule(static, 1)
#endif
  for (int th = 0; th < nt; ++th) {
    best_t bt = {-1.0, INT64_MAX, -1, -1, 0.0, 0};
    const int64_t j0 = s->nl * th / nt, j1 = s->nl * (th + 1) / nt;
    for (int64_t j = j0; j < j1; ++j) {
      const uint64_t k = (uint64_t)((t * (s->d - 1) + b) * s->nl + j);
      const uint64_t x0 = splitmix64_at(s->lseed, 2 * k), x1 = splitmix64_at(s->lseed, 2 * k + 1);
      const int64_t a = (int64_t)(uint64_t)(((unsigned __int128)x0 * (uint64_t)rows) >> 64);
      const int64_t c = (int64_t)(uint64_t)(((unsigned __int128)x1 * (uint64_t)cols) >> 64);
      take_entry(s, b, a, c, &bt);
    }
    parts[th] = bt;
  }
  best_t bt = parts[0];
  for (int th = 1; th < nt; ++th) {
    if (parts[th].a >= 0 && (bt.a < 0 || better(parts[th].v, parts[th].lin, &bt))) bt = parts[th];
    bt.bad |= parts[th].bad;
  }
  int64_t evaluated = s->nl;
  for (int round = 0; round < s->max_rook && bt.a >= 0 && !bt.bad; ++round) {
    int moved = 0;
    /* column c*: the best row */
    best_t col = {-1.0, INT64_MAX, -1, -1, 0.0, 0};
    for (int64_t a = 0; a < rows; ++a) take_entry(s, b, a, bt.c, &col);
    evaluated += rows;
    bt.bad |= col.bad;
    if (col.a >= 0 && col.v > bt.v) { bt.v = col.v; bt.lin = col.lin; bt.a = col.a; moved = 1; }
    /* row a*: the best column */
    best_t row = {-1.0, INT64_MAX, -1, -1, 0.0, 0};
    for (int64_t c = 0; c < cols; ++c) take_entry(s, b, bt.a, c, &row);
    evaluated += cols;
    bt.bad |= row.bad;
    if (row.a >= 0 && row.v > bt.v) { bt.v = row.v; bt.lin = row.lin; bt.c = row.c; moved = 1; }
    s->rook_moves += moved;
    if (!moved) break;
  }
  s->last_screened += evaluated;
  return bt;
}

double orc_residual(const orc_state *s, int b, int64_t a, int64_t c) {
  return sb_entry(s, b, a, c) -
         chain(s->T[b] + a * s->maxr[b], 1, s->R[b] + c, s->cols_cap[b], s->r[b]);
}

double orc_stored_residual(const orc_state *s, int b, int64_t a, int64_t c) {
  if (!s->stored || a >= s->st_rows[b] || c >= s->st_cols[b]) return NAN;
  return s->E[b][a * s->cols_cap[b] + c];
}

int orc_screen(orc_state *s, double *best, int64_t *lin, int32_t *row,
               int32_t *col, double *maxabs) {
  if (!s->initialized) return ORC_ERR_INVALID_ARG;
  int bad = 0;
  s->last_screened = 0;
  if (s->nl > 0 && !s->stored) {
    for (int b = 0; b < s->d - 1; ++b) {
      best_t bt = sampled_screen(s, b);
      bad |= bt.bad;
      best[b] = bt.v; lin[b] = bt.lin;
      row[b] = (int32_t)bt.a; col[b] = (int32_t)bt.c;
      maxabs[b] = 0.0;
    }
    s->screens += 1;
    return bad ? ORC_ERR_NONFINITE : ORC_OK;
  }
  for (int b = 0; b < s->d - 1; ++b) {
    int64_t rows = rows_of(s, b);
    int nt = s->nthreads;
    if (nt > rows) nt = (int)rows;
    best_t part[256];
    if (nt > 256) nt = 256;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nt) schedule(static, 1)
#endif
    for (int th = 0; th < nt; ++th) {
      int64_t a0 = rows * th / nt, a1 = rows * (th + 1) / nt;
      part[th] = screen_rows(s, b, a0, a1);
    }
    /* deterministic merge: the key order is total, so the split of rows
       between threads cannot change the winner (the global best is the best
       of the local bests, Sec. 3.2.1) */
    best_t bt = part[0];
    double mx = part[0].maxabs;
    int bd = part[0].bad;
    for (int th = 1; th < nt; ++th) {
      if (part[th].a >= 0 && (bt.a < 0 || better(part[th].v, part[th].lin, &bt))) bt = part[th];
      if (part[th].maxabs > mx) mx = part[th].maxabs;
      bd |= part[th].bad;
    }
    bt.maxabs = mx;
    bt.bad = bd;
    bad |= bt.bad;
    if (s->stored) { s->st_rows[b] = rows; s->st_cols[b] = cols_of(s, b); }
    best[b] = bt.v; lin[b] = bt.lin;
    row[b] = (int32_t)bt.a; col[b] = (int32_t)bt.c;
    maxabs[b] = bt.maxabs;
    s->last_screened += rows * cols_of(s, b);
  }
  s->screens += 1;
  return bad ? ORC_ERR_NONFINITE : ORC_OK;
}

int64_t orc_last_screened(const orc_state *s) { return s->last_screened; }
int64_t orc_rook_moves(const orc_state *s) { return s->rook_moves; }

/* ------------------------------------------------------------------------- */
/* One pivot step on every bond that adds (eq. aca_approx_T, Sec. 3.1.1),
   then the superblock extensions implied by the neighbours' new pivots
   (nestedness, eq. nestedpivots; new rows by Alg. 4).                      */
int orc_apply(orc_state *s, const int32_t *add, const int32_t *row,
              const int32_t *col) {
  int d = s->d;
  int32_t r_old[ORC_MAXD];
  for (int b = 0; b < d - 1; ++b) {
    r_old[b] = s->r[b];
    if (add[b] && s->r[b] >= s->maxr[b]) return ORC_ERR_INVALID_ARG;
    if (add[b] && (row[b] < 0 || row[b] >= rows_of(s, b) || col[b] < 0 ||
                   col[b] >= cols_of(s, b)))
      return ORC_ERR_INVALID_ARG;
  }
  /* (0) stored form, eq. aca_approx_E on the sweep-start superblock:
     E <- E - E(:,c*) E(a*,:) / E(a*,c*), entry by entry
       E(a,c) = fma(w_a, E(a*,c), E(a,c)),  w_a = -(E(a,c*) / E(a*,c*))
     (w_{a*} = -1 exactly, so row a* becomes exactly zero). */
  if (s->stored) {
    for (int b = 0; b < d - 1; ++b) {
      if (!add[b]) continue;
      int64_t rows = s->st_rows[b], cols = s->st_cols[b], ld = s->cols_cap[b];
      if (rows != rows_of(s, b) || cols != cols_of(s, b)) return ORC_ERR_INVALID_ARG;
      double *E = s->E[b];
      int64_t as = row[b], cs = col[b];
      double piv = E[as * ld + cs];
      double *erow = (double *)malloc(sizeof(double) * cols);
      double *w = (double *)malloc(sizeof(double) * rows);
      if (!erow || !w) { free(erow); free(w); return ORC_ERR_OOM; }
      for (int64_t c = 0; c < cols; ++c) erow[c] = E[as * ld + c];
      for (int64_t a = 0; a < rows; ++a) w[a] = -(E[a * ld + cs] / piv);
#ifdef _OPENMP
#pragma omp parallel for num_threads(s->nthreads) schedule(static)
#endif
      for (int64_t a = 0; a < rows; ++a)
        for (int64_t c = 0; c < cols; ++c)
          E[a * ld + c] = fma(w[a], erow[c], E[a * ld + c]);
      free(erow);
      free(w);
    }
  }
  /* (1) pivot step on the sweep-start superblocks */
  for (int b = 0; b < d - 1; ++b) {
    if (!add[b]) continue;
    int z = s->r[b];
    int64_t cap = s->maxr[b];
    int64_t as = row[b], cs = col[b];
    int64_t rows = rows_of(s, b), cols = cols_of(s, b);
    /* new pivot multi-indices: I_{<=k} gets (alpha*, i*), J_{>k} (j*, beta*) */
    int64_t p = as / s->n[b], i = as % s->n[b];
    int64_t q = cs / s->n[b + 1], j = cs % s->n[b + 1];
    int32_t *In = s->I[b] + (int64_t)z * (b + 1);
    if (b > 0) memcpy(In, s->I[b - 1] + p * b, sizeof(int32_t) * b);
    In[b] = (int32_t)i;
    int nj = d - 1 - b;
    int32_t *Jn = s->J[b] + (int64_t)z * nj;
    Jn[0] = (int32_t)j;
    if (nj > 1) memcpy(Jn + 1, s->J[b + 1] + q * (nj - 1), sizeof(int32_t) * (nj - 1));
    /* history of step z: c_z = A(I, j*) = R(:, c*), delta, T(a*,:) */
    double *cz = s->hc[b] + z * cap;
    double *Tp = s->hpiv[b] + z * cap;
    for (int t = 0; t < z; ++t) cz[t] = s->R[b][t * s->cols_cap[b] + cs];
    const double *Tas = s->T[b] + as * cap;
    for (int t = 0; t < z; ++t) Tp[t] = Tas[t];
    double piv = sb_entry(s, b, as, cs) - chain(Tas, 1, cz, 1, z);
    double delta = 1.0 / piv;
    if (!isfinite(delta)) return ORC_ERR_NONFINITE;
    s->hdelta[b][z] = delta;
    /* U_{z+1} by the bordered Sherman-Morrison form of Sec. 3.1.1 with
       a = A(I, j*) and b = A(i*, J): [[U + d U a b U, -d U a], [-d b U, d]] */
    {
      double *U = s->U[b];
      double ua[1024], bu[1024], brow[1024];
      for (int t = 0; t < z; ++t) brow[t] = sb_entry(s, b, as, s->pcol[b][t]);
      for (int t = 0; t < z; ++t) ua[t] = chain(U + t * cap, 1, cz, 1, z);
      for (int t = 0; t < z; ++t) bu[t] = chain(brow, 1, U + t, cap, z);
      for (int t = 0; t < z; ++t) {
        double du = delta * ua[t];
        for (int u = 0; u < z; ++u) U[t * cap + u] = fma(du, bu[u], U[t * cap + u]);
        U[t * cap + z] = -du;
      }
      for (int u = 0; u < z; ++u) U[z * cap + u] = -(delta * bu[u]);
      U[z * cap + z] = delta;
    }
    /* eq. aca_approx_T_sub on every sweep-start row */
#ifdef _OPENMP
#pragma omp parallel for num_threads(s->nthreads) schedule(static)
#endif
    for (int64_t a = 0; a < rows; ++a) {
      double *Ta = s->T[b] + a * cap;
      double sv = chain(Ta, 1, cz, 1, z) - sb_entry(s, b, a, cs);
      double w = delta * sv;
      for (int t = 0; t < z; ++t) Ta[t] = fma(w, Tp[t], Ta[t]);
      Ta[z] = -w;
    }
    /* R gets the pivot row A(a*, :) on the sweep-start columns */
    for (int64_t c = 0; c < cols; ++c)
      s->R[b][(int64_t)z * s->cols_cap[b] + c] = sb_entry(s, b, as, c);
    s->prow[b][z] = (int32_t)as;
    s->pcol[b][z] = (int32_t)cs;
  }
  for (int b = 0; b < d - 1; ++b)
    if (add[b]) s->r[b] += 1;
  /* (2) superblock extensions */
  for (int b = 0; b < d - 1; ++b) {
    if (b > 0 && add[b - 1]) {
      /* new prefix alpha = I[b-1][r_old]: n_b new rows, T by Alg. 4 */
      int64_t p = r_old[b - 1];
#ifdef _OPENMP
#pragma omp parallel for num_threads(s->nthreads) schedule(static)
#endif
      for (int64_t i = 0; i < s->n[b]; ++i) replay_row(s, b, p * s->n[b] + i, s->r[b]);
    }
    if (b < d - 2 && add[b + 1]) {
      /* new suffix beta = J[b+1][r_old]: n_{b+1} new columns of R */
      int64_t q = r_old[b + 1];
      for (int t = 0; t < s->r[b]; ++t)
        for (int64_t j = 0; j < s->n[b + 1]; ++j) {
          int64_t c = q * s->n[b + 1] + j;
          s->R[b][(int64_t)t * s->cols_cap[b] + c] = sb_entry(s, b, s->prow[b][t], c);
        }
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* TT cores from the pivots: eq. ttcross_build / corereshape.               */
int64_t orc_core_size(const orc_state *s, int m) {
  int d = s->d;
  int64_t sl = m == 0 ? 1 : s->r[m - 1];
  int64_t sr = m == d - 1 ? 1 : s->r[m];
  return sl * s->n[m] * sr;
}

void orc_core(const orc_state *s, int m, double *out) {
  int d = s->d;
  if (m < d - 1) {
    /* G_k = reshape(T_k, [s_{k-1}, n_k, s_k]); row a = p*n + i */
    int64_t rows = rows_of(s, m), cap = s->maxr[m];
    for (int64_t a = 0; a < rows; ++a)
      for (int t = 0; t < s->r[m]; ++t) out[a * s->r[m] + t] = s->T[m][a * cap + t];
  } else {
    /* G_d = reshape(X(I_{<=d-1}, :), [s_{d-1}, n_d, 1]) = rows of R_{d-1} */
    int b = d - 2;
    for (int t = 0; t < s->r[b]; ++t)
      for (int64_t j = 0; j < s->n[d - 1]; ++j)
        out[t * s->n[d - 1] + j] = s->R[b][t * s->cols_cap[b] + j];
  }
}

/* X~(i) = G_1(i_1) G_2(i_2) ... G_d(i_d), Sec. 2.2, left to right. */
double orc_tt_eval(const orc_state *s, const int32_t *idx) {
  int d = s->d;
  double v[1024], w[1024];
  int r0 = s->r[0];
  const double *T0 = s->T[0];
  int64_t cap0 = s->maxr[0];
  for (int t = 0; t < r0; ++t) v[t] = T0[(int64_t)idx[0] * cap0 + t];
  int rl = r0;
  for (int m = 1; m < d; ++m) {
    if (m < d - 1) {
      /* core m: rows (p, i_m) of T_m, p over I[m-1] of size rl */
      int rr = s->r[m];
      int64_t cap = s->maxr[m];
      for (int u = 0; u < rr; ++u)
        w[u] = chain(v, 1, s->T[m] + ((int64_t)idx[m]) * cap + u, s->n[m] * cap, rl);
      for (int u = 0; u < rr; ++u) v[u] = w[u];
      rl = rr;
    } else {
      int b = d - 2;
      double x = chain(v, 1, s->R[b] + idx[m], s->cols_cap[b], rl);
      return x;
    }
  }
  return v[0];
}

/* ------------------------------------------------------------------------- */
/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) in counter form: output k of
   the generator seeded with `seed` is mix(seed + (k+1) * golden gamma).     */
static uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* multi-index of sample k: SplitMix64 draws (sample-major, mode-minor),
   index = floor(x * n / 2^64); or entry k in column-major order. */
static void sample_at(const orc_state *s, int64_t k, int exhaustive, uint64_t seed,
                      int32_t *idx) {
  if (exhaustive) {
    int64_t l = k;
    for (int m = 0; m < s->d; ++m) { idx[m] = (int32_t)(l % s->n[m]); l /= s->n[m]; }
  } else {
    for (int m = 0; m < s->d; ++m) {
      uint64_t x = splitmix64_at(seed, (uint64_t)(k * s->d + m));
      unsigned __int128 pr = (unsigned __int128)x * (uint64_t)s->n[m];
      idx[m] = (int32_t)(uint64_t)(pr >> 64);
    }
  }
}

int orc_sample_indices(int d, const int64_t *n, int64_t nsamples,
                       uint64_t seed, int32_t *out) {
  for (int64_t sidx = 0; sidx < nsamples; ++sidx)
    for (int m = 0; m < d; ++m) {
      uint64_t x = splitmix64_at(seed, (uint64_t)(sidx * d + m));
      unsigned __int128 pr = (unsigned __int128)x * (uint64_t)n[m];
      out[sidx * d + m] = (int32_t)(uint64_t)(pr >> 64);
    }
  return ORC_OK;
}

/* Sec. 5: ||X - X~||^2_{F,R} = sum_R (X - X~)^2 / sum_R X^2; we return its
   square root (the relative Frobenius error of eq. FrobeniusNorm).        */
int orc_sampled_error(const orc_state *s, int64_t nsamples, uint64_t seed,
                      double *err) {
  int d = s->d;
  int64_t total = 1;
  int exhaustive = 0;
  for (int m = 0; m < d; ++m) {
    if (total > INT64_MAX / s->n[m]) { total = INT64_MAX; break; }
    total *= s->n[m];
  }
  if (nsamples <= 0 || nsamples >= total) { exhaustive = 1; nsamples = total; }
  double *xs = (double *)malloc(sizeof(double) * nsamples);
  double *ys = (double *)malloc(sizeof(double) * nsamples);
  if (!xs || !ys) { free(xs); free(ys); return ORC_ERR_OOM; }
#ifdef _OPENMP
#pragma omp parallel for num_threads(s->nthreads) schedule(static)
#endif
  for (int64_t k = 0; k < nsamples; ++k) {
    int32_t idx[ORC_MAXD];
    sample_at(s, k, exhaustive, seed, idx);
    xs[k] = orc_entry(s, idx);
    ys[k] = orc_tt_eval(s, idx);
  }
  double num = 0.0, den = 0.0;
  for (int64_t k = 0; k < nsamples; ++k) {
    double df = xs[k] - ys[k];
    num += df * df;
    den += xs[k] * xs[k];
  }
  free(xs);
  free(ys);
  *err = sqrt(num / den);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* X over the error's sample set (Sec. 5 sampling): its root mean square, and
   the start pivot = argmax |X| over the samples and the origin, i.e. Alg. 1
   line 1 with the current approximation zero (ties: lowest linear index). */
int orc_sample_scan(const orc_state *s, int64_t nsamples, uint64_t seed,
                    double *rms, int32_t *start) {
  int d = s->d;
  int64_t total = 1;
  int exhaustive = 0;
  for (int m = 0; m < d; ++m) {
    if (total > INT64_MAX / s->n[m]) { total = INT64_MAX; break; }
    total *= s->n[m];
  }
  if (nsamples <= 0 || nsamples >= total) { exhaustive = 1; nsamples = total; }
  double *xs = (double *)malloc(sizeof(double) * nsamples);
  if (!xs) return ORC_ERR_OOM;
#ifdef _OPENMP
#pragma omp parallel for num_threads(s->nthreads) schedule(static)
#endif
  for (int64_t k = 0; k < nsamples; ++k) {
    int32_t idx[ORC_MAXD];
    sample_at(s, k, exhaustive, seed, idx);
    xs[k] = orc_entry(s, idx);
  }
  double den = 0.0;
  for (int64_t k = 0; k < nsamples; ++k) den += xs[k] * xs[k];
  *rms = sqrt(den / (double)nsamples);
  int32_t zero[ORC_MAXD] = {0};
  double bv = fabs(orc_entry(s, zero));
  int64_t bl = 0;
  memcpy(start, zero, sizeof(int32_t) * d);
  for (int64_t k = 0; k < nsamples; ++k) {
    double v = fabs(xs[k]);
    if (!(v >= bv)) continue;
    int32_t idx[ORC_MAXD];
    sample_at(s, k, exhaustive, seed, idx);
    int64_t l = lin_index(s, idx);
    if (v > bv || l < bl) { bv = v; bl = l; memcpy(start, idx, sizeof(int32_t) * d); }
  }
  free(xs);
  return ORC_OK;
}

int orc_sample_rms(const orc_state *s, int64_t nsamples, uint64_t seed,
                   double *rms) {
  int32_t start[ORC_MAXD];
  return orc_sample_scan(s, nsamples, seed, rms, start);
}

/* ------------------------------------------------------------------------- */
/* The adaptive loop.  The paper prescribes ranks (Sec. 5); for an accuracy
   target eps we add a pivot on bond b while its best residual exceeds
   tau * rms(X) (rms over the error's sample set) and the rank cap allows.
   When no bond adds, the sampled error verifies the result; if it is above
   eps, tau is divided by 10 and the sweeps continue from the same state.  */
int orc_run(orc_state *s, double eps, int64_t nsamples, uint64_t seed,
            int max_refine, orc_stats *st) {
  int d = s->d;
  memset(st, 0, sizeof(*st));
  double xrms = 0.0;
  int32_t start[ORC_MAXD];
  int rc = orc_sample_scan(s, nsamples, seed, &xrms, start);
  if (rc) { st->status = rc; return rc; }
  if (!isfinite(xrms)) { st->status = ORC_ERR_NONFINITE; return ORC_ERR_NONFINITE; }
  rc = orc_init_at(s, start);
  if (rc) { st->status = rc; return rc; }
  double tau = eps;
  double best[ORC_MAXD], maxabs[ORC_MAXD];
  int64_t lin[ORC_MAXD];
  int32_t row[ORC_MAXD], col[ORC_MAXD], add[ORC_MAXD];
  for (;;) {
    rc = orc_screen(s, best, lin, row, col, maxabs);
    st->sweeps += 1;
    st->entries_screened += s->last_screened;
    if (rc) { st->status = rc; return rc; }
    double theta = tau * xrms;
    int nadd = 0;
    for (int b = 0; b < d - 1; ++b) {
      add[b] = best[b] > theta && best[b] > 0.0 && s->r[b] < s->maxr[b];
      /* the pivot step divides by A(a*,c*) - chain(T(a*,:), R(:,c*)) (Sec.
         3.1.1); where that residual, formed afresh, is zero (or so small that
         its reciprocal overflows) the screened value was rounding noise and
         the bond takes no pivot in this sweep */
      if (add[b]) {
        double piv = orc_residual(s, b, row[b], col[b]);
        if (isfinite(piv) && !isfinite(1.0 / piv)) add[b] = 0;
      }
      nadd += add[b];
    }
    if (nadd) {
      rc = orc_apply(s, add, row, col);
      if (rc) { st->status = rc; return rc; }
      continue;
    }
    double err = 0.0;
    rc = orc_sampled_error(s, nsamples, seed, &err);
    if (rc) { st->status = rc; return rc; }
    st->err = err;
    if (eps == 0.0 || err <= eps) { rc = ORC_OK; break; }
    int capped = 1;
    for (int b = 0; b < d - 1; ++b) if (s->r[b] < s->maxr[b]) capped = 0;
    if (capped || st->refinements >= max_refine) { rc = ORC_NOT_CONVERGED; break; }
    tau /= 10.0;
    st->refinements += 1;
  }
  st->tau = tau;
  st->x_rms = xrms;
  st->status = rc;
  return rc;
}

/* ------------------------------------------------------------------------- */
void orc_ranks(const orc_state *s, int32_t *r) {
  for (int b = 0; b < s->d - 1; ++b) r[b] = s->r[b];
}
void orc_dims(const orc_state *s, int b, int64_t *rows, int64_t *cols) {
  *rows = rows_of(s, b);
  *cols = cols_of(s, b);
}
void orc_pivots(const orc_state *s, int b, int32_t *I, int32_t *J) {
  memcpy(I, s->I[b], sizeof(int32_t) * s->r[b] * (b + 1));
  memcpy(J, s->J[b], sizeof(int32_t) * s->r[b] * (s->d - 1 - b));
}
void orc_pivot_coords(const orc_state *s, int b, int32_t *prow, int32_t *pcol) {
  memcpy(prow, s->prow[b], sizeof(int32_t) * s->r[b]);
  memcpy(pcol, s->pcol[b], sizeof(int32_t) * s->r[b]);
}
void orc_T(const orc_state *s, int b, double *out) {
  int64_t rows = rows_of(s, b), cap = s->maxr[b];
  for (int64_t a = 0; a < rows; ++a)
    for (int t = 0; t < s->r[b]; ++t) out[a * s->r[b] + t] = s->T[b][a * cap + t];
}
void orc_R(const orc_state *s, int b, double *out) {
  int64_t cols = cols_of(s, b);
  for (int t = 0; t < s->r[b]; ++t)
    for (int64_t c = 0; c < cols; ++c) out[t * cols + c] = s->R[b][t * s->cols_cap[b] + c];
}
void orc_U(const orc_state *s, int b, double *out) {
  int64_t cap = s->maxr[b];
  for (int t = 0; t < s->r[b]; ++t)
    for (int u = 0; u < s->r[b]; ++u) out[t * s->r[b] + u] = s->U[b][t * cap + u];
}
void orc_E(const orc_state *s, int b, double *out) {
  int64_t rows = s->st_rows[b], cols = s->st_cols[b];
  for (int64_t a = 0; a < rows; ++a)
    for (int64_t c = 0; c < cols; ++c)
      out[a * cols + c] = s->stored ? s->E[b][a * s->cols_cap[b] + c] : NAN;
}
void orc_stored_extent(const orc_state *s, int b, int64_t *rows, int64_t *cols) {
  *rows = s->stored ? s->st_rows[b] : 0;
  *cols = s->stored ? s->st_cols[b] : 0;
}
