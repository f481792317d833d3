/*
 * ttc_oracle.h -- CPU FP64 oracle for the adaptive TT cross (arXiv 2407.11290).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow reference that the GPU
 * library is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product library never
 * links or calls it, and it shares no code, header or table with it.
 *
 * What it computes (paper references are to sections / equations / algorithms):
 *   - the tensor X is given entry-wise by a function (Sec. 5 intro): Hilbert
 *     tensor (eq. HilbertTensor, 0-based: 1/(1+i_1+...+i_d)), a TT of given
 *     cores, or a Maxwellian f(x,v);
 *   - the greedy pivot search of Alg. 1 on the superblock of Alg. 2, with the
 *     sample set L taken as the whole superblock (exhaustive residual screen)
 *     or as random entries followed by the row / column refinement of Alg. 1
 *     (orc_set_sampled);
 *   - all bonds searched simultaneously (Jacobi sweep, Sec. 2.3 / 3.2.3),
 *     pivots appended with nestedness (eq. nestedpivots);
 *   - the cross factor T = C U updated by eq. aca_approx_T / aca_approx_T_sub,
 *     rows entering a superblock rebuilt by Alg. 4 (replay of the pivot
 *     history), the pivot inverse U = P^{-1} bordered by the Sherman-Morrison
 *     step of Sec. 3.1.1;
 *   - TT cores by eq. ttcross_build / corereshape and the sampled relative
 *     error of Sec. 5.
 *
 * Arithmetic contract (IEEE binary64, round to nearest, no contraction):
 *   chain(x,y,K) := acc=+0; for t=0..K-1: acc=fma(x[t],y[t],acc)
 *   residual E(a,c) = A(a,c) - chain(T(a,:), R(:,c))
 *   pivot step z (row a*, col c*): cz[t]=R(t,c*), piv=A(a*,c*)-chain(T(a*,:),cz),
 *     delta=1/piv, Tp=T(a*,0..z-1) (snapshot);
 *     every row a: s=chain(T(a,:),cz)-A(a,c*); w=delta*s;
 *       T(a,t)=fma(w,Tp[t],T(a,t)) (t<z); T(a,z)=-w
 *   ties in |E| go to the lowest column-major linear index of the entry.
 *   stored-residual form: see orc_set_stored.
 */
#ifndef TTC_ORACLE_H
#define TTC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAXD 16

enum { ORC_GEN_HILBERT = 0, ORC_GEN_TT = 1, ORC_GEN_MAXWELLIAN = 2, ORC_GEN_MAXWELLIAN_XV = 3 };

enum {
  ORC_OK = 0,
  ORC_ERR_INVALID_ARG = 1,
  ORC_ERR_OOM = 2,
  ORC_ERR_ZERO_START = 3,
  ORC_ERR_NONFINITE = 4,
  ORC_NOT_CONVERGED = 7
};

typedef struct {
  int kind;
  /* ORC_GEN_TT: ranks rho[0..d] (rho[0]=rho[d]=1) and the cores concatenated,
     core m laid out [rho_m][n_m][rho_{m+1}] row-major.  Copied at create. */
  const int32_t *tt_ranks;
  const double *tt_cores;
  /* ORC_GEN_MAXWELLIAN: modes (x_0..x_{dx-1}, v_0..v_{dv-1}); x_m = 2*pi*i/n_m,
     v = vmin + (vmax-vmin)*i/(n-1).  rho = 1 + a_rho*prod sin x,
     u_j = a_u*cos x_{(j+1) mod dx}, T = 1 + a_T*cos(sum x),
     f = rho/(2*pi*T)^{dv/2} * exp(-|v-u|^2/(2T)).
     ORC_GEN_MAXWELLIAN_XV: the 2d2v / 3d3v distribution of Sec. 5.2 with
     dx = dv = d/2 and interleaved modes, amplitudes a_rho, a_T, shift a_u
     (see maxwellian_xv in ttc_oracle.c). */
  int32_t dx, dv;
  double a_rho, a_u, a_T, vmin, vmax;
} orc_gen;

typedef struct {
  int64_t sweeps;           /* residual screens performed */
  int64_t entries_screened; /* sum over screens of superblock sizes */
  int64_t refinements;      /* tau reductions */
  double tau;               /* final tau */
  double x_rms;             /* rms of X over the error's sample set */
  double err;               /* sampled relative Frobenius error (sqrt) */
  int32_t status;
} orc_stats;

typedef struct orc_state orc_state;

/* d modes of sizes n[0..d-1]; maxr[0..d-2] the rank cap of each bond;
   nthreads = OpenMP threads used by the screen (1 = serial). */
orc_state *orc_create(int d, const int64_t *n, const orc_gen *g,
                      const int32_t *maxr, int nthreads);
void orc_destroy(orc_state *s);

/* Exact entry X(idx) (idx has d 0-based indices). */
double orc_entry(const orc_state *s, const int32_t *idx);

/* First pivot `start` (d indices) for every bond, ranks 1. */
int orc_init_at(orc_state *s, const int32_t *start);
/* The same with start = (0,...,0). */
int orc_init(orc_state *s);

/* Exhaustive screen of every bond's superblock.  Outputs per bond b:
   best |E|, its linear index, its superblock row and column, and max |A|. */
int orc_screen(orc_state *s, double *best, int64_t *lin, int32_t *row,
               int32_t *col, double *maxabs);

/* Residual E(a,c) = A(a,c) - chain(T(a,:), R(:,c)) of superblock entry (a,c)
   of bond b, as the screen computes it. */
double orc_residual(const orc_state *s, int b, int64_t a, int64_t c);

/* Stored-residual form (eq. aca_approx_E, Sec. 3.1.1): on = 1 keeps every
   bond's residual E over its superblock and updates it by rank-one steps
   instead of recomputing A - T R.  Contract:
     - an entry entering a superblock (first screen, or rows / columns added
       by a neighbour's pivot) gets E = A - chain(T(a,:), R(:,c)) with the
       current T, R, as in the recompute form;
     - when bond b appends pivot (a*, c*), every entry of the sweep-start
       superblock becomes E(a,c) = fma(w_a, E(a*,c), E(a,c)) with
       w_a = -(E(a,c*) / E(a*,c*)) (row a* becomes exactly zero);
     - the screen is the argmax of the stored |E| (same tie rule); T, U, R
       and the cores are updated exactly as in the recompute form.
   Call after orc_create and before the first screen (orc_run re-initialises
   the stored extents).  Allocates rows_cap x cols_cap doubles per bond. */
int orc_set_stored(orc_state *s, int on);
/* Stored E(a,c) of bond b (NaN outside the stored extent or when off). */
double orc_stored_residual(const orc_state *s, int b, int64_t a, int64_t c);

/* Alg. 1 with a random sample set L (Sec. 2.3), recompute form only: nl > 0
   screens nl random entries of every superblock (drawn with replacement by
   SplitMix64(seed): sample j of bond b in screen t uses outputs 2k, 2k+1 with
   k = (t (d-1) + b) nl + j, a = floor(x rows / 2^64), c = floor(x' cols /
   2^64); t counts screens from the start), takes their argmax (tie rule as
   above), then refines it: the row moves to the argmax of its column, then
   the column to the argmax of its row, each only to a strictly larger |E|,
   until a round moves neither or max_rook rounds ran.  nl = 0 restores the
   exhaustive screen.  Ignored by the stored form. */
int orc_set_sampled(orc_state *s, int64_t nl, uint64_t seed, int max_rook);
/* entries the last screen evaluated; refinement steps that moved a pivot */
int64_t orc_last_screened(const orc_state *s);
int64_t orc_rook_moves(const orc_state *s);

/* Append pivot (row[b], col[b]) to every bond b with add[b] != 0 (row/col are
   superblock coordinates of the sweep-start superblock), update T, R, U and
   the history, then extend the neighbouring superblocks. */
int orc_apply(orc_state *s, const int32_t *add, const int32_t *row,
              const int32_t *col);

/* Whole adaptive run (start pivot from orc_sample_scan, sweeps, tau
   refinement, error).  A bond adds a
   pivot while its best |E| > tau * rms(X) (tau starts at eps, /10 per failed
   verification).  eps == 0 selects prescribed-rank mode (tau = 0, stop at the
   rank caps). */
int orc_run(orc_state *s, double eps, int64_t nsamples, uint64_t seed,
            int max_refine, orc_stats *st);

/* Sampled relative error sqrt(sum (X-Xt)^2 / sum X^2) over nsamples indices
   drawn by SplitMix64(seed) (all entries when nsamples <= 0 or >= prod n). */
int orc_sampled_error(const orc_state *s, int64_t nsamples, uint64_t seed,
                      double *err);
/* rms of X over the error's sample set (scales the pivot threshold) and the
   start pivot: argmax |X| over the samples and the origin, ties to the
   lowest linear index (Alg. 1 line 1 with a zero approximation). */
int orc_sample_scan(const orc_state *s, int64_t nsamples, uint64_t seed,
                    double *rms, int32_t *start);
/* rms only. */
int orc_sample_rms(const orc_state *s, int64_t nsamples, uint64_t seed,
                   double *rms);
/* The same indices the error uses: out[nsamples*d] sample-major. */
int orc_sample_indices(int d, const int64_t *n, int64_t nsamples,
                       uint64_t seed, int32_t *out);

/* Evaluate the current TT (cores) at idx. */
double orc_tt_eval(const orc_state *s, const int32_t *idx);

/* --- state export (all copies into caller buffers) --- */
void orc_ranks(const orc_state *s, int32_t *r /* d-1 */);
/* superblock dims of bond b */
void orc_dims(const orc_state *s, int b, int64_t *rows, int64_t *cols);
/* I_{<=b} full indices [r][b+1], J_{>b} full indices [r][d-1-b] */
void orc_pivots(const orc_state *s, int b, int32_t *I, int32_t *J);
/* pivot superblock coordinates in insertion order (row, col) [r] */
void orc_pivot_coords(const orc_state *s, int b, int32_t *prow, int32_t *pcol);
/* T_b [rows][r] row-major; R_b [r][cols]; U_b [r][r] */
void orc_T(const orc_state *s, int b, double *out);
void orc_R(const orc_state *s, int b, double *out);
void orc_U(const orc_state *s, int b, double *out);
/* stored form: E_b over its stored extent [st_rows][st_cols] (the superblock
   of the last screen), row-major */
void orc_E(const orc_state *s, int b, double *out);
void orc_stored_extent(const orc_state *s, int b, int64_t *rows, int64_t *cols);
/* core m as [s_{m-1}][n_m][s_m] row-major */
void orc_core(const orc_state *s, int m, double *out);
int64_t orc_core_size(const orc_state *s, int m);

#ifdef __cplusplus
}
#endif
#endif
