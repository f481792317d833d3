// ttc_gen.cuh -- tensor entries X(i) evaluated on the device (Sec. 5: the
// tensor is a function of its indices and is never formed).
#pragma once
#include "ttc_internal.cuh"

namespace ttc {

// TT given by cores: left-to-right product of the slices, each dot product a
// serial FMA chain (ranks <= TT_GEN_RMAX; the vectors live in local memory).
__device__ __noinline__ double gen_tt(const InstDev &in, const int32_t *idx) {
  double v[TT_GEN_RMAX], w[TT_GEN_RMAX];
  const int d = in.d;
  int rl = in.rho[1];
  const double *G0 = in.tt + in.core_off[0];
  for (int t = 0; t < rl; ++t) v[t] = G0[(int64_t)idx[0] * rl + t];
  for (int m = 1; m < d; ++m) {
    const int ra = in.rho[m], rb = in.rho[m + 1];
    const double *G = in.tt + in.core_off[m];
    for (int q = 0; q < rb; ++q) {
      double acc = 0.0;
      const double *g = G + (int64_t)idx[m] * rb + q;
      const int64_t sg = in.n[m] * rb;
      for (int t = 0; t < ra; ++t) acc = __fma_rn(v[t], g[t * sg], acc);
      w[q] = acc;
    }
    for (int q = 0; q < rb; ++q) v[q] = w[q];
  }
  return v[0];
}

// Maxwellian f(x,v) = rho(x) (2 pi T(x))^{-dv/2} exp(-|v - u(x)|^2 / (2 T(x)))
// from the create-time tables (rho (2 pi T)^{-dv/2} and -1 / (2 T) per
// combination of the x indices, cos x_m per x mode): one exp per entry.
__device__ __forceinline__ double gen_maxwellian_tab(const InstDev &in, const int32_t *idx) {
  int64_t combo = 0;
  for (int m = 0; m < in.dx; ++m) combo += (int64_t)idx[m] * in.mx_stride[m];
  double q = 0.0;
  for (int j = 0; j < in.dv; ++j) {
    const int m = in.dx + j;
    const int mu = (j + 1) % in.dx;
    const double v = __dadd_rn(in.vmin, __dmul_rn(__dsub_rn(in.vmax, in.vmin), (double)idx[m]) /
                                            (double)(in.n[m] - 1));
    const double u = __dmul_rn(in.a_u, in.mx_cos[in.mx_off[mu] + idx[mu]]);
    const double dvu = __dsub_rn(v, u);
    q = __fma_rn(dvu, dvu, q);
  }
  return __dmul_rn(in.mx_coef[combo], exp(__dmul_rn(q, in.mx_nh[combo])));
}

// The interleaved 2d2v / 3d3v distribution of Sec. 5.2 (eq. 2d2vFunction)
// from the create-time tables: per position mode rho / (2 sqrt(2 pi T)) and
// 1 / (2 T), per velocity mode the grid value; two exps per entry.
__device__ __forceinline__ double gen_maxwellian_xv(const InstDev &in, const int32_t *idx) {
  double rs = 0.0, bm = 0.0, bp = 0.0;
  for (int q = 0; q < in.dx; ++q) {
    const int64_t ox = in.mx_off[2 * q] + idx[2 * q];
    const double c = in.mx_coef[ox], h = in.mx_nh[ox];
    const double v = in.mx_coef[in.mx_off[2 * q + 1] + idx[2 * q + 1]];
    const double dm = __dsub_rn(v, in.a_u), dp = __dadd_rn(v, in.a_u);
    rs = __dadd_rn(rs, c);
    bm = __dadd_rn(bm, __dmul_rn(__dmul_rn(dm, dm), h));
    bp = __dadd_rn(bp, __dmul_rn(__dmul_rn(dp, dp), h));
  }
  return __dmul_rn(rs, __dadd_rn(exp(-bm), exp(-bp)));
}

// table entry k of mode m of the interleaved distribution
__device__ void maxwellian_xv_table_entry(const InstDev &in, int m, int64_t i, double *a,
                                          double *b) {
  const double two_pi = 6.283185307179586476925286766559;
  const double t = (double)i / (double)(in.n[m] - 1);
  if ((m & 1) == 0) {
    const double sv = __dadd_rn(-0.5, t);
    const double sn = sin(__dmul_rn(two_pi, sv));
    const double rho = __dadd_rn(1.0, __dmul_rn(in.a_rho, sn));
    const double T = __dadd_rn(0.5, __dmul_rn(in.a_T, sn));
    *a = rho / __dmul_rn(2.0, sqrt(__dmul_rn(two_pi, T)));
    *b = 1.0 / __dmul_rn(2.0, T);
  } else {
    *a = __dadd_rn(in.vmin, __dmul_rn(__dsub_rn(in.vmax, in.vmin), (double)i) /
                                (double)(in.n[m] - 1));
    *b = 0.0;
  }
}

// one entry of the tables: x-index combination `combo` (column-major)
__device__ void maxwellian_table_entry(const InstDev &in, int64_t combo, double *coef,
                                       double *nh) {
  const double two_pi = 6.283185307179586476925286766559;
  double prod_sin = 1.0, sum_x = 0.0;
  int64_t l = combo;
  for (int m = 0; m < in.dx; ++m) {
    const int64_t i = l % in.n[m];
    l /= in.n[m];
    const double x = __dmul_rn(two_pi, (double)i) / (double)in.n[m];
    prod_sin = __dmul_rn(prod_sin, sin(x));
    sum_x = __dadd_rn(sum_x, x);
  }
  const double rho = __dadd_rn(1.0, __dmul_rn(in.a_rho, prod_sin));
  const double T = __dadd_rn(1.0, __dmul_rn(in.a_T, cos(sum_x)));
  *coef = rho / pow(__dmul_rn(two_pi, T), 0.5 * (double)in.dv);
  *nh = -1.0 / __dmul_rn(2.0, T);
}

// TT cores or the Maxwellian: one out-of-line copy (each is long, and the
// callers are many)
__device__ __noinline__ double gen_other(const InstDev &in, const int32_t *idx) {
  if (in.gen == 1) return gen_tt(in, idx);
  if (in.gen == 3) return gen_maxwellian_xv(in, idx);
  return gen_maxwellian_tab(in, idx);
}

__device__ __forceinline__ double gen_full(const InstDev &in, const int32_t *idx) {
  if (in.gen == 0) {
    int s = 0;
    for (int m = 0; m < in.d; ++m) s += idx[m];
    return in.hilb[s];
  }
  return gen_other(in, idx);
}

// Entry (a, c) of the superblock of bond b: rows a = p*n_b + i (p indexes
// I_{<=k-1}), columns c = q*n_{b+1} + j (q indexes J_{>k+1}), Alg. 2.
__device__ __noinline__ double sb_entry(const InstDev &in, int b, int64_t a, int64_t c) {
  const int64_t nb0 = in.n[b], nb1 = in.n[b + 1];
  const int64_t p = a / nb0, i = a - p * nb0;
  const int64_t q = c / nb1, j = c - q * nb1;
  // outside every superblock this bond can have: no entry (NaN), no access
  if (a < 0 || c < 0 || (b > 0 && p >= in.bond[b - 1].cap) ||
      (b < in.nb - 1 && q >= in.bond[b + 1].cap))
    return __longlong_as_double(0x7FF8000000000000ll);
  if (in.gen == 4) return in.bond[b].A[a * in.bond[b].ldR + c];  // the caller's values
  const SetDev &L = left_set(in, b);
  const SetDev &Rs = right_set(in, b);
  if (in.gen == 0) return in.hilb[L.sum[p] + (int)i + (int)j + Rs.sum[q]];
  int32_t idx[TTC_MAXD];
  for (int m = 0; m < b; ++m) idx[m] = L.idx[p * b + m];
  idx[b] = (int32_t)i;
  idx[b + 1] = (int32_t)j;
  const int w = in.d - b - 2;
  for (int m = 0; m < w; ++m) idx[b + 2 + m] = Rs.idx[q * w + m];
  return gen_full(in, idx);
}

// Coordinate m of error sample k, the value sample_index gives, computed
// alone (no index array in local memory on the sample path).
__device__ __forceinline__ int32_t sample_coord(const InstDev &in, int64_t k, int m) {
  if (in.exhaustive) {
    int64_t l = k;
    for (int j = 0; j < m; ++j) l /= in.n[j];
    return (int32_t)(l % in.n[m]);
  }
  const uint64_t x = splitmix64_at(in.seed, (uint64_t)(k * in.d + m));
  return (int32_t)__umul64hi(x, (uint64_t)in.n[m]);
}

// Multi-index of error sample k (SplitMix64 counter form, sample-major,
// mode-minor; index = floor(x * n / 2^64)), or entry k in column-major
// order when the error runs over every entry.
__device__ __forceinline__ void sample_index(const InstDev &in, int64_t k, int32_t *idx) {
  if (in.exhaustive) {
    int64_t l = k;
    for (int m = 0; m < in.d; ++m) {
      idx[m] = (int32_t)(l % in.n[m]);
      l /= in.n[m];
    }
  } else {
    for (int m = 0; m < in.d; ++m) {
      const uint64_t x = splitmix64_at(in.seed, (uint64_t)(k * in.d + m));
      idx[m] = (int32_t)__umul64hi(x, (uint64_t)in.n[m]);
    }
  }
}

}  // namespace ttc
