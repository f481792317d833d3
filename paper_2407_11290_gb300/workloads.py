"""Seeded synthetic workloads (inputs only -- no step of the method lives here).

Both the GPU library's tests/benchmark and the CPU oracle take their inputs
from this module, so it holds nothing but the descriptions of the tensors and
the recipes that draw random parameters.  The tensors are analytic functions
of their indices (Sec. 5 of the paper): nothing is read from disk.

Workloads:
  * ``hilbert``: X(i) = 1/(1 + i_1 + ... + i_d), 0-based (eq. HilbertTensor).
  * ``maxwellian``: f(x,v) = rho(x) (2 pi T(x))^{-dv/2} exp(-|v-u(x)|^2/(2T(x)))
    on x in [0, 2 pi)^dx (periodic grid, endpoint excluded) and
    v in [vmin, vmax]^dv (endpoints included), modes ordered (x..., v...),
    rho = 1 + a_rho prod sin x, u_j = a_u cos x_{(j+1) mod dx},
    T = 1 + a_T cos(sum x).
  * ``maxwellian_xv``: the 2d2v / 3d3v distributions of Sec. 5.2,
    f = sum_q rho(s_q) / (2 sqrt(2 pi T(s_q)))
        * (exp(-sum_q (v_q - 0.75)^2 / (2 T(s_q))) + exp(-sum_q (v_q + 0.75)^2 / (2 T(s_q)))),
    rho = 1 + 0.875 sin(2 pi s), T = 0.5 + 0.4 sin(2 pi s), positions on
    [-1/2, 1/2], velocities on [-3, 3] (end points included), modes
    interleaved (x, v_x, y, v_y[, z, v_z]).
  * ``tt``: a tensor given by TT cores with Gaussian entries (known ranks).
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 20240715
MASK64 = (1 << 64) - 1


def splitmix64(seed: int, k: int) -> int:
    """Output k of SplitMix64 seeded with ``seed`` (counter form)."""
    z = (seed + (k + 1) * 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def uniform01(seed: int, k: int) -> float:
    """53-bit uniform double in [0, 1) from output k."""
    return (splitmix64(seed, k) >> 11) * (1.0 / (1 << 53))


def hilbert(d: int, n: int):
    return dict(n=[int(n)] * d, gen={"kind": "hilbert"})


def maxwellian(dx: int, dv: int, n, a_rho=0.5, a_u=0.3, a_T=0.2, vmin=-8.0, vmax=8.0):
    ns = [int(n)] * (dx + dv) if np.isscalar(n) else [int(v) for v in n]
    return dict(n=ns, gen={"kind": "maxwellian", "dx": dx, "dv": dv, "a_rho": float(a_rho),
                           "a_u": float(a_u), "a_T": float(a_T), "vmin": float(vmin),
                           "vmax": float(vmax)})


def maxwellian_xv(D: int, n_pos: int, n_vel: int, a_rho=0.875, a_T=0.4, a_u=0.75, vmin=-3.0,
                  vmax=3.0):
    """The 2d2v (D = 2) / 3d3v (D = 3) distribution of Sec. 5.2 with modes
    interleaved (x, v_x, y, v_y[, z, v_z]) and sizes (n_pos, n_vel, ...)."""
    return dict(n=[int(n_pos), int(n_vel)] * D,
                gen={"kind": "maxwellian_xv", "dx": D, "dv": D, "a_rho": float(a_rho),
                     "a_u": float(a_u), "a_T": float(a_T), "vmin": float(vmin),
                     "vmax": float(vmax)})


def random_tt(n, ranks, seed: int = 1, positive_first: bool = True):
    """TT with Gaussian cores of the given ranks (rho_0 = rho_d = 1).

    With ``positive_first`` the entry X(0,...,0) is made strictly positive so
    the cross can start at the origin."""
    rng = np.random.default_rng(seed)
    d = len(n)
    cores = [rng.standard_normal((ranks[m], n[m], ranks[m + 1])) for m in range(d)]
    if positive_first:
        for m in range(d):
            cores[m][:, 0, :] = np.abs(cores[m][:, 0, :]) + 0.5
    return dict(n=[int(v) for v in n], gen={"kind": "tt", "ranks": [int(r) for r in ranks],
                                            "cores": cores})


def separable(n, seed: int = 2):
    """Rank-1 tensor prod_m f_m(i_m) with f_m in [0.5, 1.5]."""
    rng = np.random.default_rng(seed)
    d = len(n)
    cores = [(0.5 + rng.random((1, n[m], 1))) for m in range(d)]
    return dict(n=[int(v) for v in n], gen={"kind": "tt", "ranks": [1] * (d + 1), "cores": cores})


# The five configurations the benchmark and the parity tests use.
CONFIGS = {
    "hilbert3d_n32": dict(**hilbert(3, 32), eps=1e-10, max_rank=64, grid=[1, 1, 1],
                          nsamples=0, precision="fp64"),
    "hilbert6d_n64": dict(**hilbert(6, 64), eps=1e-8, max_rank=64, grid=[2] * 6,
                          nsamples=10**6, precision="fp64"),
    "maxwellian6d_n64": dict(**maxwellian(3, 3, 64), eps=1e-6, max_rank=256,
                             grid=[4, 4, 4, 1, 1, 1], nsamples=10**6, precision="fp32"),
    "hilbert6d_n256": dict(**hilbert(6, 256), eps=1e-10, max_rank=128, grid=[4] * 6,
                           nsamples=10**6, precision="split"),
}


# The paper's own workloads (Sec. 5.1 and 5.2, Table 4), prescribed ranks
# (eps = 0: every bond grows to its rank), the subtensor grids of its 64-rank
# strong-scaling partitions (Tables 2 and 3).
PAPER_WORKLOADS = {
    "paper_hilbert3d_n2000": dict(**hilbert(3, 2000), eps=0.0, bond_ranks=[25, 25],
                                  grid=[4, 4, 4], nsamples=10**6, paper_pivot_s=99.99),
    "paper_hilbert6d_n300": dict(**hilbert(6, 300), eps=0.0, bond_ranks=[15, 17, 18, 17, 15],
                                 grid=[1, 2, 4, 4, 2, 1], nsamples=10**6, paper_pivot_s=260.72),
    "paper_2d2v_n1000": dict(**maxwellian_xv(2, 2000, 1000), eps=0.0, bond_ranks=[10, 5, 20],
                             grid=[1, 8, 8, 1], nsamples=10**6, paper_pivot_s=147.34),
    "paper_3d3v_n400": dict(**maxwellian_xv(3, 800, 400), eps=0.0,
                            bond_ranks=[10, 5, 30, 5, 20], grid=[1, 2, 4, 4, 2, 1],
                            nsamples=10**6, paper_pivot_s=184.16),
}


def maxwellian_batch(count: int = 256, seed: int = 3):
    """Batch of independent Maxwellians: d ~ U{4,5,6} (2x+2v, 2x+3v, 3x+3v),
    n ~ U{32,48,64,96,128} (same n on every mode of an instance),
    a_rho, a_u, a_T ~ U(0, 0.5), all drawn from one SplitMix64 stream."""
    layouts = {4: (2, 2), 5: (2, 3), 6: (3, 3)}
    sizes = [32, 48, 64, 96, 128]
    out = []
    k = 0
    for _ in range(count):
        d = 4 + (splitmix64(seed, k) % 3); k += 1
        n = sizes[splitmix64(seed, k) % 5]; k += 1
        a_rho = 0.5 * uniform01(seed, k); k += 1
        a_u = 0.5 * uniform01(seed, k); k += 1
        a_T = 0.5 * uniform01(seed, k); k += 1
        dx, dv = layouts[d]
        out.append(maxwellian(dx, dv, n, a_rho=a_rho, a_u=a_u, a_T=a_T))
    return out
