"""Pins for the CPU oracle: checks against what the paper and the mathematics
fix, never against the oracle itself.  CPU only."""
import os

import numpy as np
import pytest

import oracle
from paper_2407_11290_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def full_from_cores(cores):
    """Contract TT cores [s_{m-1}, n_m, s_m] into the full tensor (numpy)."""
    X = cores[0]
    for G in cores[1:]:
        X = np.tensordot(X, G, axes=([-1], [0]))
    return X[0, ..., 0]


def full_tensor(n, gen):
    """The exact tensor, evaluated entry by entry by numpy expressions."""
    grids = np.meshgrid(*[np.arange(v) for v in n], indexing="ij")
    if gen["kind"] == "hilbert":
        return 1.0 / (1.0 + sum(grids))
    if gen["kind"] == "tt":
        return full_from_cores([np.asarray(c) for c in gen["cores"]])
    raise ValueError


def matrix_as_tt(A):
    """An n1 x n2 matrix as a d=2 TT that reproduces it exactly: G0 = I, G1 = A."""
    n1, n2 = A.shape
    G0 = np.eye(n1).reshape(1, n1, n1)
    G1 = A.reshape(n1, n2, 1)
    return {"kind": "tt", "ranks": [1, n1, 1], "cores": [G0, G1]}


# --------------------------------------------------------------------------
# Sampling generator: published SplitMix64 outputs (golden file).
def test_splitmix64_published_outputs():
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    # index = floor(x * n / 2^64) with n = 2^31 is x >> 33
    idx = oracle.sample_indices([2**31], len(vals), seed=0)[:, 0]
    assert [int(v) for v in idx] == [v >> 33 for v in vals]
    assert [W.splitmix64(0, k) for k in range(len(vals))] == vals


def test_sample_indices_in_range_and_uniform():
    n = [7, 64, 3]
    s = oracle.sample_indices(n, 60000, seed=5)
    assert s.min() == 0 and all(s[:, m].max() == n[m] - 1 for m in range(3))
    counts = np.bincount(s[:, 0], minlength=7)
    chi2 = ((counts - 60000 / 7) ** 2 / (60000 / 7)).sum()
    assert chi2 < 30  # 6 dof; p ~ 4e-5


# --------------------------------------------------------------------------
# d = 2: the cross with an exhaustive screen is Gaussian elimination with
# complete pivoting after the fixed first pivot (Sec. 2.3; eq. aca_approx_E).
def lu_complete_pivoting(A, steps):
    S = A.copy()
    n1, n2 = A.shape
    piv, vals = [(0, 0)], []
    S = S - np.outer(S[:, 0], S[0, :]) / S[0, 0]
    for _ in range(steps - 1):
        mag = np.abs(S)
        m = mag.max()
        cand = np.argwhere(mag == m)
        lin = cand[:, 0] + n1 * cand[:, 1]          # column-major linear index
        i, j = cand[np.argmin(lin)]
        vals.append(m)
        piv.append((int(i), int(j)))
        S = S - np.outer(S[:, j], S[i, :]) / S[i, j]
    return piv, vals


@pytest.mark.parametrize("shape,seed", [((8, 8), 0), ((13, 29), 1), ((40, 17), 2), ((1, 9), 3)])
def test_d2_matches_complete_pivoting_lu(shape, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal(shape)
    A[0, 0] = 2.0
    steps = min(shape)
    o = oracle.Oracle(list(shape), matrix_as_tt(A), steps)
    assert o.init() == 0
    got_vals = []
    for _ in range(steps - 1):
        rc, s = o.screen()
        assert rc == 0
        got_vals.append(s["best"][0])
        assert o.apply([1], s["row"], s["col"]) == 0
    I, J = o.pivots(0)
    piv, vals = lu_complete_pivoting(A, steps)
    assert [(int(a), int(b)) for a, b in zip(I[:, 0], J[:, 0])] == piv
    np.testing.assert_allclose(got_vals, vals, rtol=1e-10, atol=1e-13)


def test_tie_goes_to_lowest_column_major_index():
    # after the pivot (0,0) the residual has |E| = 1 at (2,1) and (1,3):
    # column-major lin 2+4*1=6 < 1+4*3=13, row-major would pick (1,3)
    A = np.zeros((4, 4))
    A[0, 0] = 1.0
    A[2, 1] = 1.0
    A[1, 3] = -1.0
    o = oracle.Oracle([4, 4], matrix_as_tt(A), 3)
    o.init()
    rc, s = o.screen()
    assert s["best"][0] == 1.0
    assert (s["row"][0], s["col"][0]) == (2, 1)
    assert s["lin"][0] == 6


# --------------------------------------------------------------------------
# Fig. 1 (Sec. 3.1.1): on the 100 x 100 Hilbert matrix the iterative formula
# reaches machine precision while C P^{-1} R degrades beyond rank ~12.
def test_fig1_iterative_vs_direct_hilbert_matrix():
    n = 100
    i = np.arange(n)
    H = 1.0 / (1 + i[:, None] + i[None, :])
    o = oracle.Oracle([n, n], {"kind": "hilbert"}, 24)
    o.init()
    err_it, err_dir = {}, {}
    for z in range(1, 23):
        T, R = o.T(0), o.R(0)
        err_it[z] = np.linalg.norm(H - T @ R) / np.linalg.norm(H)
        I, J = o.pivots(0)
        P = H[np.ix_(I[:, 0], J[:, 0])]
        try:  # the direct method forms the inverse of the cross section
            with np.errstate(all="ignore"):
                D = H[:, J[:, 0]] @ np.linalg.inv(P) @ H[I[:, 0], :]
            err_dir[z] = np.linalg.norm(H - D) / np.linalg.norm(H)
        except np.linalg.LinAlgError:
            err_dir[z] = np.inf
        rc, s = o.screen()
        o.apply([1], s["row"], s["col"])
    assert min(err_it.values()) < 1e-15
    assert err_it[20] < 1e-15
    assert err_dir[20] > 1e4 * err_it[20]
    # both agree while the pivot block is well conditioned
    assert abs(err_dir[8] - err_it[8]) < 1e-3 * err_it[8]


# --------------------------------------------------------------------------
def test_separable_rank1_is_exact():
    w = W.separable([7, 9, 5, 6])
    o = oracle.Oracle(w["n"], w["gen"], 8)
    rc, st = o.run(1e-12, nsamples=0)
    assert rc == 0
    assert list(o.ranks()) == [1, 1, 1]
    X = full_tensor(w["n"], w["gen"])
    Y = full_from_cores(o.cores())
    assert np.abs(X - Y).max() <= 1e-15 * np.abs(X).max()


def test_random_tt_known_ranks_recovered():
    w = W.random_tt([12, 12, 12, 12], [1, 3, 4, 3, 1], seed=7)
    o = oracle.Oracle(w["n"], w["gen"], 10)
    rc, st = o.run(1e-12, nsamples=0)
    assert rc == 0
    assert list(o.ranks()) == [3, 4, 3]
    X = full_tensor(w["n"], w["gen"])
    Y = full_from_cores(o.cores())
    assert np.linalg.norm(X - Y) / np.linalg.norm(X) <= 1e-12


def _interp_points(o, m):
    """Multi-indices (alpha in I_{<=m-1}, i_m, beta in J_{>m})."""
    d = o.d
    if m == 0:
        lefts = [()]
    else:
        I, _ = o.pivots(m - 1)
        lefts = [tuple(r) for r in I]
    if m == d - 1:
        rights = [()]
    else:
        _, J = o.pivots(m)
        rights = [tuple(r) for r in J]
    for a in lefts:
        for i in range(int(o.n[m])):
            for b in rights:
                yield a + (i,) + b


@pytest.mark.parametrize("case", ["hilbert", "tt"])
def test_interpolation_and_nestedness(case):
    if case == "hilbert":
        w = W.hilbert(4, 10)
        eps = 1e-9
    else:
        w = W.random_tt([6, 7, 8, 5], [1, 4, 6, 3, 1], seed=11)
        eps = 1e-3
    o = oracle.Oracle(w["n"], w["gen"], 6)
    rc, _ = o.run(eps, nsamples=0)
    assert rc in (0, oracle.NOT_CONVERGED)
    X = full_tensor(w["n"], w["gen"])
    Y = full_from_cores(o.cores())
    tol = 1e-13 * np.abs(X).max()
    # Sec. 3.2.1: the cross reproduces X exactly on (I_{<=k-1}, i_k, J_{>k})
    for m in range(o.d):
        for idx in _interp_points(o, m):
            assert abs(Y[idx] - X[idx]) <= tol, (m, idx)
    # eq. nestedpivots: I_{<=k} subset I_{<=k-1} x I_k, J_{>k} subset I_{k+1} x J_{>k+1}
    for b in range(o.d - 1):
        I, J = o.pivots(b)
        if b > 0:
            Ip, _ = o.pivots(b - 1)
            prev = {tuple(r) for r in Ip}
            assert all(tuple(r[:-1]) in prev for r in I)
        if b < o.d - 2:
            _, Jn = o.pivots(b + 1)
            nxt = {tuple(r) for r in Jn}
            assert all(tuple(r[1:]) in nxt for r in J)
        assert len({tuple(r) for r in I}) == len(I)
        assert len({tuple(r) for r in J}) == len(J)


def test_factor_identities():
    """T_k = C_k U_k with U_k = P_k^{-1} from the bordered Sherman-Morrison
    update (Sec. 3.1.1-3.1.3), and T_k R_k = C_k P_k^{-1} R_k."""
    w = W.hilbert(4, 9)
    o = oracle.Oracle(w["n"], w["gen"], 5)
    rc, _ = o.run(1e-6, nsamples=0)
    X = full_tensor(w["n"], w["gen"])
    for b in range(o.d - 1):
        rows, cols = o.dims(b)
        T, R, U = o.T(b), o.R(b), o.U(b)
        I, J = o.pivots(b)
        Il = o.pivots(b - 1)[0] if b > 0 else np.zeros((1, 0), np.int32)
        Jr = o.pivots(b + 1)[1] if b < o.d - 2 else np.zeros((1, 0), np.int32)
        n_b, n_b1 = int(o.n[b]), int(o.n[b + 1])
        # superblock rows (alpha, i_b) and the pivot columns (j, beta) of J_{>k}
        C = np.array([[X[tuple(Il[a // n_b]) + (a % n_b,) + tuple(Jrow)] for Jrow in J]
                      for a in range(rows)])
        P = np.array([[X[tuple(Irow) + tuple(Jrow)] for Jrow in J] for Irow in I])
        Rx = np.array([[X[tuple(Irow) + (c % n_b1,) + tuple(Jr[c // n_b1])] for c in range(cols)]
                       for Irow in I])
        np.testing.assert_array_equal(R, Rx)
        assert np.abs(U @ P - np.eye(len(I))).max() < 1e-9 * np.linalg.cond(P)
        # rounding of C U grows with |C||U| (U = P^{-1} is ill conditioned)
        np.testing.assert_allclose(T, C @ U, rtol=0, atol=1e-13 * (np.abs(C) @ np.abs(U)).max())
        direct = C @ np.linalg.solve(P, Rx)
        np.testing.assert_allclose(T @ R, direct, rtol=0, atol=1e-10 * np.abs(direct).max())


def test_tt_eval_and_sampled_error_against_numpy():
    w = W.hilbert(4, 11)
    o = oracle.Oracle(w["n"], w["gen"], 4)
    o.run(1e-4, nsamples=5000, seed=3)
    X = full_tensor(w["n"], w["gen"])
    Y = full_from_cores(o.cores())
    S = oracle.sample_indices(w["n"], 5000, seed=3)
    xs = X[tuple(S.T)]
    ys = Y[tuple(S.T)]
    ref = np.sqrt(((xs - ys) ** 2).sum() / (xs ** 2).sum())
    assert abs(o.sampled_error(5000, seed=3) - ref) <= 1e-14
    for idx in S[:50]:
        assert abs(o.tt_eval(idx) - Y[tuple(idx)]) <= 1e-15
    # exhaustive mode == full-tensor relative Frobenius error (eq. FrobeniusNorm)
    full = np.linalg.norm(X - Y) / np.linalg.norm(X)
    assert abs(o.sampled_error(0) - full) <= 1e-15


def test_config0_end_to_end_and_svd_bound():
    """3D Hilbert n=32, eps=1e-10: full-tensor error below eps; no TT with the
    cross's ranks can beat the tail of the unfoldings' singular values."""
    w = W.CONFIGS["hilbert3d_n32"]
    o = oracle.Oracle(w["n"], w["gen"], w["max_rank"])
    rc, st = o.run(w["eps"], nsamples=0)
    assert rc == 0
    X = full_tensor(w["n"], w["gen"])
    Y = full_from_cores(o.cores())
    err = np.linalg.norm(X - Y) / np.linalg.norm(X)
    assert err <= w["eps"]
    assert abs(err - st["err"]) <= 1e-15
    r = o.ranks()
    n = w["n"]
    for b in range(2):
        sv = np.linalg.svd(X.reshape(int(np.prod(n[:b + 1])), -1, order="F"), compute_uv=False)
        tail = np.sqrt((sv[r[b]:] ** 2).sum()) / np.linalg.norm(X)
        assert err >= tail * (1 - 1e-6)
        # TT-SVD (delta-truncation at eps/sqrt(d-1)) needs about as many
        delta = w["eps"] / np.sqrt(2)
        k = int(np.searchsorted(-np.sqrt(np.cumsum((sv ** 2)[::-1])[::-1] / (X ** 2).sum()), -delta))
        assert r[b] <= k + 6


def test_thread_split_does_not_change_pivots():
    """The global best pivot is the best of local bests (Sec. 3.2.1)."""
    w = W.hilbert(4, 12)
    piv = []
    for nt in (1, 3, 8):
        o = oracle.Oracle(w["n"], w["gen"], 8, nthreads=nt)
        o.run(1e-9, nsamples=2000)
        piv.append([o.pivot_coords(b) for b in range(3)])
    for other in piv[1:]:
        for (a, b), (c, d) in zip(piv[0], other):
            np.testing.assert_array_equal(a, c)
            np.testing.assert_array_equal(b, d)


def test_start_pivot_is_argmax_over_samples_and_origin():
    """Alg. 1 line 1 with a zero approximation: argmax |X| over the random
    samples (plus the origin), ties to the lowest column-major index."""
    w = W.maxwellian(2, 2, [6, 7, 16, 16])
    o = oracle.Oracle(w["n"], w["gen"], 4)
    rms, start = o.sample_scan(3000, seed=9)
    S = oracle.sample_indices(w["n"], 3000, seed=9)
    cand = np.vstack([np.zeros((1, 4), np.int32), S])
    vals = np.array([abs(o.entry(c)) for c in cand])
    best = cand[vals == vals.max()]
    lin = best[:, 0] + 6 * (best[:, 1] + 7 * (best[:, 2] + 16 * best[:, 3]))
    np.testing.assert_array_equal(start, best[np.argmin(lin)])
    assert abs(rms - np.sqrt((vals[1:] ** 2).mean())) <= 1e-15 * rms
    # the Hilbert tensor peaks at the origin, which is then the start
    h = oracle.Oracle([9, 9, 9], {"kind": "hilbert"}, 4)
    assert list(h.sample_scan(500, seed=1)[1]) == [0, 0, 0]


def test_zero_start_and_nonfinite():
    w = W.random_tt([4, 5, 6], [1, 2, 2, 1], seed=3)
    w["gen"]["cores"][0][:, 0, :] = 0.0
    o = oracle.Oracle(w["n"], w["gen"], 3)
    assert o.init() == oracle.ERR_ZERO_START
    w = W.random_tt([4, 5, 6], [1, 2, 2, 1], seed=3)
    w["gen"]["cores"][1][:, 3, :] = np.nan
    o = oracle.Oracle(w["n"], w["gen"], 3)
    rc, st = o.run(1e-6, nsamples=0)
    assert rc == oracle.ERR_NONFINITE


def test_table5_weak_range():
    """Table 5: one-process TT-ACA reaches 1.40e-6 on the n=250 Hilbert tensor
    with ranks (1,25,25,1); the exhaustive greedy search must be at least as
    accurate, within the 10x slack of a different search."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table5_hilbert3d.txt"))
            if l.strip() and not l.startswith("#")]
    ttaca_err = {int(r[0]): float(r[4]) for r in rows}
    w = W.hilbert(3, 250)
    o = oracle.Oracle(w["n"], w["gen"], 25, nthreads=os.cpu_count() or 1)
    rc, st = o.run(0.0, nsamples=10**5, seed=W.DEFAULT_SEED)
    assert rc == 0 and list(o.ranks()) == [25, 25]
    assert st["err"] <= 10 * ttaca_err[250]


def _spike_tt(n, a, delta):
    """Rank-2 TT on four modes: a smooth rank-1 term s(i) = 1 / (1 + i / 10)
    in every mode plus a * v(i1) v(i2) v(i3) v(i4), v = delta at index 0 and
    1 elsewhere.  Near the start pivot (the origin) the second term is
    scaled down by delta^2 or more, so the rank-1 screens see only a small
    trace of it while most entries carry all of it."""
    i = np.arange(n)
    s = 1.0 / (1.0 + 0.1 * i)
    v = np.where(i == 0, delta, 1.0)
    c1 = np.zeros((1, n, 2)); c1[0, :, 0] = s; c1[0, :, 1] = v
    mid = np.zeros((2, n, 2)); mid[0, :, 0] = s; mid[1, :, 1] = v
    c4 = np.zeros((2, n, 1)); c4[0, :, 0] = s; c4[1, :, 0] = a * v
    cores = [c1, mid, mid.copy(), c4]
    return dict(n=[n] * 4, gen={"kind": "tt", "ranks": [1, 2, 2, 2, 1], "cores": cores})


@pytest.mark.parametrize("a,delta", [(1e-4, 0.01), (1e-4, 0.03), (1e-3, 0.01)])
def test_tau_refinement_follows_the_stop_rule(a, delta):
    """The stop rule with tau refinement (a bond adds a pivot while its best
    |E| > tau rms(X); tau starts at eps and drops tenfold while the verified
    error is above eps), checked from numpy on the full tensor: the number
    of refinements is the smallest j with max |E| > eps 10^-j rms over the
    rank-1 superblocks at the start pivot; one refinement fewer leaves the
    rank-1 cross, NOT_CONVERGED, with the error of its interpolant."""
    eps, n = 1e-6, 10
    w = _spike_tt(n, a, delta)
    X = np.einsum("aib,bjc,ckd,dle->ijkl", *w["gen"]["cores"])
    p = np.unravel_index(int(np.argmax(np.abs(X.reshape(-1, order="F")))), X.shape, order="F")
    rms = np.sqrt(np.mean(X ** 2))
    M = 0.0
    for k in range(3):
        B = X[tuple(slice(None) if m in (k, k + 1) else p[m] for m in range(4))]
        E = B - np.outer(B[:, p[k + 1]], B[p[k], :]) / B[p[k], p[k + 1]]
        M = max(M, np.abs(E).max())
    j = 0
    while not M > eps * 10.0 ** (-j) * rms:
        j += 1
    assert 1 <= j <= 4
    o = oracle.Oracle(w["n"], w["gen"], 8)
    rc, st = o.run(eps, nsamples=0, max_refine=6)
    assert rc == 0 and st["refinements"] == j
    assert abs(st["tau"] - eps * 10.0 ** (-j)) <= 1e-12 * eps
    assert [int(r) for r in o.ranks()] == [2, 2, 2] and st["err"] <= 1e-10
    # one refinement fewer: the rank-1 cross through p
    o = oracle.Oracle(w["n"], w["gen"], 8)
    rc, st = o.run(eps, nsamples=0, max_refine=j - 1)
    assert rc == 7 and [int(r) for r in o.ranks()] == [1, 1, 1]
    i1, i2, i3, i4 = np.meshgrid(*[np.arange(n)] * 4, indexing="ij")
    Xt = (X[i1, p[1], p[2], p[3]] * X[p[0], i2, p[2], p[3]] * X[p[0], p[1], i3, p[3]] *
          X[p[0], p[1], p[2], i4]) / X[p] ** 3
    exact = np.linalg.norm(X - Xt) / np.linalg.norm(X)
    assert exact > eps and abs(st["err"] - exact) <= 1e-9 * exact


def test_maxwellian_moments():
    """Velocity moments of the Maxwellian (Sec. 5.2 family): on a wide v-grid
    the quadrature of f over v returns rho(x), rho u(x) and dv rho T(x)."""
    n = 48
    w = W.maxwellian(2, 2, [5, 6, n, n], a_rho=0.4, a_u=0.3, a_T=0.25, vmin=-9.0, vmax=9.0)
    o = oracle.Oracle(w["n"], w["gen"], 2)
    g = w["gen"]
    v = g["vmin"] + (g["vmax"] - g["vmin"]) * np.arange(n) / (n - 1)
    h = (g["vmax"] - g["vmin"]) / (n - 1)
    for ix in [(0, 0), (1, 2), (4, 5), (3, 1)]:
        x = [2 * np.pi * ix[0] / 5, 2 * np.pi * ix[1] / 6]
        F = np.array([[o.entry(ix + (a, b)) for b in range(n)] for a in range(n)])
        m0 = F.sum() * h * h
        rho = 1 + g["a_rho"] * np.sin(x[0]) * np.sin(x[1])
        T = 1 + g["a_T"] * np.cos(x[0] + x[1])
        u = [g["a_u"] * np.cos(x[1]), g["a_u"] * np.cos(x[0])]
        m1 = [(F * v[:, None]).sum() * h * h / m0, (F * v[None, :]).sum() * h * h / m0]
        m2 = ((F * ((v[:, None] - m1[0]) ** 2 + (v[None, :] - m1[1]) ** 2)).sum() * h * h
              / m0 / 2)
        assert abs(m0 - rho) < 1e-10
        assert abs(m1[0] - u[0]) < 1e-10 and abs(m1[1] - u[1]) < 1e-10
        assert abs(m2 - T) < 1e-9


def test_maxwellian_dx3_velocity_moments():
    """The 6D Maxwellian (d_x = 3, d_v = 3) of the single-tensor workload:
    rho = 1 + a_rho sin x1 sin x2 sin x3, u = a_u (cos x2, cos x3, cos x1),
    T = 1 + a_T cos(x1 + x2 + x3) on the periodic grid x = 2 pi i / n.  On a
    wide v-grid the quadrature over the three velocities returns rho, u and
    T (the uniform-grid sum of a Gaussian is exact far below 1e-10 at these
    spacings), and at x = 0 the distribution is the standard Gaussian up to
    the shift u = (a_u, a_u, a_u) and T = 1 + a_T."""
    nv = 32
    w = W.maxwellian(3, 3, [5, 6, 7, nv, nv, nv], a_rho=0.45, a_u=0.3, a_T=0.2,
                     vmin=-9.0, vmax=9.0)
    o = oracle.Oracle(w["n"], w["gen"], 2)
    g = w["gen"]
    v = g["vmin"] + (g["vmax"] - g["vmin"]) * np.arange(nv) / (nv - 1)
    h = (g["vmax"] - g["vmin"]) / (nv - 1)
    V = np.meshgrid(v, v, v, indexing="ij")
    for ix in [(0, 0, 0), (1, 2, 3), (4, 5, 6), (2, 1, 5)]:
        x = [2 * np.pi * ix[m] / w["n"][m] for m in range(3)]
        F = np.empty((nv, nv, nv))
        for a in range(nv):
            for b in range(nv):
                for c in range(nv):
                    F[a, b, c] = o.entry(ix + (a, b, c))
        rho = 1 + g["a_rho"] * np.sin(x[0]) * np.sin(x[1]) * np.sin(x[2])
        u = [g["a_u"] * np.cos(x[1]), g["a_u"] * np.cos(x[2]), g["a_u"] * np.cos(x[0])]
        T = 1 + g["a_T"] * np.cos(x[0] + x[1] + x[2])
        m0 = F.sum() * h ** 3
        m1 = [(F * V[j]).sum() * h ** 3 / m0 for j in range(3)]
        m2 = sum((F * (V[j] - m1[j]) ** 2).sum() for j in range(3)) * h ** 3 / m0 / 3
        assert abs(m0 - rho) < 1e-10
        assert max(abs(m1[j] - u[j]) for j in range(3)) < 1e-10
        assert abs(m2 - T) < 1e-9
        if ix == (0, 0, 0):
            t = 1 + g["a_T"]
            q = sum((V[j] - g["a_u"]) ** 2 for j in range(3))
            np.testing.assert_allclose(F, np.exp(-q / (2 * t)) / (2 * np.pi * t) ** 1.5,
                                       rtol=1e-13, atol=1e-300)


def test_maxwellian_xv_3d3v_velocity_moments():
    """The 3d3v distribution of Sec. 5.2 (modes x, v_x, y, v_y, z, v_z): for
    fixed positions the quadrature over the three velocities of f is
    2 varrho (2 pi)^(3/2) sqrt(T_x T_y T_z), with varrho the sum over the
    three positions of rho / (2 sqrt(2 pi T)); the second moment in v_q is
    T_q + a_u^2 and the first moments vanish.  Positions s = -1/2, 0, 1/4,
    1/2 (T = 1/2, 1/2, 0.9, 1/2)."""
    nv = 49
    w = W.maxwellian_xv(3, 5, nv, vmin=-8.0, vmax=8.0)
    o = oracle.Oracle(w["n"], w["gen"], 2)
    g = w["gen"]
    v = -8.0 + 16.0 * np.arange(nv) / (nv - 1)
    h = 16.0 / (nv - 1)
    V = np.meshgrid(v, v, v, indexing="ij")
    for pos in [(2, 3, 0), (3, 4, 2)]:
        F = np.empty((nv, nv, nv))
        for a in range(nv):
            for b in range(nv):
                for c in range(nv):
                    F[a, b, c] = o.entry((pos[0], a, pos[1], b, pos[2], c))
        s = [-0.5 + i / 4 for i in pos]
        rho = [1 + g["a_rho"] * np.sin(2 * np.pi * t) for t in s]
        T = [0.5 + g["a_T"] * np.sin(2 * np.pi * t) for t in s]
        varrho = sum(r / (2 * np.sqrt(2 * np.pi * t)) for r, t in zip(rho, T))
        mass = 2 * varrho * (2 * np.pi) ** 1.5 * np.sqrt(T[0] * T[1] * T[2])
        m0 = F.sum() * h ** 3
        assert abs(m0 - mass) < 1e-9 * mass
        for q in range(3):
            assert abs((F * V[q]).sum() * h ** 3) < 1e-9 * mass
            m2 = (F * V[q] ** 2).sum() * h ** 3 / m0
            assert abs(m2 - (T[q] + g["a_u"] ** 2)) < 1e-9


def test_maxwellian_xv_velocity_moments():
    """The 2d2v distribution of Sec. 5.2 on a wide v-grid: for fixed
    positions (x, y) the quadrature over (v_x, v_y) of f, of v_x^2 f and of
    v_y^2 f returns what a sum of two Gaussians centred at -(0.75, 0.75) and
    +(0.75, 0.75) with variances (T(x), T(y)) and weight
    varrho(x, y) = rho(x) / (2 sqrt(2 pi T(x))) + rho(y) / (2 sqrt(2 pi T(y)))
    integrates to: 2 varrho 2 pi sqrt(T(x) T(y)) times 1, T(x) + 0.75^2 and
    T(y) + 0.75^2; the first moments vanish.  At s = 0 the paper's rho and T
    are 1 and 1/2, at s = 1/4 they are 1.875 and 0.9 (sin = 1)."""
    nv = 97
    w = W.maxwellian_xv(2, 5, nv, vmin=-12.0, vmax=12.0)
    o = oracle.Oracle(w["n"], w["gen"], 2)
    v = -12.0 + 24.0 * np.arange(nv) / (nv - 1)
    h = 24.0 / (nv - 1)
    s_of = lambda i: -0.5 + i / 4  # noqa: E731  positions -1/2, -1/4, 0, 1/4, 1/2
    for ix, iy in [(2, 2), (3, 2), (2, 3), (1, 3), (0, 4)]:
        F = np.array([[o.entry((ix, a, iy, b)) for b in range(nv)] for a in range(nv)])
        rx, tx = 1 + 0.875 * np.sin(2 * np.pi * s_of(ix)), 0.5 + 0.4 * np.sin(2 * np.pi * s_of(ix))
        ry, ty = 1 + 0.875 * np.sin(2 * np.pi * s_of(iy)), 0.5 + 0.4 * np.sin(2 * np.pi * s_of(iy))
        if ix == 3:
            assert abs(rx - 1.875) < 1e-15 and abs(tx - 0.9) < 1e-15
        if ix == 2:
            assert abs(rx - 1.0) < 1e-15 and abs(tx - 0.5) < 1e-15
        rho = rx / (2 * np.sqrt(2 * np.pi * tx)) + ry / (2 * np.sqrt(2 * np.pi * ty))
        mass = 2 * rho * 2 * np.pi * np.sqrt(tx * ty)
        m0 = F.sum() * h * h
        assert abs(m0 - mass) < 1e-9 * mass
        assert abs((F * v[:, None]).sum() * h * h) < 1e-9 * mass
        assert abs((F * v[None, :]).sum() * h * h) < 1e-9 * mass
        assert abs((F * v[:, None] ** 2).sum() * h * h / m0 - (tx + 0.75 ** 2)) < 1e-9
        assert abs((F * v[None, :] ** 2).sum() * h * h / m0 - (ty + 0.75 ** 2)) < 1e-9
    # interleaved order: swapping the (x, v_x) and (y, v_y) pairs of modes
    # leaves the function unchanged
    for idx in [(0, 3, 4, 50), (1, 96, 2, 7), (3, 40, 3, 41)]:
        assert o.entry(idx) == o.entry((idx[2], idx[3], idx[0], idx[1]))
