"""Pins for the oracle's stored-residual form (eq. aca_approx_E): the residual
kept in memory and carried through each pivot's rank-one step.  Each check is
against mathematics the paper fixes (the Schur complement, interpolation,
exact recovery), never against the oracle itself.  CPU only."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2407_11290_gb300 import workloads as W

from test_oracle import full_from_cores, full_tensor, matrix_as_tt


def exact_schur(A, I, J):
    """A - A(:,J) A(I,J)^{-1} A(I,:) in exact rational arithmetic (the
    textbook Schur complement; the inverse by Gauss-Jordan on Fractions)."""
    F = [[Fraction(float(x)) for x in row] for row in A]
    k = len(I)
    P = [[F[i][j] for j in J] for i in I]
    inv = [[Fraction(int(r == c)) for c in range(k)] for r in range(k)]
    for col in range(k):
        piv = next(r for r in range(col, k) if P[r][col] != 0)
        P[col], P[piv] = P[piv], P[col]
        inv[col], inv[piv] = inv[piv], inv[col]
        f = P[col][col]
        P[col] = [x / f for x in P[col]]
        inv[col] = [x / f for x in inv[col]]
        for r in range(k):
            if r != col and P[r][col] != 0:
                g = P[r][col]
                P[r] = [x - g * y for x, y in zip(P[r], P[col])]
                inv[r] = [x - g * y for x, y in zip(inv[r], inv[col])]
    n1, n2 = len(F), len(F[0])
    # W = inv @ A(I,:)
    Wm = [[sum(inv[t][u] * F[I[u]][c] for u in range(k)) for c in range(n2)] for t in range(k)]
    return [[F[a][c] - sum(F[a][J[t]] * Wm[t][c] for t in range(k)) for c in range(n2)]
            for a in range(n1)]


def stored_run_d2(A, steps):
    o = oracle.Oracle(list(A.shape), matrix_as_tt(A), steps, stored=True)
    assert o.init() == 0
    return o


# --------------------------------------------------------------------------
# d = 2: the stored residual after z pivots is the Schur complement of the
# pivot block, and every pivot is the exact argmax of it (complete pivoting).
@pytest.mark.parametrize("shape,seed", [((9, 7), 0), ((6, 11), 1)])
def test_stored_d2_is_exact_schur_complement(shape, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal(shape)
    A[0, 0] = 2.5
    steps = min(shape) - 1
    o = stored_run_d2(A, steps + 1)
    n1 = shape[0]
    amax = np.abs(A).max()
    for z in range(steps):
        rc, s = o.screen()
        assert rc == 0
        pr, pc = o.pivot_coords(0)
        S = exact_schur(A, list(pr), list(pc))
        E = o.stored_block(0)
        Sf = np.array([[float(x) for x in row] for row in S])
        np.testing.assert_allclose(E, Sf, rtol=0, atol=1e-12 * amax)
        # the exact argmax of |S| (ties: lowest column-major index) is the pivot
        mag = [(abs(S[a][c]), -(a + n1 * c), a, c) for a in range(shape[0]) for c in range(shape[1])]
        best = max(mag)
        second = sorted(mag)[-2]
        assert float(best[0] - second[0]) > 1e-9 * amax  # no near-tie in these draws
        assert (s["row"][0], s["col"][0]) == (best[2], best[3])
        assert o.apply([1], s["row"], s["col"]) == 0


def test_stored_pivot_row_becomes_exactly_zero():
    # w = -(E(a*,c*) / E(a*,c*)) = -1 exactly, so fma(-1, E(a*,c), E(a*,c)) = 0
    rng = np.random.default_rng(7)
    A = rng.standard_normal((10, 12))
    A[0, 0] = 3.0
    o = stored_run_d2(A, 6)
    for _ in range(4):
        rc, s = o.screen()
        a, c = int(s["row"][0]), int(s["col"][0])
        assert o.apply([1], s["row"], s["col"]) == 0
        o.screen()
        E = o.stored_block(0)
        assert np.all(E[a, :] == 0.0)
        # the pivot column is zero up to the rounding of w * E(a*, c*)
        assert np.abs(E[:, c]).max() <= 2.0**-52 * np.abs(A).max() * 4


# --------------------------------------------------------------------------
# d > 2: the carried residual tracks A - T R (formed independently by the
# factor recurrence) on every bond and every sweep, rows / columns that
# entered the superblock included.
@pytest.mark.parametrize("case", ["hilbert", "tt"])
def test_stored_tracks_recomputed_residual(case):
    if case == "hilbert":
        n, gen, cap = [12, 10, 11], {"kind": "hilbert"}, 8
    else:
        n, cap = [7, 8, 6, 9], 6
        gen = W.random_tt(n, [1, 3, 5, 4, 1], seed=11)["gen"]
    o = oracle.Oracle(n, gen, cap, stored=True, nthreads=2)
    xrms, start = o.sample_scan(0)
    assert o.init_at(start) == 0
    X = full_tensor(n, gen)
    amax = np.abs(X).max()
    for sweep in range(cap - 1):
        rc, s = o.screen()
        assert rc == 0
        for b in range(len(n) - 1):
            rows, cols = o.dims(b)
            E = o.stored_block(b)
            assert E.shape == (rows, cols)
            ref = np.array([[o.residual(b, a, c) for c in range(cols)] for a in range(rows)])
            np.testing.assert_allclose(E, ref, rtol=0, atol=1e-12 * amax)
        add = (s["best"] > 1e-14 * amax).astype(np.int32)
        add &= (o.ranks() < cap).astype(np.int32)
        if not add.any():
            break
        assert o.apply(add, s["row"], s["col"]) == 0


def test_stored_random_tt_stops_at_its_ranks():
    n = [10, 9, 11, 8]
    ranks = [1, 3, 4, 3, 1]
    gen = W.random_tt(n, ranks, seed=3)["gen"]
    o = oracle.Oracle(n, gen, 8, stored=True, nthreads=2)
    rc, st = o.run(1e-12, nsamples=0)
    assert rc == 0
    assert list(o.ranks()) == ranks[1:-1]
    X = full_tensor(n, gen)
    Xt = full_from_cores(o.cores())
    assert np.linalg.norm(X - Xt) / np.linalg.norm(X) <= 1e-12


def test_stored_separable_stays_rank_one():
    n = [9, 7, 8]
    gen = W.separable(n, seed=2)["gen"]
    o = oracle.Oracle(n, gen, 4, stored=True)
    rc, st = o.run(1e-12, nsamples=0)
    assert rc == 0 and list(o.ranks()) == [1, 1]
    X = full_tensor(n, gen)
    Xt = full_from_cores(o.cores())
    assert np.abs(X - Xt).max() <= 1e-15 * np.abs(X).max()


def test_stored_hilbert3d_config0_reaches_eps():
    o = oracle.Oracle([32, 32, 32], {"kind": "hilbert"}, 32, stored=True, nthreads=4)
    rc, st = o.run(1e-10, nsamples=0)
    assert rc == 0 and st["err"] <= 1e-10
    X = full_tensor([32, 32, 32], {"kind": "hilbert"})
    Xt = full_from_cores(o.cores())
    assert np.linalg.norm(X - Xt) / np.linalg.norm(X) == pytest.approx(st["err"], rel=1e-6)
