"""Pins for the oracle's Alg. 1 with a random sample set L and the row /
column refinement of its while loop (recompute form).  Checked against what
the algorithm and the mathematics fix: the drawn samples follow the
published SplitMix64 outputs, the unrefined pivot is the brute-force argmax
over them, a refined pivot dominates its row and its column of the residual,
and exact low-rank tensors are still recovered.  CPU only."""
import os

import numpy as np

import oracle
from paper_2407_11290_gb300 import workloads as W

from test_oracle import full_tensor, matrix_as_tt

NT = min(os.cpu_count() or 1, 8)


def _mulhi(x, n):
    return (x * n) >> 64


def test_samples_follow_splitmix64_and_pivot_is_their_argmax():
    """max_rook = 0: the pivot of each bond is the argmax over the nl drawn
    entries, recomputed here from the published generator (outputs 2k and
    2k + 1 of SplitMix64 with k = (t (d-1) + b) nl + j) and the oracle's own
    residuals of those entries, ties to the lowest linear index."""
    w = W.hilbert(3, 9)
    nl, seed = 40, 1234
    o = oracle.Oracle(w["n"], w["gen"], 6)
    o.set_sampled(nl, seed=seed, max_rook=0)
    assert o.init() == 0
    n = w["n"]
    for t in range(3):
        rc, sc = o.screen()
        assert rc == 0
        assert o.last_screened() == nl * (o.d - 1)
        for b in range(o.d - 1):
            rows, cols = o.dims(b)
            best = None
            for j in range(nl):
                k = (t * (o.d - 1) + b) * nl + j
                a = _mulhi(W.splitmix64(seed, 2 * k), rows)
                c = _mulhi(W.splitmix64(seed, 2 * k + 1), cols)
                v = abs(o.residual(b, a, c))
                # linear index of superblock entry (a, c): prefix / suffix sets
                p, i = divmod(a, n[b])
                q, jj = divmod(c, n[b + 1])
                idx = []
                if b > 0:
                    idx += list(o.pivots(b - 1)[0][p])
                idx += [i, jj]
                if b < o.d - 2:
                    idx += list(o.pivots(b + 1)[1][q])
                lin = sum(int(x) * int(np.prod(n[:m])) for m, x in enumerate(idx))
                key = (-v, lin)
                if best is None or key < best[0]:
                    best = (key, a, c)
            assert (sc["row"][b], sc["col"][b]) == (best[1], best[2]), (t, b)
            assert sc["best"][b] == -best[0][0]
        r = o.ranks()
        add = [int(sc["best"][b] > 0 and r[b] < 6) for b in range(o.d - 1)]
        assert o.apply(add, sc["row"], sc["col"]) == 0


def test_refined_pivot_dominates_its_row_and_column():
    """With enough refinement rounds the pivot of Alg. 1 is a rook pivot: no
    entry of its row or its column of the residual is larger (d = 2: the
    superblock is the whole matrix)."""
    rng = np.random.default_rng(11)
    A = rng.standard_normal((23, 31))
    w = {"n": [23, 31], "gen": matrix_as_tt(A)}
    o = oracle.Oracle(w["n"], w["gen"], 12)
    o.set_sampled(5, seed=7, max_rook=50)
    assert o.init() == 0
    moves = 0
    for step in range(11):
        rc, sc = o.screen()
        assert rc == 0
        a, c = int(sc["row"][0]), int(sc["col"][0])
        E = np.array([[o.residual(0, i, j) for j in range(31)] for i in range(23)])
        assert abs(E[a, c]) == sc["best"][0]
        assert np.all(np.abs(E[:, c]) <= abs(E[a, c]))
        assert np.all(np.abs(E[a, :]) <= abs(E[a, c]))
        assert o.apply([1], sc["row"], sc["col"]) == 0
    assert o.rook_moves() > 0  # the refinement did move pivots


def test_sampled_screen_recovers_random_tt_and_rank_one():
    """Random sample sets still find the exact ranks of a random TT (every
    nonzero residual of a low-rank remainder is found by the refinement) and
    keep a rank-one tensor at rank one."""
    w = W.random_tt([10, 11, 9, 8], [1, 3, 4, 2, 1], seed=3)
    o = oracle.Oracle(w["n"], w["gen"], 8, nthreads=NT)
    o.set_sampled(30, seed=5, max_rook=8)
    rc, st = o.run(1e-12, nsamples=0)
    assert rc == 0
    assert list(o.ranks()) == [3, 4, 2]
    X = full_tensor(w["n"], w["gen"])
    from test_oracle import full_from_cores
    Y = full_from_cores(o.cores())
    assert np.linalg.norm(X - Y) <= 1e-12 * np.linalg.norm(X)
    ws = W.separable([6, 7, 5])
    o = oracle.Oracle(ws["n"], ws["gen"], 4)
    o.set_sampled(10, seed=1, max_rook=4)
    rc, st = o.run(1e-12, nsamples=0)
    assert rc == 0 and list(o.ranks()) == [1, 1]


def test_sampled_screen_reaches_eps_on_hilbert3d_with_fewer_entries():
    """The 32^3 Hilbert tensor at eps = 1e-10 with 200 samples per bond and
    refinement: the verified error reaches eps while the screens evaluate a
    small share of the entries the exhaustive screens do."""
    w = W.CONFIGS["hilbert3d_n32"]
    o = oracle.Oracle(w["n"], w["gen"], w["max_rank"], nthreads=NT)
    o.set_sampled(200, seed=9, max_rook=8)
    rc, st = o.run(w["eps"], nsamples=0)
    assert rc == 0 and st["err"] <= w["eps"]
    e = oracle.Oracle(w["n"], w["gen"], w["max_rank"], nthreads=NT)
    rc2, st2 = e.run(w["eps"], nsamples=0)
    assert rc2 == 0
    assert st["entries_screened"] < 0.5 * st2["entries_screened"]
