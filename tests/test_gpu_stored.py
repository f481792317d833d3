"""GPU stored-residual form (eq. aca_approx_E) vs the oracle's stored form:
identical pivots and factors (both follow the same arithmetic contract for
the carried residual), sampled error within 1e-12.  Every call goes through
the C ABI."""
import os

import numpy as np
import pytest

import oracle
from paper_2407_11290_gb300 import workloads as W

from test_gpu_parity import assert_same

pytestmark = pytest.mark.gpu

NT = os.cpu_count() or 1


@pytest.fixture(scope="module")
def tt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2407_11290_gb300 import ttcross
    return ttcross


def run_stored(tt, w, eps, max_rank, nsamples, grid=None, **kw):
    g = tt.TTCross(w["n"], w["gen"], max_rank=max_rank, nsamples=nsamples, residual="stored", **kw)
    g.run(eps, subtensor_grid=grid)
    rc = g.sync()
    o = oracle.Oracle(w["n"], w["gen"], max_rank, nthreads=NT, stored=True)
    orc, ost = o.run(eps, nsamples=nsamples)
    return g, rc, o, orc, ost


def test_stored_config0_hilbert3d(tt):
    w = W.CONFIGS["hilbert3d_n32"]
    g, rc, o, orc, ost = run_stored(tt, w, w["eps"], w["max_rank"], 0, grid=w["grid"])
    assert rc == orc == 0
    assert_same(g, o)
    st = g.stats()
    assert abs(st["err"] - ost["err"]) <= 1e-12 and st["err"] <= w["eps"]
    for k in range(1, o.d):
        np.testing.assert_array_equal(g.pivot_inverse(k), o.U(k - 1))
    # after the first screen only entries new to a superblock are formed
    assert st["entries_fresh"] < st["entries_screened"]
    assert st["stored_bytes"] > 0


def test_stored_config1_hilbert6d_full_size(tt):
    w = W.CONFIGS["hilbert6d_n64"]
    g, rc, o, orc, ost = run_stored(tt, w, w["eps"], w["max_rank"], w["nsamples"], grid=w["grid"])
    assert rc == orc == 0
    assert_same(g, o)
    st = g.stats()
    assert abs(st["err"] - ost["err"]) <= 1e-12 and st["err"] <= w["eps"]
    assert st["sweeps"] == ost["sweeps"] and st["entries_screened"] == ost["entries_screened"]


@pytest.mark.parametrize("grid", [None, [4] * 5, [3, 1, 2, 5, 7]])
def test_stored_ragged_tiles_and_grids(tt, grid):
    # n not a multiple of the 64-wide tiles: without a grid, tiles straddle the
    # boundary between stored and new rows / columns
    w = W.hilbert(5, 1)
    w["n"] = [37, 50, 23, 41, 29]
    g, rc, o, orc, ost = run_stored(tt, w, 1e-10, 20, 20000, grid=grid)
    assert rc == orc == 0
    assert_same(g, o)
    assert abs(g.stats()["err"] - ost["err"]) <= 1e-12


def test_stored_random_tt_and_separable(tt):
    w = W.random_tt([12, 12, 12, 12], [1, 3, 4, 3, 1], seed=7)
    g, rc, o, orc, ost = run_stored(tt, w, 1e-12, 10, 0)
    assert rc == orc == 0
    assert list(g.ranks()) == [1, 3, 4, 3, 1]
    assert_same(g, o)
    w = W.separable([7, 9, 5, 6, 3])
    g, rc, o, orc, ost = run_stored(tt, w, 1e-12, 8, 0)
    assert rc == orc == 0 and list(g.ranks()) == [1] * 6
    assert_same(g, o)


@pytest.mark.parametrize("shape,seed", [((70, 45), 2), ((65, 130), 4)])
def test_stored_d2_matrix_prescribed(tt, shape, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal(shape)
    A[0, 0] = 2.0
    n1, n2 = shape
    gen = {"kind": "tt", "ranks": [1, min(n1, 32), 1],
           "cores": [np.eye(n1)[:, :32].reshape(1, n1, -1), A[:32].reshape(min(n1, 32), n2, 1)]}
    w = {"n": [n1, n2], "gen": gen}
    cap = min(n1, n2, 32)
    g, rc, o, orc, ost = run_stored(tt, w, 0.0, cap, 0)
    assert rc == orc == 0
    assert_same(g, o)


def test_stored_host_stepped_equals_persistent(tt):
    w = W.hilbert(5, 20)
    a = tt.TTCross(w["n"], w["gen"], max_rank=32, nsamples=30000, residual="stored")
    a.run(1e-9)
    a.sync()
    b = tt.TTCross(w["n"], w["gen"], max_rank=32, nsamples=30000, residual="stored",
                   host_loop=True)
    b.run(1e-9)
    b.sync()
    for k in range(1, 6):
        np.testing.assert_array_equal(a.core(k), b.core(k))
    assert a.stats()["err"] == b.stats()["err"]


def test_stored_prescribed_ranks_and_rerun(tt):
    w = W.hilbert(4, 30)
    caps = [3, 6, 4]
    g = tt.TTCross(w["n"], w["gen"], max_rank=8, nsamples=10000, bond_max_rank=caps,
                   residual="stored")
    g.run(0.0)
    assert g.sync() == 0
    o = oracle.Oracle(w["n"], w["gen"], caps, nthreads=NT, stored=True)
    o.run(0.0, nsamples=10000)
    assert_same(g, o)
    # a second run on the same handle starts over (stored extents reset)
    g.run(0.0)
    assert g.sync() == 0
    assert_same(g, o)


def test_stored_config4_scale_error_and_cost(tt):
    """6D Hilbert n = 256 (the largest workload), stored form: error <= eps on
    the 10^6 samples, cross-checked at 2000 samples by the oracle's own TT
    evaluation of the GPU cores; only a small share of the screened entries is
    formed as A - T R."""
    w = W.CONFIGS["hilbert6d_n256"]
    g = tt.TTCross(w["n"], w["gen"], max_rank=w["max_rank"], nsamples=w["nsamples"],
                   residual="stored")
    g.run(w["eps"], subtensor_grid=w["grid"])
    assert g.sync() == 0
    st = g.stats()
    assert st["err"] <= w["eps"]
    assert st["entries_fresh"] < 0.5 * st["entries_screened"]
    cores = g.cores()
    idx = oracle.sample_indices(w["n"], 2000, seed=99)
    o = oracle.Oracle(w["n"], w["gen"], 1)
    num = den = 0.0
    for s in idx:
        x = o.entry(s)
        v = cores[0][:, s[0], :]
        for m in range(1, 6):
            v = v @ cores[m][:, s[m], :]
        num += (x - v[0, 0]) ** 2
        den += x * x
    assert (num / den) ** 0.5 <= 10 * w["eps"]


def test_stored_batch_equals_single(tt):
    ws = [W.hilbert(3, 20), W.hilbert(4, 11), W.random_tt([6, 7, 8], [1, 2, 3, 1], seed=5)]
    singles, batch = [], []
    for w in ws:
        a = tt.TTCross(w["n"], w["gen"], max_rank=16, nsamples=5000, residual="stored")
        a.run(1e-9)
        a.sync()
        singles.append(a)
        batch.append(tt.TTCross(w["n"], w["gen"], max_rank=16, nsamples=5000, residual="stored"))
    tt.run_batch(batch, 1e-9)
    for a, b in zip(singles, batch):
        assert b.sync() == a.sync()
        assert list(a.ranks()) == list(b.ranks())
        for k in range(1, len(a.n) + 1):
            np.testing.assert_array_equal(a.core(k), b.core(k))


def test_stored_maxwellian6d_reaches_eps_above_rank_128(tt):
    """The 6D Maxwellian (3x + 3v, n = 64) needs ranks above 128 at eps = 1e-6:
    the stored form reaches eps with rank cap 256; its error is cross-checked
    at 2000 samples from the oracle's entries and a numpy contraction of the
    GPU cores."""
    w = W.CONFIGS["maxwellian6d_n64"]
    g = tt.TTCross(w["n"], w["gen"], max_rank=w["max_rank"], nsamples=w["nsamples"],
                   residual="stored")
    g.run(w["eps"], subtensor_grid=w["grid"])
    assert g.sync() == 0
    st = g.stats()
    assert st["err"] <= w["eps"]
    assert max(g.ranks()) > 128
    cores = g.cores()
    idx = oracle.sample_indices(w["n"], 2000, seed=77)
    o = oracle.Oracle(w["n"], w["gen"], 1)
    num = den = 0.0
    for s in idx:
        x = o.entry(s)
        v = cores[0][:, s[0], :]
        for m in range(1, 6):
            v = v @ cores[m][:, s[m], :]
        num += (x - v[0, 0]) ** 2
        den += x * x
    assert (num / den) ** 0.5 <= 3 * w["eps"]


@pytest.mark.parametrize("ranks,n", [([1, 10, 48, 48, 10, 1], 10), ([1, 10, 100, 100, 10, 1], 10),
                                     ([1, 12, 132, 132, 12, 1], 12)])
def test_stored_long_replay_histories(tt, ranks, n):
    """Two adjacent bonds of rank above 32: rows entering a superblock replay
    pivot histories longer than a warp (Alg. 4 with 2, 4 and 8 entries of
    T(a, :) per lane).  Pivots, T, R and U equal the oracle's bit for bit, and
    the cross stops at the TT's own ranks."""
    w = W.random_tt([n] * 5, ranks, seed=21)
    g, rc, o, orc, ost = run_stored(tt, w, 1e-12, max(ranks) + 8, 0)
    assert rc == orc == 0
    assert list(g.ranks()) == ranks
    assert_same(g, o)


def test_recompute_long_replay_histories(tt):
    """The recompute form on the same replays (ranks 48, two register tiles)."""
    ranks = [1, 10, 48, 48, 10, 1]
    w = W.random_tt([10] * 5, ranks, seed=21)
    g = tt.TTCross(w["n"], w["gen"], max_rank=56, nsamples=0)
    g.run(1e-12)
    assert g.sync() == 0
    o = oracle.Oracle(w["n"], w["gen"], 56, nthreads=NT)
    orc, ost = o.run(1e-12, nsamples=0)
    assert orc == 0
    assert list(g.ranks()) == ranks
    assert_same(g, o)
