"""GPU Alg. 1 with a random sample set L and the row / column refinement of
its while loop (recompute form, FP64) vs the oracle's: the same SplitMix64
samples, the same refinement, so pivots, T factors and cores are equal bit
for bit on exactly specified entries, sampled error within 1e-12.  Every
call goes through the C ABI."""
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


def run_sampled(tt, w, eps, cap, ns, nl, rook, grid=None, seed=77, **kw):
    g = tt.TTCross(w["n"], w["gen"], max_rank=cap, nsamples=ns, screen_samples=nl,
                   screen_seed=seed, rook_rounds=rook, **kw)
    g.run(eps, subtensor_grid=grid)
    rc = g.sync(allow=(tt.OK, tt.NOT_CONVERGED))
    o = oracle.Oracle(w["n"], w["gen"], cap, nthreads=NT)
    o.set_sampled(nl, seed=seed, max_rook=rook)
    orc, ost = o.run(eps, nsamples=ns)
    return g, rc, o, orc, ost


@pytest.mark.parametrize("nl,rook", [(64, 0), (64, 8), (1000, 3)])
def test_sampled_hilbert3d_equals_oracle(tt, nl, rook):
    w = W.CONFIGS["hilbert3d_n32"]
    g, rc, o, orc, ost = run_sampled(tt, w, w["eps"], w["max_rank"], 0, nl, rook)
    assert rc == orc
    assert_same(g, o)
    st = g.stats()
    assert abs(st["err"] - ost["err"]) <= 1e-12
    assert st["sweeps"] == ost["sweeps"] and st["entries_screened"] == ost["entries_screened"]


def test_sampled_ragged_random_tt_and_host_loop(tt):
    w = dict(n=[37, 50, 23, 41, 29], gen={"kind": "hilbert"})
    g, rc, o, orc, ost = run_sampled(tt, w, 1e-9, 24, 20000, 500, 6)
    assert rc == orc
    assert_same(g, o)
    assert abs(g.stats()["err"] - ost["err"]) <= 1e-12
    h = tt.TTCross(w["n"], w["gen"], max_rank=24, nsamples=20000, screen_samples=500,
                   screen_seed=77, rook_rounds=6, host_loop=True)
    h.run(1e-9)
    h.sync(allow=(tt.OK, tt.NOT_CONVERGED))
    for k in range(1, 6):
        np.testing.assert_array_equal(g.core(k), h.core(k))
    wt = W.random_tt([12, 12, 12, 12], [1, 3, 4, 3, 1], seed=7)
    g, rc, o, orc, ost = run_sampled(tt, wt, 1e-12, 10, 0, 40, 8)
    assert rc == orc == 0
    assert list(g.ranks()) == [1, 3, 4, 3, 1]
    assert_same(g, o)


def test_sampled_batch_equals_single(tt):
    ws = [W.hilbert(3, 20), W.hilbert(4, 11)]
    singles, batch = [], []
    for w in ws:
        a = tt.TTCross(w["n"], w["gen"], max_rank=16, nsamples=5000, screen_samples=200,
                       rook_rounds=4)
        a.run(1e-9)
        a.sync(allow=(tt.OK, tt.NOT_CONVERGED))
        singles.append(a)
        batch.append(tt.TTCross(w["n"], w["gen"], max_rank=16, nsamples=5000,
                                screen_samples=200, rook_rounds=4))
    # a batch mixing a sampled instance with an exhaustive one
    e = tt.TTCross(W.hilbert(3, 16)["n"], {"kind": "hilbert"}, max_rank=16, nsamples=5000)
    e1 = tt.TTCross(W.hilbert(3, 16)["n"], {"kind": "hilbert"}, max_rank=16, nsamples=5000)
    e1.run(1e-9)
    e1.sync()
    tt.run_batch(batch + [e], 1e-9)
    for a, b in zip(singles + [e1], batch + [e]):
        b.sync(allow=(tt.OK, tt.NOT_CONVERGED))
        assert list(a.ranks()) == list(b.ranks())
        for k in range(1, len(a.n) + 1):
            np.testing.assert_array_equal(a.core(k), b.core(k))


def test_sampled_config4_prescribed_rank_128(tt):
    """The 6D Hilbert tensor n = 256 grown to rank 128 on every bond
    (prescribed-rank mode) with 2^20 samples per screen: far fewer entries
    evaluated than the superblocks hold; the first sweeps' pivots equal the
    oracle's (checked on a rank-6 run of both)."""
    w = W.CONFIGS["hilbert6d_n256"]
    g = tt.TTCross(w["n"], w["gen"], max_rank=128, nsamples=10**5, screen_samples=1 << 20,
                   rook_rounds=4)
    g.run(0.0)
    assert g.sync() == tt.OK
    st = g.stats()
    assert max(g.ranks()) == 128
    full = sum((128 * 256) ** 2 for _ in range(3)) + 2 * 256 * 128 * 256
    assert st["entries_screened"] < 0.05 * full * st["sweeps"]
    small = tt.TTCross(w["n"], w["gen"], max_rank=6, nsamples=10**5, screen_samples=1 << 14,
                       rook_rounds=4)
    small.run(0.0)
    assert small.sync() == tt.OK
    o = oracle.Oracle(w["n"], w["gen"], 6, nthreads=NT)
    o.set_sampled(1 << 14, seed=20240715, max_rook=4)
    orc, ost = o.run(0.0, nsamples=10**5)
    assert orc == 0
    assert_same(small, o)
    print(f"config 4 at rank 128, sampled screen: {st['device_ms']:.1f} ms, "
          f"{st['sweeps']} sweeps, err {st['err']:.3e}, "
          f"{st['entries_screened'] / st['sweeps']:.3e} entries per sweep")
