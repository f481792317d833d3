"""GPU FP64 form vs the CPU oracle: identical pivots (bit-exact integer
work), identical T factors (same arithmetic contract), sampled error within
1e-12.  Every call goes through the C ABI."""
import os

import numpy as np
import pytest

import oracle
from paper_2407_11290_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NT = os.cpu_count() or 1


@pytest.fixture(scope="module")
def tt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2407_11290_gb300 import ttcross
    return ttcross


def run_both(tt, w, eps, max_rank, nsamples, grid=None, **kw):
    g = tt.TTCross(w["n"], w["gen"], max_rank=max_rank, nsamples=nsamples, **kw)
    g.run(eps, subtensor_grid=grid)
    rc = g.sync()
    o = oracle.Oracle(w["n"], w["gen"], max_rank, nthreads=NT)
    orc, ost = o.run(eps, nsamples=nsamples)
    return g, rc, o, orc, ost


def assert_same(g, o, cores=True):
    d = o.d
    assert g.stats()["unscreened_slots"] == 0
    r = g.ranks()
    assert list(r[1:-1]) == list(o.ranks())
    for k in range(1, d):
        I, J = g.pivots(k)
        Io, Jo = o.pivots(k - 1)
        np.testing.assert_array_equal(I, Io)
        np.testing.assert_array_equal(J, Jo)
    if cores:
        for k, (a, b) in enumerate(zip(g.cores(), o.cores()), start=1):
            np.testing.assert_array_equal(a, b, err_msg=f"core {k}")


def test_config0_hilbert3d(tt):
    w = W.CONFIGS["hilbert3d_n32"]
    g, rc, o, orc, ost = run_both(tt, w, w["eps"], w["max_rank"], 0, grid=w["grid"])
    assert rc == orc == 0
    assert_same(g, o)
    st = g.stats()
    assert abs(st["err"] - ost["err"]) <= 1e-12
    assert st["err"] <= w["eps"]
    for k in range(1, o.d):
        np.testing.assert_array_equal(g.pivot_inverse(k), o.U(k - 1))


def test_config1_hilbert6d_full_size(tt):
    w = W.CONFIGS["hilbert6d_n64"]
    g, rc, o, orc, ost = run_both(tt, w, w["eps"], w["max_rank"], w["nsamples"], grid=w["grid"])
    assert rc == orc == 0
    assert_same(g, o)
    st = g.stats()
    assert abs(st["err"] - ost["err"]) <= 1e-12
    assert st["err"] <= w["eps"]
    assert st["sweeps"] == ost["sweeps"] and st["entries_screened"] == ost["entries_screened"]


@pytest.mark.parametrize("grid", [[1] * 6, [4] * 6, [3, 1, 2, 5, 1, 7]])
def test_grid_invariance(tt, grid):
    w = W.hilbert(6, 24)
    ref = tt.TTCross(w["n"], w["gen"], max_rank=32, nsamples=20000)
    ref.run(1e-9)
    ref.sync()
    g = tt.TTCross(w["n"], w["gen"], max_rank=32, nsamples=20000)
    g.run(1e-9, subtensor_grid=grid)
    g.sync()
    assert list(g.ranks()) == list(ref.ranks())
    for k in range(1, 6):
        for a, b in zip(g.pivots(k), ref.pivots(k)):
            np.testing.assert_array_equal(a, b)


def test_host_stepped_equals_persistent(tt):
    w = W.hilbert(5, 20)
    a = tt.TTCross(w["n"], w["gen"], max_rank=32, nsamples=30000)
    a.run(1e-9)
    a.sync()
    b = tt.TTCross(w["n"], w["gen"], max_rank=32, nsamples=30000, host_loop=True)
    b.run(1e-9)
    b.sync()
    for k in range(1, 6):
        np.testing.assert_array_equal(a.core(k), b.core(k))
    assert a.stats()["err"] == b.stats()["err"]


def test_random_tt_known_ranks(tt):
    w = W.random_tt([12, 12, 12, 12], [1, 3, 4, 3, 1], seed=7)
    g, rc, o, orc, ost = run_both(tt, w, 1e-12, 10, 0)
    assert rc == orc == 0
    assert list(g.ranks()) == [1, 3, 4, 3, 1]
    assert_same(g, o)
    assert abs(g.stats()["err"] - ost["err"]) <= 1e-12


def test_separable_rank1(tt):
    w = W.separable([7, 9, 5, 6, 3])
    g, rc, o, orc, ost = run_both(tt, w, 1e-12, 8, 0)
    assert rc == orc == 0
    assert list(g.ranks()) == [1, 1, 1, 1, 1, 1]
    assert_same(g, o)


@pytest.mark.parametrize("shape,seed", [((13, 29), 1), ((70, 45), 2), ((1, 9), 3), ((65, 130), 4)])
def test_d2_matrix_prescribed(tt, shape, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal(shape)
    A[0, 0] = 2.0
    n1, n2 = shape
    gen = {"kind": "tt", "ranks": [1, min(n1, 32), 1],
           "cores": [np.eye(n1)[:, :32].reshape(1, n1, -1), A[:32].reshape(min(n1, 32), n2, 1)]}
    w = {"n": [n1, n2], "gen": gen}
    cap = min(n1, n2, 32)
    g, rc, o, orc, ost = run_both(tt, w, 0.0, cap, 0)
    assert rc == orc == 0
    assert_same(g, o)


def test_ragged_and_unit_modes(tt):
    w = W.hilbert(4, 1)
    w["n"] = [1, 67, 3, 130]
    g, rc, o, orc, ost = run_both(tt, w, 1e-10, 24, 0)
    assert rc == orc == 0
    assert_same(g, o)


def _coords(o, b, Irow, Jrow):
    """Superblock (row, col) of the pivot (I_{<=k} entry, J_{>k} entry) in the
    oracle's current index sets."""
    n = o.n
    p = 0
    if b > 0:
        Il, _ = o.pivots(b - 1)
        p = int(np.flatnonzero((Il == Irow[:-1]).all(axis=1))[0])
    q = 0
    if b < o.d - 2:
        _, Jr = o.pivots(b + 1)
        q = int(np.flatnonzero((Jr == Jrow[1:]).all(axis=1))[0])
    return p * int(n[b]) + int(Irow[-1]), q * int(n[b + 1]) + int(Jrow[0])


def replay_with_resync(g, w, eps, cap, nsamples, rel=1e-13, stored=False, max_refine=6,
                       floor=0.0, first_stage=False):
    """Step the oracle sweep by sweep beside the GPU's pivots.  Where the two
    differ, the GPU's pivot must be a near-tie: its FP64 residual within
    rel * max|X| of the oracle's best (ulp-level differences of the entries
    reach the residual through A - T R, so they scale with |X|, not |E|); the
    oracle then continues from it.  ``stored``: the oracle's stored-residual
    form, whose screen reads the carried E (the near-tie check too).  When no
    bond adds, the oracle's sampled error decides as in its own run: done at
    eps, else tau / 10 while ranks and refinements remain.  ``floor``: below
    floor * max|X| the two residuals are rounding noise of comparable size,
    so a differing pivot there is re-synced without the near-tie check.
    ``first_stage``: stop when no bond adds at tau = eps (the GPU's pivots of
    that stage are then a prefix of its lists).
    Returns (oracle, number of re-synced pivots)."""
    o = oracle.Oracle(w["n"], w["gen"], cap, nthreads=NT, stored=stored)
    caps = list(np.broadcast_to(np.asarray(cap), (o.d - 1,)))
    rms, start = o.sample_scan(nsamples)
    gI = [g.pivots(k) for k in range(1, o.d)]
    np.testing.assert_array_equal(np.concatenate([gI[0][0][0], gI[0][1][0]]), start)
    assert o.init_at(start) == 0
    xmax = abs(o.entry(start))
    ties = 0
    tau = eps
    refinements = 0
    while True:
        rc, sc = o.screen()
        assert rc == 0
        r = o.ranks()
        theta = tau * rms
        add = [int(sc["best"][b] > theta and sc["best"][b] > 0 and r[b] < caps[b])
               for b in range(o.d - 1)]
        if not any(add):
            if first_stage or eps == 0.0 or o.sampled_error(nsamples) <= eps:
                break
            if all(r[b] >= caps[b] for b in range(o.d - 1)) or refinements >= max_refine:
                break
            tau /= 10.0
            refinements += 1
            continue
        rows, cols = sc["row"].copy(), sc["col"].copy()
        for b in range(o.d - 1):
            if not add[b]:
                continue
            z = int(r[b])
            if z >= len(gI[b][0]) and sc["best"][b] <= floor * xmax:
                add[b] = 0  # below the noise floor the GPU stopped this bond
                continue
            assert z < len(gI[b][0]), f"GPU stopped bond {b + 1} at rank {z}"
            a, c = _coords(o, b, gI[b][0][z], gI[b][1][z])
            piv = o.residual(b, a, c)
            with np.errstate(divide="ignore", over="ignore"):
                inv = np.float64(1.0) / np.float64(piv)
            if np.isfinite(piv) and not np.isfinite(inv):
                add[b] = 0  # a zero pivot: the bond takes none (in both runs)
                continue
            if (a, c) != (rows[b], cols[b]):
                e = abs(o.stored_residual(b, a, c) if stored else o.residual(b, a, c))
                if sc["best"][b] > floor * xmax:
                    assert e >= sc["best"][b] - rel * xmax, (b, e, sc["best"][b])
                ties += 1
                rows[b], cols[b] = a, c
        if any(add):
            assert o.apply(add, rows, cols) == 0
    return o, ties


def test_maxwellian_small(tt):
    """Entries come from CUDA's sin/cos/exp/pow, which may differ from glibc's
    in the last bit: pivots must agree except at near-ties (re-synced)."""
    w = W.maxwellian(2, 2, 16, a_rho=0.4, a_u=0.3, a_T=0.2)
    g = tt.TTCross(w["n"], w["gen"], max_rank=64, nsamples=50000)
    g.run(1e-6)
    assert g.sync() == 0
    assert g.stats()["refinements"] == 0
    o, ties = replay_with_resync(g, w, 1e-6, 64, 50000)
    assert list(g.ranks()[1:-1]) == list(o.ranks())
    for k in range(1, o.d):
        for a, b in zip(g.pivots(k), o.pivots(k - 1)):
            np.testing.assert_array_equal(a, b)
    assert abs(g.stats()["err"] - o.sampled_error(50000)) <= 1e-12
    print(f"maxwellian 2x2v n=16: {ties} near-tie(s) re-synced")


def test_prescribed_ranks_per_bond(tt):
    w = W.hilbert(5, 30)
    caps = [3, 5, 6, 4]
    g = tt.TTCross(w["n"], w["gen"], max_rank=8, nsamples=10000, bond_max_rank=caps)
    g.run(0.0)
    assert g.sync() == 0
    assert list(g.ranks()) == [1] + caps + [1]
    o = oracle.Oracle(w["n"], w["gen"], caps, nthreads=NT)
    o.run(0.0, nsamples=10000)
    assert_same(g, o)


def test_zero_start_and_nonfinite(tt):
    # X(0,...,0) = 0 but other entries are not: the start moves to the max
    w = W.random_tt([4, 5, 6], [1, 2, 2, 1], seed=3)
    w["gen"]["cores"][0][:, 0, :] = 0.0
    g, rc, o, orc, ost = run_both(tt, w, 1e-10, 4, 0)
    assert rc == orc == 0
    assert_same(g, o)
    # X = 0 everywhere
    w["gen"]["cores"][1][:] = 0.0
    g = tt.TTCross(w["n"], w["gen"], max_rank=3, nsamples=0)
    g.run(1e-6)
    assert g.sync(allow=(tt.ERR_ZERO_START,)) == tt.ERR_ZERO_START
    w = W.random_tt([4, 5, 6], [1, 2, 2, 1], seed=3)
    w["gen"]["cores"][1][:, 3, :] = np.nan
    g = tt.TTCross(w["n"], w["gen"], max_rank=3, nsamples=0)
    g.run(1e-6)
    assert g.sync(allow=(tt.ERR_NONFINITE,)) == tt.ERR_NONFINITE


def test_device_wait_limit_returns_status(tt):
    """A wait that runs out returns TTC_ERR_DEVICE_TIMEOUT; the context stays usable."""
    w = W.hilbert(4, 16)
    g = tt.TTCross(w["n"], w["gen"], max_rank=16, nsamples=1000, wait_limit_s=1e-9)
    g.run(1e-8)
    assert g.sync(allow=(tt.ERR_DEVICE_TIMEOUT,)) == tt.ERR_DEVICE_TIMEOUT
    h = tt.TTCross(w["n"], w["gen"], max_rank=16, nsamples=1000)
    h.run(1e-8)
    assert h.sync() == 0


def test_batch_equals_single(tt):
    ws = [W.hilbert(3, 20), W.hilbert(4, 11), W.random_tt([6, 7, 8], [1, 2, 3, 1], seed=5)]
    singles, batch = [], []
    for w in ws:
        a = tt.TTCross(w["n"], w["gen"], max_rank=16, nsamples=5000)
        a.run(1e-9)
        a.sync()
        singles.append(a)
        batch.append(tt.TTCross(w["n"], w["gen"], max_rank=16, nsamples=5000))
    tt.run_batch(batch, [1e-9] * 3)
    for a, b in zip(singles, batch):
        b.sync()
        assert list(a.ranks()) == list(b.ranks())
        for k in range(1, a.d + 1):
            np.testing.assert_array_equal(a.core(k), b.core(k))


# ---------------------------------------------------------------------------
# mixed forms: FP32 / float-float screens with FP64 re-scoring and FP64
# refinement of every tile whose error bound could hide the FP64 argmax, so
# the pivots must still equal the FP64 oracle's.

@pytest.mark.parametrize("prec", ["split", "fp32"])
def test_mixed_config1_pivots_equal_oracle(tt, prec):
    w = W.CONFIGS["hilbert6d_n64"]
    g = tt.TTCross(w["n"], w["gen"], max_rank=w["max_rank"], nsamples=w["nsamples"],
                   precision=prec)
    g.run(w["eps"], subtensor_grid=w["grid"])
    assert g.sync() == 0
    o = oracle.Oracle(w["n"], w["gen"], w["max_rank"], nthreads=NT)
    orc, ost = o.run(w["eps"], nsamples=w["nsamples"])
    assert_same(g, o)
    st = g.stats()
    assert abs(st["err"] - ost["err"]) <= 1e-12
    assert st["unscreened_slots"] == 0
    print(f"{prec}: tiles refined in FP64 {st['tiles_refined']}, sweeps {st['sweeps']}")


@pytest.mark.parametrize("prec", ["split", "fp32"])
def test_mixed_small_cases(tt, prec):
    for w, eps, cap, ns in [(W.hilbert(3, 32), 1e-10, 64, 0),
                            (W.random_tt([12, 12, 12, 12], [1, 3, 4, 3, 1], seed=7), 1e-12, 10, 0),
                            (W.hilbert(4, 1), 1e-10, 24, 0)]:
        if w["n"] == [1] * 4:
            w["n"] = [1, 67, 3, 130]
        g = tt.TTCross(w["n"], w["gen"], max_rank=cap, nsamples=ns, precision=prec)
        g.run(eps)
        assert g.sync() == 0
        o = oracle.Oracle(w["n"], w["gen"], cap, nthreads=NT)
        orc, ost = o.run(eps, nsamples=ns)
        assert orc == 0
        assert_same(g, o)


def test_maxwellian_batch_recipe_small(tt):
    """The batch recipe's instances (uneven d, n, amplitudes) run in one
    launch equal their single runs; the smallest also matches the oracle."""
    ws = W.maxwellian_batch(3)
    for w in ws:
        w["n"] = [min(v, 12) for v in w["n"]]
    singles = []
    for w in ws:
        a = tt.TTCross(w["n"], w["gen"], max_rank=24, nsamples=20000)
        a.run(1e-5)
        a.sync(allow=(tt.OK, tt.NOT_CONVERGED))
        singles.append(a)
    batch = [tt.TTCross(w["n"], w["gen"], max_rank=24, nsamples=20000) for w in ws]
    tt.run_batch(batch, 1e-5)
    for a, b in zip(singles, batch):
        b.sync(allow=(tt.OK, tt.NOT_CONVERGED))
        assert list(a.ranks()) == list(b.ranks())
        for k in range(1, a.d + 1):
            np.testing.assert_array_equal(a.core(k), b.core(k))
    w = ws[0]
    if singles[0].stats()["refinements"] == 0 and singles[0].stats()["status"] == tt.OK:
        o, ties = replay_with_resync(singles[0], w, 1e-5, 24, 20000)
        assert list(singles[0].ranks()[1:-1]) == list(o.ranks())


def test_mixed_host_stepped_and_batch(tt):
    w = W.hilbert(5, 20)
    a = tt.TTCross(w["n"], w["gen"], max_rank=32, nsamples=30000, precision="split")
    a.run(1e-9)
    a.sync()
    b = tt.TTCross(w["n"], w["gen"], max_rank=32, nsamples=30000, precision="split", host_loop=True)
    b.run(1e-9)
    b.sync()
    c = tt.TTCross(w["n"], w["gen"], max_rank=32, nsamples=30000, precision="fp64")
    d = tt.TTCross(W.hilbert(3, 40)["n"], w["gen"], max_rank=32, nsamples=30000, precision="split")
    tt.run_batch([c, d], [1e-9, 1e-9])
    c.sync()
    d.sync()
    for k in range(1, 6):
        np.testing.assert_array_equal(a.core(k), b.core(k))
        np.testing.assert_array_equal(a.core(k), c.core(k))
    e = tt.TTCross(W.hilbert(3, 40)["n"], w["gen"], max_rank=32, nsamples=30000)
    e.run(1e-9)
    e.sync()
    for k in range(1, 4):
        np.testing.assert_array_equal(d.core(k), e.core(k))
