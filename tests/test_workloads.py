"""The seeded input recipes (CPU only): the workload table and the batch of
Maxwellians are what the workloads are defined to be, and they are
reproducible."""
import collections

from paper_2407_11290_gb300 import workloads as W


def test_workload_table():
    h3 = W.CONFIGS["hilbert3d_n32"]
    assert h3["n"] == [32] * 3 and h3["gen"]["kind"] == "hilbert"
    assert h3["eps"] == 1e-10 and h3["nsamples"] == 0 and h3["grid"] == [1, 1, 1]
    h64 = W.CONFIGS["hilbert6d_n64"]
    assert h64["n"] == [64] * 6 and h64["eps"] == 1e-8 and h64["max_rank"] == 64
    assert h64["grid"] == [2] * 6 and h64["nsamples"] == 10**6
    h256 = W.CONFIGS["hilbert6d_n256"]
    assert h256["n"] == [256] * 6 and h256["eps"] == 1e-10 and h256["max_rank"] == 128
    assert h256["grid"] == [4] * 6 and h256["nsamples"] == 10**6
    m = W.CONFIGS["maxwellian6d_n64"]
    g = m["gen"]
    assert m["n"] == [64] * 6 and m["eps"] == 1e-6 and m["grid"] == [4, 4, 4, 1, 1, 1]
    assert (g["kind"], g["dx"], g["dv"]) == ("maxwellian", 3, 3)
    assert (g["a_rho"], g["a_u"], g["a_T"], g["vmin"], g["vmax"]) == (0.5, 0.3, 0.2, -8.0, 8.0)


def test_paper_workloads_sizes_and_ranks():
    """Sec. 5.1 / 5.2: the Hilbert 3D n = 2000 and 6D n = 300 tensors and the
    interleaved 2d2v / 3d3v distributions with sizes (2n, n, ...)."""
    P = W.PAPER_WORKLOADS
    assert P["paper_hilbert3d_n2000"]["n"] == [2000] * 3
    assert P["paper_hilbert6d_n300"]["bond_ranks"] == [15, 17, 18, 17, 15]
    assert P["paper_2d2v_n1000"]["n"] == [2000, 1000, 2000, 1000]
    assert P["paper_3d3v_n400"]["n"] == [800, 400] * 3
    for w in P.values():
        assert w["eps"] == 0.0 and len(w["bond_ranks"]) == len(w["n"]) - 1


def test_batch_recipe():
    """256 Maxwellians: d in {4, 5, 6} with the (x, v) split 2+2, 2+3, 3+3,
    one n in {32, 48, 64, 96, 128} per instance, amplitudes in [0, 0.5);
    reproducible, and a shorter batch is a prefix of the longer one."""
    ws = W.maxwellian_batch(256)
    assert len(ws) == 256
    assert W.maxwellian_batch(256) == ws and W.maxwellian_batch(16) == ws[:16]
    ds, ns = collections.Counter(), collections.Counter()
    for w in ws:
        d, g = len(w["n"]), w["gen"]
        assert (g["dx"], g["dv"]) == {4: (2, 2), 5: (2, 3), 6: (3, 3)}[d]
        assert len(set(w["n"])) == 1 and w["n"][0] in (32, 48, 64, 96, 128)
        for key in ("a_rho", "a_u", "a_T"):
            assert 0.0 <= g[key] < 0.5
        ds[d] += 1
        ns[w["n"][0]] += 1
    # every class is drawn, none overwhelmingly (uniform draws: 256/3 and 256/5 expected)
    assert set(ds) == {4, 5, 6} and min(ds.values()) > 256 / 3 / 2
    assert set(ns) == {32, 48, 64, 96, 128} and min(ns.values()) > 256 / 5 / 2
    assert W.maxwellian_batch(8, seed=4) != W.maxwellian_batch(8)
