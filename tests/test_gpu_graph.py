"""A run and a batch captured in a CUDA graph: replays rerun the whole cross
(the persistent kernel and its control-block set-up) and give the results of
an ordinary run, also after other runs of the same handles in between."""
import numpy as np
import pytest

from paper_2407_11290_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2407_11290_gb300 import ttcross
    return ttcross


def _state(c):
    return list(c.ranks()), c.stats()["err"], [c.core(k) for k in range(1, c.d + 1)]


def _same(c, ref):
    r, e, cores = ref
    assert list(c.ranks()) == r
    assert c.stats()["err"] == e
    for k in range(c.d):
        np.testing.assert_array_equal(c.core(k + 1), cores[k])


@pytest.mark.parametrize("precision,residual", [("fp64", "stored"), ("split", "stored"),
                                                ("fp64", "recompute")])
def test_run_captured_in_a_cuda_graph(tt, precision, residual):
    import torch
    w = W.CONFIGS["hilbert6d_n64"]
    g = tt.TTCross(w["n"], w["gen"], max_rank=w["max_rank"], nsamples=w["nsamples"],
                   precision=precision, residual=residual)
    g.run(w["eps"], subtensor_grid=w["grid"])
    assert g.sync() == tt.OK
    ref = _state(g)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        g.run(w["eps"], subtensor_grid=w["grid"], stream=s)
    # an ordinary run to another accuracy in between
    g.run(1e-4, subtensor_grid=w["grid"])
    assert g.sync() == tt.OK
    assert list(g.ranks()) != ref[0]
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        assert g.sync() == tt.OK
        _same(g, ref)
    g.close()


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_capture_that_would_allocate_is_refused(tt):
    """A subtensor grid of one-index pieces needs more candidate slots than
    the handle holds: the captured call refuses on the host (it would have
    to allocate); the same run outside a capture grows the slots."""
    import torch
    w = W.hilbert(3, 64)
    g = tt.TTCross(w["n"], w["gen"], max_rank=16, nsamples=4096, residual="stored")
    fine = [64, 64, 64]
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with pytest.raises(tt.TTCError) as e:
        with torch.cuda.graph(graph, stream=s):
            g.run(1e-8, subtensor_grid=fine, stream=s)
    assert e.value.status == tt.ERR_INVALID_ARG
    g.run(1e-8, subtensor_grid=fine)
    assert g.sync() == tt.OK
    g.close()


def test_batch_captured_in_a_cuda_graph(tt):
    import torch
    shapes = [(3, 32), (4, 16), (5, 12), (3, 24)]
    cs = []
    for d, n in shapes:
        w = W.hilbert(d, n)
        cs.append(tt.TTCross(w["n"], w["gen"], max_rank=16, nsamples=10**4, residual="stored"))
    eps = 1e-8
    tt.run_batch(cs, eps)
    for c in cs:
        assert c.sync() in (tt.OK, tt.NOT_CONVERGED)
    refs = [_state(c) for c in cs]
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        tt.run_batch(cs, eps, stream=s)
    # other batches led by the same handle in between
    tt.run_batch(cs[::-1], 1e-3)
    for c in cs:
        assert c.sync() in (tt.OK, tt.NOT_CONVERGED)
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        for c, ref in zip(cs, refs):
            assert c.sync() in (tt.OK, tt.NOT_CONVERGED)
            _same(c, ref)
    for c in cs:
        c.close()
