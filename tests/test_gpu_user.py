"""The user generator (an unfused batch callback that fills a device buffer
of values for a device buffer of int32 multi-indices, in stream order): a
callback computing the Hilbert tensor with torch reproduces the built-in
Hilbert generator bit for bit (pivots, pivot inverses, cores, error), in
both residual forms.  Every call goes through the C ABI."""
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


def hilbert_values(calls):
    def fn(idx, out):
        import torch
        calls.append(int(idx.shape[0]))
        s = idx.to(torch.int64).sum(dim=1) + 1
        out.copy_(1.0 / s.to(torch.float64))
    return fn


@pytest.mark.parametrize("residual,shape,eps,cap,ns,grid", [
    ("stored", [20, 18, 22, 19], 1e-10, 24, 30000, None),
    ("recompute", [20, 18, 22, 19], 1e-10, 24, 30000, [2, 3, 1, 2]),
    ("stored", [64] * 6, 1e-8, 64, 10**6, [2] * 6),
])
def test_user_callback_equals_builtin_hilbert(tt, residual, shape, eps, cap, ns, grid):
    calls = []
    u = tt.TTCross(shape, {"kind": "user", "fn": hilbert_values(calls)}, max_rank=cap,
                   nsamples=ns, residual=residual)
    u.run(eps, subtensor_grid=grid)
    assert u.sync() == tt.OK
    h = tt.TTCross(shape, {"kind": "hilbert"}, max_rank=cap, nsamples=ns, residual=residual)
    h.run(eps, subtensor_grid=grid)
    assert h.sync() == tt.OK
    assert list(u.ranks()) == list(h.ranks())
    for k in range(1, len(shape)):
        for a, b in zip(u.pivots(k), h.pivots(k)):
            np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(u.pivot_inverse(k), h.pivot_inverse(k))
    for k, (a, b) in enumerate(zip(u.cores(), h.cores()), start=1):
        np.testing.assert_array_equal(a, b, err_msg=f"core {k}")
    su, sh = u.stats(), h.stats()
    assert su["err"] == sh["err"] and su["sweeps"] == sh["sweeps"]
    # the samples and the origin first, then one call per decision that
    # brought new superblock entries
    assert calls[0] == (ns if ns < np.prod(shape) else np.prod(shape)) + 1
    assert 2 <= len(calls) <= su["sweeps"] + 2


def test_user_callback_errors_reach_python(tt):
    def bad(idx, out):
        raise ValueError("callback failed on purpose")
    u = tt.TTCross([8, 9, 10], {"kind": "user", "fn": bad}, max_rank=4, nsamples=100)
    with pytest.raises(ValueError):
        u.run(1e-6)
