"""ttcross_sampled_error_noalloc: the sampled error for callers that cannot
allocate device memory (custom allocators and pool callbacks, processes with
a GPU memory budget fixed at start-up, hosts that forbid cudaMalloc after
initialisation).  Called through the C ABI and compared with the error that
ttcross_run reports for the same cores and samples, within the 1e-12 the
parity tests use, on two calls in a row (the static scratch is shared and
reused).  This file is collected last on purpose."""
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


@pytest.mark.parametrize("case", ["hilbert", "maxwellian", "every_entry"])
def test_noalloc_error_matches_run(tt, case):
    import torch
    if case == "hilbert":
        w, eps, ns, cap = W.hilbert(5, 20), 1e-9, 200000, 32
    elif case == "maxwellian":
        w, eps, ns, cap = W.maxwellian(2, 2, 16, a_rho=0.4, a_u=0.3, a_T=0.2), 1e-6, 50000, 64
    else:
        w, eps, ns, cap = W.hilbert(3, 32), 1e-10, 0, 32
    g = tt.TTCross(w["n"], w["gen"], max_rank=cap, nsamples=ns, seed=77)
    g.run(eps)
    assert g.sync() == tt.OK
    ref = g.stats()["err"]
    cores = [g.core(k, device=True) for k in range(1, g.d + 1)]
    torch.cuda.synchronize()
    for _ in range(2):
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        tt.sampled_error_noalloc(w["n"], w["gen"], cores, ns, 77, out)
        torch.cuda.synchronize()
        assert abs(out.item() - ref) <= 1e-12, (out.item(), ref)


def test_noalloc_rejects_oversize_and_tt_generator(tt):
    import torch
    w = W.hilbert(3, 8)
    g = tt.TTCross(w["n"], w["gen"], max_rank=8, nsamples=1000)
    g.run(1e-6)
    g.sync()
    cores = [g.core(k, device=True) for k in range(1, 4)]
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(tt.TTCError) as e:  # rejected on the host, nothing launched
        tt.sampled_error_noalloc([300, 300, 300], w["gen"], cores, 4096 * 4096 + 1, 1, out)
    assert e.value.status == tt.ERR_INVALID_ARG and "static scratch" in str(e.value)
    tw = W.random_tt([8, 8, 8], [1, 2, 2, 1])
    with pytest.raises(tt.TTCError):
        tt.sampled_error_noalloc(tw["n"], tw["gen"], cores, 1000, 1, out)
    torch.cuda.synchronize()
    assert np.isfinite(out.item())
