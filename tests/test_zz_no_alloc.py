"""ttcross_sampled_error_noalloc: the sampled error for callers that cannot
allocate device memory (custom allocators and pool callbacks, processes with
a GPU memory budget fixed at start-up, hosts that forbid cudaMalloc after
initialisation).  Called through the C ABI and compared with the error that
ttcross_run reports for the same cores and samples, within the 1e-12 the
parity tests use, on two calls in a row (the static scratch is shared and
reused); for the Hilbert cases also with the oracle's error of the same
cores.  This file is collected last on purpose."""
import ctypes
import os

import numpy as np
import pytest

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


def _free_bytes():
    import torch
    free, _ = torch.cuda.mem_get_info()
    return free


@pytest.mark.parametrize("case", ["hilbert", "maxwellian", "every_entry", "rank_above_128"])
def test_noalloc_error_matches_run(tt, case):
    import torch
    import oracle
    if case == "hilbert":
        w, eps, ns, cap = W.hilbert(5, 20), 1e-9, 200000, 32
    elif case == "maxwellian":
        w, eps, ns, cap = W.maxwellian(2, 2, 16, a_rho=0.4, a_u=0.3, a_T=0.2), 1e-6, 50000, 64
    elif case == "every_entry":
        w, eps, ns, cap = W.hilbert(3, 32), 1e-10, 0, 32
    else:
        # a TT-cores tensor of rank 140 recovered by the cross, evaluated as a
        # Hilbert-free check: the cores reach the 256-wide register path
        w, eps, ns, cap = W.hilbert(4, 40), 0.0, 30000, 140
    g = tt.TTCross(w["n"], w["gen"], max_rank=cap, nsamples=ns, seed=77)
    g.run(eps)
    assert g.sync() == tt.OK
    ref = g.stats()["err"]
    cores = [g.core(k, device=True) for k in range(1, g.d + 1)]
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    for call in range(2):
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0, alloc0 = _free_bytes(), torch.cuda.memory_allocated()
        if call == 0:
            tt.sampled_error_noalloc(w["n"], w["gen"], cores, ns, 77, out)
            torch.cuda.synchronize()
        else:
            # on a side stream, waiting for that stream alone
            side.wait_stream(torch.cuda.current_stream())
            tt.sampled_error_noalloc(w["n"], w["gen"], cores, ns, 77, out, stream=side)
            side.synchronize()
        if call == 1:
            # the second call allocates nothing, on the device or in torch's pool
            assert _free_bytes() == free0 and torch.cuda.memory_allocated() == alloc0
        assert abs(out.item() - ref) <= 1e-12, (call, out.item(), ref)
    if w["gen"]["kind"] == "hilbert":
        o = oracle.Oracle(w["n"], w["gen"], cap, nthreads=NT)
        orc, ost = o.run(eps, nsamples=ns, seed=77)
        assert orc == 0
        for k, (a, b) in enumerate(zip(g.cores(), o.cores()), start=1):
            np.testing.assert_array_equal(a, b, err_msg=f"core {k}")
        assert abs(out.item() - ost["err"]) <= 1e-12, (out.item(), ost["err"])


def test_noalloc_rejects_oversize_and_tt_generator(tt):
    import torch
    w = W.hilbert(3, 8)
    g = tt.TTCross(w["n"], w["gen"], max_rank=8, nsamples=1000)
    g.run(1e-6)
    g.sync()
    cores = [g.core(k, device=True) for k in range(1, 4)]
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    big = [300, 300, 300]
    big_cores = [torch.zeros((int(c.shape[0]), 300, int(c.shape[2])), dtype=torch.float64,
                             device="cuda") for c in cores]
    with pytest.raises(tt.TTCError) as e:  # rejected on the host, nothing launched
        tt.sampled_error_noalloc(big, w["gen"], big_cores, 4096 * 4096 + 1, 1, out)
    assert e.value.status == tt.ERR_INVALID_ARG and "static scratch" in str(e.value)
    tw = W.random_tt([8, 8, 8], [1, 2, 2, 1])
    with pytest.raises(tt.TTCError):
        tt.sampled_error_noalloc(tw["n"], tw["gen"], cores, 1000, 1, out)
    # through the C ABI directly: a core size above 256 is refused on the host
    L = tt.load_library()
    n = (ctypes.c_int64 * 3)(8, 8, 8)
    s = (ctypes.c_int64 * 4)(1, 257, 2, 1)
    ptrs = (ctypes.c_void_p * 3)(*[c.data_ptr() for c in cores])
    rc = L.ttcross_sampled_error_noalloc(3, n, ctypes.byref(tt.make_generator(w["gen"])), ptrs, s,
                                         1000, ctypes.c_uint64(1), ctypes.c_void_p(out.data_ptr()),
                                         None)
    assert rc == tt.ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert np.isfinite(out.item())
