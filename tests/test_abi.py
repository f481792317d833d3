"""The C-ABI library builds, loads and exports every symbol include/ttcross.h
declares (no compute calls: CPU only)."""
import ctypes
import os
import re

import pytest

from paper_2407_11290_gb300 import build as B
from paper_2407_11290_gb300 import ttcross

HEADER = os.path.join(B.INCLUDE, "ttcross.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ttcross_\w+)\s*\(", text)))


def test_library_exports_the_probe_symbols():
    text = open(os.path.join(B.INCLUDE, "ttcross_probe.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = sorted(set(re.findall(r"\b(ttcross_\w+)\s*\(", text)))
    assert names == ["ttcross_probe_fma_peak", "ttcross_probe_fp64_chain",
                     "ttcross_probe_fp64_ilp"]
    L = ctypes.CDLL(B.build())
    for name in names:
        assert hasattr(L, name), name


def test_library_builds_and_exports_header_symbols():
    lib = B.build()
    L = ctypes.CDLL(lib)
    names = declared_functions()
    assert names, "no declarations found"
    for name in names:
        assert hasattr(L, name), name
    assert sorted(ttcross.ABI_SYMBOLS) == names


C_CLIENT = r"""
#include <stdio.h>
#include "ttcross.h"
#include "ttcross_probe.h"
int main(void) {
  ttc_options o;
  if (ttcross_default_options(&o) != TTC_OK || o.max_rank != 64) return 1;
  const int64_t n[3] = {100, 100, 100};
  const int32_t r[2] = {5, 7}, caps[2] = {8, 8};
  int64_t tiles[2], cap[2], bad = -1;
  if (ttcross_check_tiles(3, n, r, caps, NULL, NULL, 64, 0, tiles, cap, &bad) != TTC_OK) return 2;
  printf("%lld %lld %lld\n", (long long)tiles[0], (long long)tiles[1], (long long)bad);
  return 0;
}
"""


def test_plain_c_client(tmp_path):
    """The boundary is plain C: a C99 program (-pedantic -Werror) includes
    both headers, links the library and calls its host-side entry points."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib = B.build()
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", B.INCLUDE,
                    str(src), "-o", str(exe), os.path.abspath(lib),
                    "-Wl,-rpath," + os.path.dirname(os.path.abspath(lib))], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    assert out.stdout.split() == ["22", "16", "0"]


def test_default_options_without_gpu():
    o = ttcross.default_options()
    assert o.max_rank == 64 and o.nsamples == 10**6 and o.seed == 20240715
    assert o.wait_limit_s == 2.0 and o.precision == ttcross.PREC_FP64
    assert o.residual == ttcross.RESIDUAL_RECOMPUTE


def test_missing_library_raises(tmp_path):
    """No CPU fallback: without the built library the binding raises."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("ttcross_copy", ttcross.__file__)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with pytest.raises(RuntimeError, match="not built"):
        mod.load_library(str(tmp_path / "libttcross.so"))


def test_create_fails_loudly_without_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(ttcross.TTCError):
        ttcross.TTCross([4, 4], {"kind": "hilbert"}, max_rank=4)


def test_invalid_arguments_rejected_on_host():
    L = ttcross.load_library()
    h = ctypes.c_void_p()
    n = (ctypes.c_int64 * 1)(4)
    g = ttcross.Generator()
    g.kind = ttcross.GEN_HILBERT
    rc = L.ttcross_create(1, n, ctypes.byref(g), None, ctypes.byref(h))
    assert rc == ttcross.ERR_INVALID_ARG
    assert b"d=1" in L.ttcross_last_error_string()
    assert L.ttcross_run(None, 1e-3, 0, None, None) == ttcross.ERR_INVALID_ARG


def test_stored_form_option_checked_on_host():
    L = ttcross.load_library()
    h = ctypes.c_void_p()
    n = (ctypes.c_int64 * 3)(8, 8, 8)
    g = ttcross.Generator()
    g.kind = ttcross.GEN_HILBERT
    o = ttcross.default_options()
    o.residual = 5
    assert L.ttcross_create(3, n, ctypes.byref(g), ctypes.byref(o), ctypes.byref(h)) == \
        ttcross.ERR_INVALID_ARG
    assert b"residual form" in L.ttcross_last_error_string()



def test_run_batch_checks_arguments_on_host():
    L = ttcross.load_library()
    eps = (ctypes.c_double * 1)(1e-6)
    assert L.ttcross_run_batch(None, 1, eps, None, None, None) == ttcross.ERR_INVALID_ARG
    hs = (ctypes.c_void_p * 1)(None)
    assert L.ttcross_run_batch(hs, 1, eps, None, None, None) == ttcross.ERR_INVALID_ARG
    assert b"null handle" in L.ttcross_last_error_string()


def test_noalloc_wrapper_rejects_bad_cores_before_the_call():
    """The C side sees only core pointers and sizes: the wrapper checks every
    core's rank, shape, dtype, layout and device before calling it."""
    import torch
    gen = {"kind": "hilbert"}
    n = [4, 5, 6]
    good = [torch.zeros(1, 4, 2, dtype=torch.float64), torch.zeros(2, 5, 3, dtype=torch.float64),
            torch.zeros(3, 6, 1, dtype=torch.float64)]
    out = torch.zeros(1, dtype=torch.float64)
    cases = [good[:2],                                                      # too few cores
             [good[0], torch.zeros(3, 5, 3, dtype=torch.float64), good[2]],  # s mismatch
             [good[0], torch.zeros(2, 4, 3, dtype=torch.float64), good[2]],  # n mismatch
             [good[0], good[1].float(), good[2]],                           # float32
             [good[0], good[1].transpose(0, 2), good[2]],                   # permuted view
             good]                                                          # host tensors
    for cores in cases:
        with pytest.raises(ttcross.TTCError) as e:
            ttcross.sampled_error_noalloc(n, gen, cores, 100, 1, out)
        assert e.value.status == ttcross.ERR_INVALID_ARG


def test_sampled_screen_options_checked_on_host():
    """The Python options struct matches the C one (defaults read back), and
    a sampled screen with the stored form or a mixed precision is refused
    before any device call."""
    o = ttcross.default_options()
    assert o.screen_samples == 0 and o.screen_seed == 20240715 and o.rook_rounds == 8
    L = ttcross.load_library()
    h = ctypes.c_void_p()
    n = (ctypes.c_int64 * 3)(8, 8, 8)
    g = ttcross.Generator()
    g.kind = ttcross.GEN_HILBERT
    o.screen_samples = 100
    o.residual = ttcross.RESIDUAL_STORED
    assert L.ttcross_create(3, n, ctypes.byref(g), ctypes.byref(o), ctypes.byref(h)) == \
        ttcross.ERR_INVALID_ARG
    assert b"sampled screen" in L.ttcross_last_error_string()
    o.residual = ttcross.RESIDUAL_RECOMPUTE
    o.rook_rounds = 65
    assert L.ttcross_create(3, n, ctypes.byref(g), ctypes.byref(o), ctypes.byref(h)) == \
        ttcross.ERR_INVALID_ARG


def test_user_generator_needs_a_callback():
    L = ttcross.load_library()
    h = ctypes.c_void_p()
    n = (ctypes.c_int64 * 3)(8, 8, 8)
    g = ttcross.Generator()
    g.kind = ttcross.GEN_USER
    assert L.ttcross_create(3, n, ctypes.byref(g), None, ctypes.byref(h)) == \
        ttcross.ERR_INVALID_ARG
    assert b"callback" in L.ttcross_last_error_string()


def test_fp64_chain_probe_rejects_bad_arguments_on_the_host():
    """The latency probe checks its arguments before any device call, so the
    refusals need no GPU."""
    for args in [(0, 32, 0), (1, 0, 0), (1, 33, 0), (1, 32, -1), (20, 32, 13)]:
        with pytest.raises(ttcross.TTCError):
            ttcross.probe_fp64_chain(*args)
    with pytest.raises(ttcross.TTCError):
        ttcross.probe_fp64_chain(1, 32, 0, iters=0)
    for args in [(0, 4), (33, 4), (1, 3), (1, 16)]:
        with pytest.raises(ttcross.TTCError):
            ttcross.probe_fp64_ilp(*args)
