"""Thin ctypes binding of the C ABI in ``include/ttcross.h``.

Argument marshalling only: every step of the TT cross runs in the CUDA library
``_lib/libttcross.so``.  There is no CPU fallback -- if the library is missing
or no GPU is present, the calls raise.  PyTorch supplies the CUDA stream
(``torch.cuda.current_stream()``) and device buffers for device-side outputs.
"""
from __future__ import annotations

import ctypes as C
import json
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libttcross.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_ZERO_START, ERR_NONFINITE, ERR_DEVICE_TIMEOUT, ERR_CUDA, \
    NOT_CONVERGED = range(8)
STATUS_NAMES = {0: "OK", 1: "ERR_INVALID_ARG", 2: "ERR_OOM", 3: "ERR_ZERO_START",
                4: "ERR_NONFINITE", 5: "ERR_DEVICE_TIMEOUT", 6: "ERR_CUDA", 7: "NOT_CONVERGED"}
GEN_HILBERT, GEN_TT, GEN_MAXWELLIAN, GEN_MAXWELLIAN_XV, GEN_USER = 0, 1, 2, 3, 4
PREC_FP64, PREC_FP32, PREC_SPLIT, PREC_AUTO = 0, 1, 2, 3
PRECISIONS = {"fp64": PREC_FP64, "fp32": PREC_FP32, "split": PREC_SPLIT, "auto": PREC_AUTO}
RESIDUAL_RECOMPUTE, RESIDUAL_STORED = 0, 1
RESIDUALS = {"recompute": RESIDUAL_RECOMPUTE, "stored": RESIDUAL_STORED}

# every symbol include/ttcross.h declares
ABI_SYMBOLS = ("ttcross_default_options", "ttcross_create", "ttcross_run", "ttcross_run_batch",
               "ttcross_sync", "ttcross_get_ranks", "ttcross_get_cores", "ttcross_get_pivots",
               "ttcross_get_pivot_inverse", "ttcross_get_stats", "ttcross_destroy",
               "ttcross_sampled_error_noalloc", "ttcross_last_error_string",
               "ttcross_set_plan", "ttcross_autotune", "ttcross_rebuild_cores",
               "ttcross_check_tiles")


class TTCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Generator(C.Structure):
    _fields_ = [("kind", C.c_int32),
                ("tt_ranks", C.POINTER(C.c_int32)),
                ("tt_cores", C.POINTER(C.c_double)),
                ("dx", C.c_int32), ("dv", C.c_int32),
                ("a_rho", C.c_double), ("a_u", C.c_double), ("a_T", C.c_double),
                ("vmin", C.c_double), ("vmax", C.c_double),
                ("user_fn", C.c_void_p), ("user", C.c_void_p)]


# ttc_user_fn: (idx, count, values, user, stream)
USER_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p)


class _DeviceView:
    """A device buffer of the library seen by torch without a copy."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


def _user_callback(fn, d, errors):
    """ctypes callback around fn(idx, values): idx an int32 [count, d] and
    values a float64 [count] torch CUDA tensor over the library's buffers;
    fn fills values on torch's current stream, which is the run's stream.
    Exceptions are kept in ``errors`` (they cannot cross the C ABI)."""

    def cb(idx_ptr, count, val_ptr, user, stream):
        try:
            import torch
            st = torch.cuda.ExternalStream(stream) if stream else torch.cuda.current_stream()
            with torch.cuda.stream(st):
                idx = torch.as_tensor(_DeviceView(idx_ptr, (count, d), "<i4"), device="cuda")
                out = torch.as_tensor(_DeviceView(val_ptr, (count,), "<f8"), device="cuda")
                fn(idx, out)
        except BaseException as e:  # noqa: BLE001 - re-raised on the Python side
            errors.append(e)

    return USER_FN(cb)


class Options(C.Structure):
    _fields_ = [("max_rank", C.c_int32),
                ("bond_max_rank", C.POINTER(C.c_int32)),
                ("precision", C.c_int32),
                ("nsamples", C.c_int64),
                ("seed", C.c_uint64),
                ("max_refine", C.c_int32),
                ("topk", C.c_int32),
                ("host_loop", C.c_int32),
                ("grid_ctas", C.c_int32),
                ("wait_limit_s", C.c_double),
                ("residual", C.c_int32),
                ("screen_samples", C.c_int64),
                ("screen_seed", C.c_uint64),
                ("rook_rounds", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("sweeps", C.c_int64), ("entries_screened", C.c_int64),
                ("refinements", C.c_int64), ("tiles_refined", C.c_int64),
                ("unscreened_slots", C.c_int64),
                ("screen_fmas", C.c_int64), ("error_fmas", C.c_int64),
                ("tau", C.c_double), ("x_rms", C.c_double), ("err", C.c_double),
                ("device_ms", C.c_double), ("phase_ms", C.c_double * 6),
                ("status", C.c_int32),
                ("device_error_where", C.c_int32),
                ("entries_fresh", C.c_int64), ("stored_bytes", C.c_int64),
                ("rebuild_ms", C.c_double)]


_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH):
    """Load libttcross.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
        L = C.CDLL(path)
        P = C.c_void_p
        st = C.c_int
        L.ttcross_default_options.argtypes = [C.POINTER(Options)]
        L.ttcross_create.argtypes = [C.c_int, C.POINTER(C.c_int64), C.POINTER(Generator),
                                     C.POINTER(Options), C.POINTER(P)]
        L.ttcross_run.argtypes = [P, C.c_double, C.c_int, C.POINTER(C.c_int32), P]
        L.ttcross_run_batch.argtypes = [C.POINTER(P), C.c_int, C.POINTER(C.c_double),
                                        C.POINTER(C.c_int32), C.POINTER(P), P]
        L.ttcross_sync.argtypes = [P]
        L.ttcross_get_ranks.argtypes = [P, C.POINTER(C.c_int64)]
        L.ttcross_get_cores.argtypes = [P, C.c_int, P, C.c_int, P]
        L.ttcross_get_pivots.argtypes = [P, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.ttcross_get_pivot_inverse.argtypes = [P, C.c_int, C.POINTER(C.c_double)]
        L.ttcross_get_stats.argtypes = [P, C.POINTER(Stats)]
        L.ttcross_destroy.argtypes = [P]
        L.ttcross_sampled_error_noalloc.argtypes = [C.c_int, C.POINTER(C.c_int64),
                                                    C.POINTER(Generator), C.POINTER(P),
                                                    C.POINTER(C.c_int64), C.c_int64, C.c_uint64,
                                                    P, P]
        L.ttcross_set_plan.argtypes = [P, C.c_int32, C.c_int32]
        L.ttcross_rebuild_cores.argtypes = [P, P]
        L.ttcross_autotune.argtypes = [P, C.c_double, C.c_int, C.POINTER(C.c_int32), P,
                                       C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                       C.POINTER(C.c_double)]
        L.ttcross_check_tiles.argtypes = [C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                          C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                          C.POINTER(C.c_int32), C.c_int, C.c_int,
                                          C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                          C.POINTER(C.c_int64)]
        L.ttcross_last_error_string.restype = C.c_char_p
        for name in ABI_SYMBOLS:
            f = getattr(L, name)
            if name != "ttcross_last_error_string":
                f.restype = st
        _lib = L
        return L


def _check(rc: int, allow=(OK,)):
    if rc not in allow:
        msg = _lib.ttcross_last_error_string().decode(errors="replace") if _lib else ""
        raise TTCError(rc, msg)
    return rc


def _stream_handle(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def default_options() -> Options:
    L = load_library()
    o = Options()
    _check(L.ttcross_default_options(C.byref(o)))
    return o


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class TTCross:
    """One adaptive TT-cross instance on the current CUDA device.

    ``n``: mode sizes; ``gen``: generator dict as produced by
    :mod:`paper_2407_11290_gb300.workloads` (``{"kind": "hilbert"}``,
    ``{"kind": "tt", ...}``, ``{"kind": "maxwellian", ...}``).
    """

    def __init__(self, n, gen, max_rank: int = 64, precision="fp64", nsamples: int = 10**6,
                 seed: int = 20240715, max_refine: int = 6, topk: int = 8, host_loop: bool = False,
                 grid_ctas: int = 0, wait_limit_s: float = 2.0, bond_max_rank=None,
                 residual="recompute", screen_samples: int = 0, screen_seed: int = 20240715,
                 rook_rounds: int = 8):
        L = load_library()
        self._L = L
        self.n = np.ascontiguousarray(n, dtype=np.int64)
        self.d = int(self.n.size)
        o = default_options()
        o.max_rank = int(max_rank)
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        o.nsamples = int(nsamples)
        o.seed = int(seed)
        o.max_refine = int(max_refine)
        o.topk = int(topk)
        o.host_loop = 1 if host_loop else 0
        o.grid_ctas = int(grid_ctas)
        o.wait_limit_s = float(wait_limit_s)
        o.residual = RESIDUALS[residual] if isinstance(residual, str) else int(residual)
        o.screen_samples = int(screen_samples)
        o.screen_seed = int(screen_seed)
        o.rook_rounds = int(rook_rounds)
        keep = []
        if bond_max_rank is not None:
            bm = _i32(bond_max_rank)
            keep.append(bm)
            o.bond_max_rank = bm.ctypes.data_as(C.POINTER(C.c_int32))
        g = Generator()
        kind = gen["kind"]
        self._user_errors = []
        if kind == "hilbert":
            g.kind = GEN_HILBERT
        elif kind == "user":
            g.kind = GEN_USER
            cb = _user_callback(gen["fn"], self.d, self._user_errors)
            keep.append(cb)
            g.user_fn = C.cast(cb, C.c_void_p)
        elif kind == "tt":
            g.kind = GEN_TT
            ranks = _i32(gen["ranks"])
            cores = np.ascontiguousarray(np.concatenate(
                [np.asarray(c, dtype=np.float64).ravel() for c in gen["cores"]]))
            keep += [ranks, cores]
            g.tt_ranks = ranks.ctypes.data_as(C.POINTER(C.c_int32))
            g.tt_cores = cores.ctypes.data_as(C.POINTER(C.c_double))
        elif kind in ("maxwellian", "maxwellian_xv"):
            g.kind = GEN_MAXWELLIAN if kind == "maxwellian" else GEN_MAXWELLIAN_XV
            g.dx, g.dv = int(gen["dx"]), int(gen["dv"])
            g.a_rho, g.a_u, g.a_T = float(gen["a_rho"]), float(gen["a_u"]), float(gen["a_T"])
            g.vmin, g.vmax = float(gen["vmin"]), float(gen["vmax"])
        else:
            raise ValueError(f"unknown generator kind {kind!r}")
        h = C.c_void_p()
        _check(L.ttcross_create(self.d, self.n.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(g),
                                C.byref(o), C.byref(h)))
        self._h = h
        self._keep = keep  # the user callback must outlive the handle

    # ------------------------------------------------------------------
    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._L.ttcross_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def run(self, eps: float, max_rank: int = 0, subtensor_grid=None, stream=None):
        """Launch the cross (asynchronous); returns immediately."""
        grid = None
        if subtensor_grid is not None:
            grid = _i32(subtensor_grid)
            if grid.size != self.d:
                raise ValueError("subtensor_grid needs d entries")
        rc = self._L.ttcross_run(self._h, float(eps), int(max_rank),
                                 grid.ctypes.data_as(C.POINTER(C.c_int32)) if grid is not None
                                 else None, _stream_handle(stream))
        if self._user_errors:
            raise self._user_errors.pop(0)
        _check(rc)

    def rebuild_cores(self, stream=None):
        """Rebuild T_k (and the last core) from the pivot sets alone (Alg. 5)."""
        _check(self._L.ttcross_rebuild_cores(self._h, _stream_handle(stream)))

    def set_plan(self, tile_edge: int = 0, queue_split: int = 0):
        """Tile edge (0, 32, 64) and queue split (0, 1..7 eighths) of later runs."""
        _check(self._L.ttcross_set_plan(self._h, int(tile_edge), int(queue_split)))

    def autotune(self, eps: float, max_rank: int = 0, subtensor_grid=None, stream=None):
        """Measure the candidate plans on this instance and keep the fastest.
        Returns (tile_edge, queue_split, best_ms)."""
        grid = _i32(subtensor_grid) if subtensor_grid is not None else None
        te, qs, ms = C.c_int32(), C.c_int32(), C.c_double()
        _check(self._L.ttcross_autotune(self._h, float(eps), int(max_rank),
                                        grid.ctypes.data_as(C.POINTER(C.c_int32))
                                        if grid is not None else None,
                                        _stream_handle(stream), C.byref(te), C.byref(qs),
                                        C.byref(ms)))
        return te.value, qs.value, ms.value

    def sync(self, allow=(OK, NOT_CONVERGED)) -> int:
        return _check(self._L.ttcross_sync(self._h), allow)

    def ranks(self) -> np.ndarray:
        s = np.zeros(self.d + 1, np.int64)
        _check(self._L.ttcross_get_ranks(self._h, s.ctypes.data_as(C.POINTER(C.c_int64))))
        return s

    def core(self, k: int, device: bool = False, stream=None):
        """Core k (1-based) as [s_{k-1}, n_k, s_k]; a torch CUDA tensor if device."""
        s = self.ranks()
        shape = (int(s[k - 1]), int(self.n[k - 1]), int(s[k]))
        if device:
            import torch
            out = torch.empty(shape, dtype=torch.float64, device="cuda")
            _check(self._L.ttcross_get_cores(self._h, int(k), C.c_void_p(out.data_ptr()), 1,
                                             _stream_handle(stream)))
            return out
        out = np.zeros(shape, np.float64)
        _check(self._L.ttcross_get_cores(self._h, int(k), out.ctypes.data_as(C.c_void_p), 0,
                                         _stream_handle(stream)))
        return out

    def cores(self, stream=None):
        """Every core to host memory (one wait for the run)."""
        s = self.ranks()
        out = []
        for k in range(1, self.d + 1):
            c = np.zeros((int(s[k - 1]), int(self.n[k - 1]), int(s[k])), np.float64)
            _check(self._L.ttcross_get_cores(self._h, int(k), c.ctypes.data_as(C.c_void_p), 0,
                                             _stream_handle(stream)))
            out.append(c)
        return out

    def pivots(self, k: int):
        """(I_{<=k}, J_{>k}) of bond k (1-based) as int32 arrays."""
        r = int(self.ranks()[k])
        I = np.zeros((r, k), np.int32)
        J = np.zeros((r, self.d - k), np.int32)
        _check(self._L.ttcross_get_pivots(self._h, int(k), I.ctypes.data_as(C.POINTER(C.c_int32)),
                                          J.ctypes.data_as(C.POINTER(C.c_int32))))
        return I, J

    def pivot_inverse(self, k: int) -> np.ndarray:
        r = int(self.ranks()[k])
        U = np.zeros((r, r), np.float64)
        _check(self._L.ttcross_get_pivot_inverse(self._h, int(k),
                                                 U.ctypes.data_as(C.POINTER(C.c_double))))
        return U

    def stats(self) -> dict:
        st = Stats()
        _check(self._L.ttcross_get_stats(self._h, C.byref(st)))
        out = {f: getattr(st, f) for f, _ in Stats._fields_}
        out["phase_ms"] = dict(zip(("init", "screen", "decide", "update", "verify", "refine"),
                                   list(st.phase_ms)))
        return out


def make_generator(gen):
    """ctypes Generator for a Hilbert / Maxwellian generator dict."""
    g = Generator()
    if gen["kind"] == "hilbert":
        g.kind = GEN_HILBERT
    elif gen["kind"] in ("maxwellian", "maxwellian_xv"):
        g.kind = GEN_MAXWELLIAN if gen["kind"] == "maxwellian" else GEN_MAXWELLIAN_XV
        g.dx, g.dv = int(gen["dx"]), int(gen["dv"])
        g.a_rho, g.a_u, g.a_T = float(gen["a_rho"]), float(gen["a_u"]), float(gen["a_T"])
        g.vmin, g.vmax = float(gen["vmin"]), float(gen["vmax"])
    else:
        g.kind = GEN_TT
    return g


def sampled_error_noalloc(n, gen, cores, nsamples: int, seed: int, out, stream=None):
    """Enqueue ttcross_sampled_error_noalloc: ``cores`` are CUDA float64 torch
    tensors [s_{m-1}, n_m, s_m]; the error is written to the CUDA float64
    tensor ``out`` (one element).  Allocates nothing.

    The C side sees only the core pointers and the sizes s, so every core's
    shape, dtype, device and layout is checked here: a permuted view or a
    float32 core would make the kernel read past the end of the core."""
    L = load_library()
    n = np.ascontiguousarray(n, dtype=np.int64)
    d = int(n.size)

    def reject(msg):
        raise TTCError(ERR_INVALID_ARG, msg)

    if len(cores) != d:
        reject(f"{len(cores)} cores for a {d}-way tensor")
    s = [1]
    for m, c in enumerate(cores):
        if getattr(c, "dtype", None) is None or str(c.dtype) != "torch.float64":
            reject(f"core {m + 1} is not a float64 tensor")
        if not getattr(c, "is_cuda", False):
            reject(f"core {m + 1} is not in device memory")
        if c.dim() != 3 or not c.is_contiguous():
            reject(f"core {m + 1} must be a contiguous [s, n, s] tensor")
        if int(c.shape[0]) != s[-1] or int(c.shape[1]) != int(n[m]):
            reject(f"core {m + 1} has shape {tuple(c.shape)}, expected ({s[-1]}, {int(n[m])}, *)")
        s.append(int(c.shape[2]))
    if s[-1] != 1:
        reject("the last core must end with size 1")
    if (getattr(out, "dtype", None) is None or str(out.dtype) != "torch.float64"
            or not getattr(out, "is_cuda", False) or out.numel() < 1):
        reject("out must be a float64 device tensor with at least one element")
    s = np.ascontiguousarray(s, dtype=np.int64)
    ptrs = (C.c_void_p * d)(*[c.data_ptr() for c in cores])
    g = make_generator(gen)
    _check(L.ttcross_sampled_error_noalloc(d, n.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(g),
                                           ptrs, s.ctypes.data_as(C.POINTER(C.c_int64)),
                                           int(nsamples), C.c_uint64(seed),
                                           C.c_void_p(out.data_ptr()), _stream_handle(stream)))


def probe_fma_peak(fp64: bool = True, blocks_per_sm: int = 4, iters: int = 1 << 16):
    """Measured FMA/s of the FP64 (or FP32) pipe on the current device."""
    L = load_library()
    f = L.ttcross_probe_fma_peak
    f.argtypes = [C.c_int, C.c_int, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    f.restype = C.c_int
    rate, ms = C.c_double(), C.c_double()
    _check(f(1 if fp64 else 0, int(blocks_per_sm), int(iters), C.byref(rate), C.byref(ms)))
    return rate.value, ms.value


def probe_fp64_chain(chain_warps: int = 1, active_lanes: int = 32, busy_warps: int = 0,
                     iters: int = 1 << 14) -> float:
    """Clock cycles per dependent FP64 FMA of one warp on one SM, with
    ``chain_warps`` such warps and ``busy_warps`` warps of independent FMAs."""
    L = load_library()
    f = L.ttcross_probe_fp64_chain
    f.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int64, C.POINTER(C.c_double)]
    f.restype = C.c_int
    cyc = C.c_double()
    _check(f(int(chain_warps), int(active_lanes), int(busy_warps), int(iters), C.byref(cyc)))
    return cyc.value


def probe_fp64_ilp(warps: int = 1, chains: int = 4, iters: int = 1 << 12) -> float:
    """Clock cycles per FP64 FMA instruction of one warp running ``chains``
    independent chains, with ``warps`` such warps on one SM."""
    L = load_library()
    f = L.ttcross_probe_fp64_ilp
    f.argtypes = [C.c_int, C.c_int, C.c_int64, C.POINTER(C.c_double)]
    f.restype = C.c_int
    cyc = C.c_double()
    _check(f(int(warps), int(chains), int(iters), C.byref(cyc)))
    return cyc.value


def check_tiles(n, ranks, caps, grid=None, tile_edge: int = 64, stored: bool = False,
                stored_ranks=None):
    """ttcross_check_tiles: the kernels' tile arithmetic replayed on the host
    for bond ranks ``ranks`` (bond k = ranks[k-1]); ``stored_ranks`` (the
    ranks the stored residual was written at) adds the carried-tile check.
    Returns (tiles per bond, candidate slots per bond at the rank caps
    ``caps``, violations).  Needs no GPU."""
    L = load_library()
    d = len(n)
    nn = np.ascontiguousarray(n, dtype=np.int64)
    rr, cc = _i32(ranks), _i32(caps)
    rs = _i32(stored_ranks) if stored_ranks is not None else None
    g = _i32(grid) if grid is not None else None
    tiles = np.zeros(d - 1, dtype=np.int64)
    cap = np.zeros(d - 1, dtype=np.int64)
    bad = C.c_int64(0)
    p64 = C.POINTER(C.c_int64)
    p32 = C.POINTER(C.c_int32)
    _check(L.ttcross_check_tiles(d, nn.ctypes.data_as(p64), rr.ctypes.data_as(p32),
                                 cc.ctypes.data_as(p32),
                                 rs.ctypes.data_as(p32) if rs is not None else None,
                                 g.ctypes.data_as(p32) if g is not None else None,
                                 int(tile_edge), int(bool(stored)),
                                 tiles.ctypes.data_as(p64), cap.ctypes.data_as(p64),
                                 C.byref(bad)))
    return tiles, cap, int(bad.value)


def run_batch(crosses, eps, max_rank=None, grids=None, stream=None):
    """Run several instances in one persistent launch (asynchronous).
    ``grids``: None, or one subtensor grid (or None) per instance."""
    L = load_library()
    cnt = len(crosses)
    hs = (C.c_void_p * cnt)(*[c.handle.value for c in crosses])
    e = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, np.float64), (cnt,)))
    mr = None
    if max_rank is not None:
        mr = np.ascontiguousarray(np.broadcast_to(np.asarray(max_rank, np.int32), (cnt,)))
    gp = None
    keep = []
    if grids is not None:
        if len(grids) != cnt:
            raise ValueError("grids needs one entry per instance")
        gp = (C.c_void_p * cnt)()
        for i, (c, g) in enumerate(zip(crosses, grids)):
            if g is None:
                continue
            a = _i32(g)
            if a.size != c.d:
                raise ValueError(f"grid {i} needs {c.d} entries")
            keep.append(a)
            gp[i] = a.ctypes.data
    _check(L.ttcross_run_batch(hs, cnt, e.ctypes.data_as(C.POINTER(C.c_double)),
                               mr.ctypes.data_as(C.POINTER(C.c_int32)) if mr is not None else None,
                               gp, _stream_handle(stream)))


def plan_cache_path() -> str:
    """The autotuner's cache of plans per shape class (TTCROSS_PLAN_CACHE, else
    ~/.cache/ttcross_gb300/plans.json)."""
    return os.environ.get("TTCROSS_PLAN_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "ttcross_gb300",
                                       "plans.json"))


def shape_class(tc, eps, max_rank, subtensor_grid, precision, residual) -> str:
    """Key of a plan: mode sizes, the rank cap, eps, grid, precision, form."""
    grid = None if subtensor_grid is None else [int(v) for v in subtensor_grid]
    return json.dumps({"n": [int(v) for v in tc.n], "max_rank": int(max_rank), "eps": float(eps),
                       "grid": grid, "precision": str(precision), "residual": str(residual)},
                      sort_keys=True)


def tuned_plan(tc, eps, max_rank, subtensor_grid, precision, residual, stream=None):
    """The plan of this shape class from the cache, else measured by the
    library's autotuner and cached.  Returns (tile_edge, queue_split, source)."""
    path = plan_cache_path()
    key = shape_class(tc, eps, max_rank, subtensor_grid, precision, residual)
    cache = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        te, qs = cache[key]["tile_edge"], cache[key]["queue_split"]
        tc.set_plan(te, qs)
        return te, qs, "cache"
    te, qs, ms = tc.autotune(eps, max_rank, subtensor_grid, stream)
    cache[key] = {"tile_edge": te, "queue_split": qs, "ms": ms}
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path + ".tmp", "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(path + ".tmp", path)
    except OSError:
        pass
    return te, qs, "measured"
