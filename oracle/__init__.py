"""CPU FP64 oracle for the adaptive TT cross (arXiv 2407.11290).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the GPU library (``paper_2407_11290_gb300``) and never imports it.

The C source (``ttc_oracle.c``) is the oracle proper: plain loops in binary64
with explicit ``fma`` and no contraction, following Alg. 1-4 and
eqs. aca_approx_T / aca_approx_T_sub / ttcross_build of the paper.  This module
only compiles it and marshals arguments through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ttc_oracle.c")
_LIB = os.path.join(_HERE, "libttc_oracle.so")
_lock = threading.Lock()
_lib = None

GEN_HILBERT, GEN_TT, GEN_MAXWELLIAN, GEN_MAXWELLIAN_XV = 0, 1, 2, 3
OK, ERR_INVALID_ARG, ERR_OOM, ERR_ZERO_START, ERR_NONFINITE, NOT_CONVERGED = 0, 1, 2, 3, 4, 7


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FP contraction, OpenMP screen)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB) >= os.path.getmtime(os.path.join(_HERE, "ttc_oracle.h"))):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Gen(C.Structure):
    _fields_ = [("kind", C.c_int),
                ("tt_ranks", C.POINTER(C.c_int32)),
                ("tt_cores", C.POINTER(C.c_double)),
                ("dx", C.c_int32), ("dv", C.c_int32),
                ("a_rho", C.c_double), ("a_u", C.c_double), ("a_T", C.c_double),
                ("vmin", C.c_double), ("vmax", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("sweeps", C.c_int64), ("entries_screened", C.c_int64),
                ("refinements", C.c_int64), ("tau", C.c_double),
                ("x_rms", C.c_double), ("err", C.c_double), ("status", C.c_int32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            P = C.c_void_p
            i64p = C.POINTER(C.c_int64)
            i32p = C.POINTER(C.c_int32)
            f64p = C.POINTER(C.c_double)
            L.orc_create.restype = P
            L.orc_create.argtypes = [C.c_int, i64p, C.POINTER(_Gen), i32p, C.c_int]
            L.orc_destroy.argtypes = [P]
            L.orc_entry.restype = C.c_double
            L.orc_entry.argtypes = [P, i32p]
            L.orc_init.argtypes = [P]
            L.orc_init_at.argtypes = [P, i32p]
            L.orc_sample_scan.argtypes = [P, C.c_int64, C.c_uint64, f64p, i32p]
            L.orc_screen.argtypes = [P, f64p, i64p, i32p, i32p, f64p]
            L.orc_residual.restype = C.c_double
            L.orc_residual.argtypes = [P, C.c_int, C.c_int64, C.c_int64]
            L.orc_apply.argtypes = [P, i32p, i32p, i32p]
            L.orc_set_stored.argtypes = [P, C.c_int]
            L.orc_set_sampled.argtypes = [P, C.c_int64, C.c_uint64, C.c_int]
            L.orc_last_screened.restype = C.c_int64
            L.orc_last_screened.argtypes = [P]
            L.orc_rook_moves.restype = C.c_int64
            L.orc_rook_moves.argtypes = [P]
            L.orc_stored_residual.restype = C.c_double
            L.orc_stored_residual.argtypes = [P, C.c_int, C.c_int64, C.c_int64]
            L.orc_E.argtypes = [P, C.c_int, f64p]
            L.orc_stored_extent.argtypes = [P, C.c_int, i64p, i64p]
            L.orc_run.argtypes = [P, C.c_double, C.c_int64, C.c_uint64, C.c_int, C.POINTER(Stats)]
            L.orc_sampled_error.argtypes = [P, C.c_int64, C.c_uint64, f64p]
            L.orc_sample_rms.argtypes = [P, C.c_int64, C.c_uint64, f64p]
            L.orc_sample_indices.argtypes = [C.c_int, i64p, C.c_int64, C.c_uint64, i32p]
            L.orc_tt_eval.restype = C.c_double
            L.orc_tt_eval.argtypes = [P, i32p]
            L.orc_ranks.argtypes = [P, i32p]
            L.orc_dims.argtypes = [P, C.c_int, i64p, i64p]
            L.orc_pivots.argtypes = [P, C.c_int, i32p, i32p]
            L.orc_pivot_coords.argtypes = [P, C.c_int, i32p, i32p]
            for f in (L.orc_T, L.orc_R, L.orc_U, L.orc_core):
                f.argtypes = [P, C.c_int, f64p]
            L.orc_core_size.restype = C.c_int64
            L.orc_core_size.argtypes = [P, C.c_int]
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


class Oracle:
    """One adaptive TT cross instance evaluated on the CPU.

    ``gen`` is a dict: ``{"kind": "hilbert"}``, ``{"kind": "tt", "ranks": [...],
    "cores": [core_0, ...]}`` (core m shaped ``[rho_m, n_m, rho_{m+1}]``) or
    ``{"kind": "maxwellian", "dx":..., "dv":..., "a_rho":..., "a_u":..., "a_T":...,
    "vmin":..., "vmax":...}``.
    """

    def __init__(self, n, gen, max_rank, nthreads: int = 1, stored: bool = False):
        L = lib()
        self.n = np.ascontiguousarray(n, dtype=np.int64)
        self.d = int(self.n.size)
        mr = np.broadcast_to(np.asarray(max_rank, dtype=np.int32), (self.d - 1,))
        self.maxr = np.ascontiguousarray(mr, dtype=np.int32)
        g = _Gen()
        kind = gen["kind"]
        self._keep = []
        if kind == "hilbert":
            g.kind = GEN_HILBERT
        elif kind == "tt":
            g.kind = GEN_TT
            ranks = np.ascontiguousarray(gen["ranks"], dtype=np.int32)
            cores = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.float64).ravel()
                                                         for c in gen["cores"]]))
            self._keep += [ranks, cores]
            g.tt_ranks = _p(ranks, C.c_int32)
            g.tt_cores = _p(cores, C.c_double)
        elif kind in ("maxwellian", "maxwellian_xv"):
            g.kind = GEN_MAXWELLIAN if kind == "maxwellian" else GEN_MAXWELLIAN_XV
            g.dx, g.dv = int(gen["dx"]), int(gen["dv"])
            g.a_rho, g.a_u, g.a_T = float(gen["a_rho"]), float(gen["a_u"]), float(gen["a_T"])
            g.vmin, g.vmax = float(gen["vmin"]), float(gen["vmax"])
        else:
            raise ValueError(f"unknown generator kind {kind!r}")
        self._h = L.orc_create(self.d, _p(self.n, C.c_int64), C.byref(g), _p(self.maxr, C.c_int32),
                               int(nthreads))
        if not self._h:
            raise ValueError("orc_create rejected the arguments")
        self._L = L
        self.stored = bool(stored)
        if stored and L.orc_set_stored(self._h, 1):
            raise MemoryError("orc_set_stored: no memory for the stored residuals")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_destroy(h)
            self._h = None

    # --- entries -----------------------------------------------------------
    def entry(self, idx) -> float:
        a = np.ascontiguousarray(idx, dtype=np.int32)
        return float(self._L.orc_entry(self._h, _p(a, C.c_int32)))

    def tt_eval(self, idx) -> float:
        a = np.ascontiguousarray(idx, dtype=np.int32)
        return float(self._L.orc_tt_eval(self._h, _p(a, C.c_int32)))

    # --- steps -------------------------------------------------------------
    def init(self) -> int:
        return int(self._L.orc_init(self._h))

    def init_at(self, start) -> int:
        a = np.ascontiguousarray(start, dtype=np.int32)
        return int(self._L.orc_init_at(self._h, _p(a, C.c_int32)))

    def sample_scan(self, nsamples: int = 10**6, seed: int = 20240715):
        """(rms of X over the samples, start pivot multi-index)."""
        rms = C.c_double()
        start = np.zeros(self.d, np.int32)
        rc = self._L.orc_sample_scan(self._h, int(nsamples), C.c_uint64(seed), C.byref(rms),
                                     _p(start, C.c_int32))
        if rc:
            raise RuntimeError(f"orc_sample_scan -> {rc}")
        return rms.value, start

    def screen(self):
        nb = self.d - 1
        best = np.zeros(nb); lin = np.zeros(nb, np.int64)
        row = np.zeros(nb, np.int32); col = np.zeros(nb, np.int32); mx = np.zeros(nb)
        rc = self._L.orc_screen(self._h, _p(best, C.c_double), _p(lin, C.c_int64),
                                _p(row, C.c_int32), _p(col, C.c_int32), _p(mx, C.c_double))
        return rc, dict(best=best, lin=lin, row=row, col=col, maxabs=mx)

    def residual(self, b, a, c) -> float:
        return float(self._L.orc_residual(self._h, int(b), int(a), int(c)))

    def stored_residual(self, b, a, c) -> float:
        """Stored-residual form: the kept E(a, c) of bond b (NaN if none)."""
        return float(self._L.orc_stored_residual(self._h, int(b), int(a), int(c)))

    def stored_block(self, b) -> np.ndarray:
        """Stored-residual form: E of bond b over the superblock of the last
        screen, [rows, cols]."""
        rows, cols = C.c_int64(), C.c_int64()
        self._L.orc_stored_extent(self._h, int(b), C.byref(rows), C.byref(cols))
        out = np.zeros((rows.value, cols.value))
        self._L.orc_E(self._h, int(b), _p(out, C.c_double))
        return out

    def set_sampled(self, nl: int, seed: int = 20240715, max_rook: int = 8):
        """Alg. 1 with a random sample set of nl entries per superblock and up
        to max_rook rounds of row / column refinement (nl = 0: exhaustive)."""
        rc = self._L.orc_set_sampled(self._h, int(nl), C.c_uint64(seed), int(max_rook))
        if rc:
            raise ValueError(f"orc_set_sampled -> {rc}")

    def last_screened(self) -> int:
        return int(self._L.orc_last_screened(self._h))

    def rook_moves(self) -> int:
        return int(self._L.orc_rook_moves(self._h))

    def apply(self, add, row, col) -> int:
        add = np.ascontiguousarray(add, dtype=np.int32)
        row = np.ascontiguousarray(row, dtype=np.int32)
        col = np.ascontiguousarray(col, dtype=np.int32)
        return int(self._L.orc_apply(self._h, _p(add, C.c_int32), _p(row, C.c_int32),
                                     _p(col, C.c_int32)))

    def run(self, eps: float, nsamples: int = 10**6, seed: int = 20240715, max_refine: int = 6):
        st = Stats()
        rc = self._L.orc_run(self._h, float(eps), int(nsamples), C.c_uint64(seed), int(max_refine),
                             C.byref(st))
        return int(rc), {f: getattr(st, f) for f, _ in Stats._fields_}

    def sampled_error(self, nsamples: int = 10**6, seed: int = 20240715) -> float:
        e = C.c_double()
        rc = self._L.orc_sampled_error(self._h, int(nsamples), C.c_uint64(seed), C.byref(e))
        if rc:
            raise RuntimeError(f"orc_sampled_error -> {rc}")
        return e.value

    # --- state ------------------------------------------------------------
    def ranks(self) -> np.ndarray:
        r = np.zeros(self.d - 1, np.int32)
        self._L.orc_ranks(self._h, _p(r, C.c_int32))
        return r

    def dims(self, b):
        rows, cols = C.c_int64(), C.c_int64()
        self._L.orc_dims(self._h, int(b), C.byref(rows), C.byref(cols))
        return rows.value, cols.value

    def pivots(self, b):
        r = int(self.ranks()[b])
        I = np.zeros((r, b + 1), np.int32)
        J = np.zeros((r, self.d - 1 - b), np.int32)
        self._L.orc_pivots(self._h, int(b), _p(I, C.c_int32), _p(J, C.c_int32))
        return I, J

    def pivot_coords(self, b):
        r = int(self.ranks()[b])
        pr = np.zeros(r, np.int32); pc = np.zeros(r, np.int32)
        self._L.orc_pivot_coords(self._h, int(b), _p(pr, C.c_int32), _p(pc, C.c_int32))
        return pr, pc

    def T(self, b):
        rows, _ = self.dims(b)
        r = int(self.ranks()[b])
        out = np.zeros((rows, r))
        self._L.orc_T(self._h, int(b), _p(out, C.c_double))
        return out

    def R(self, b):
        _, cols = self.dims(b)
        r = int(self.ranks()[b])
        out = np.zeros((r, cols))
        self._L.orc_R(self._h, int(b), _p(out, C.c_double))
        return out

    def U(self, b):
        r = int(self.ranks()[b])
        out = np.zeros((r, r))
        self._L.orc_U(self._h, int(b), _p(out, C.c_double))
        return out

    def cores(self):
        rk = self.ranks()
        out = []
        for m in range(self.d):
            sl = 1 if m == 0 else int(rk[m - 1])
            sr = 1 if m == self.d - 1 else int(rk[m])
            buf = np.zeros(sl * int(self.n[m]) * sr)
            self._L.orc_core(self._h, m, _p(buf, C.c_double))
            out.append(buf.reshape(sl, int(self.n[m]), sr))
        return out


def sample_indices(n, nsamples: int, seed: int = 20240715) -> np.ndarray:
    """The multi-indices the sampled error uses (SplitMix64 counter form)."""
    L = lib()
    n = np.ascontiguousarray(n, dtype=np.int64)
    out = np.zeros((nsamples, n.size), np.int32)
    L.orc_sample_indices(int(n.size), _p(n, C.c_int64), int(nsamples), C.c_uint64(seed),
                         _p(out, C.c_int32))
    return out
