"""Thin ctypes binding of libmg.so (C ABI in include/mg.h).

Argument marshalling only: every step of assembly, compression and solving
runs in the CUDA library.  Loading fails loudly if the library is missing;
there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import inputs as _inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmg.so")

MG_OK, MG_ERR_INVALID, MG_ERR_OOM, MG_ERR_CUDA, MG_ERR_TIMEOUT = 0, 1, 2, 3, 4
MG_ERR_DIVERGED, MG_ERR_NOT_CONVERGED, MG_ERR_PENDING, MG_ERR_CANCELLED, MG_ERR_INJECTED = 5, 6, 7, 8, 9
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CUDA", 4: "TIMEOUT", 5: "DIVERGED",
                6: "NOT_CONVERGED", 7: "PENDING", 8: "CANCELLED", 9: "INJECTED"}

PATH_FP64_PLAIN, PATH_FP64_DELAYED, PATH_MIXED_DELAYED, PATH_MIXED_PLAIN = 0, 1, 2, 3
OUTER_FCG, OUTER_RICHARDSON = 0, 1
CYCLE_V, CYCLE_ADDITIVE, CYCLE_ADAFAC_PI, CYCLE_ADAFAC_JAC = 0, 1, 2, 3
MAX_MODES, MAX_BOXES = 32, 64


class mg_eps_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_modes", ctypes.c_int32), ("n_boxes", ctypes.c_int32),
                ("pad0", ctypes.c_int32), ("v_out", ctypes.c_double), ("v_in", ctypes.c_double),
                ("center", ctypes.c_double * 3), ("radius", ctypes.c_double), ("sigma", ctypes.c_double),
                ("theta", ctypes.c_double), ("jump_x", ctypes.c_double), ("jump_factor", ctypes.c_double),
                ("k", (ctypes.c_int32 * 3) * MAX_MODES), ("phase", ctypes.c_double * MAX_MODES),
                ("box_lo", (ctypes.c_double * 3) * MAX_BOXES), ("box_hi", (ctypes.c_double * 3) * MAX_BOXES)]


class mg_problem_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n_cells", ctypes.c_int32), ("eps", mg_eps_desc),
                ("f_const", ctypes.c_double), ("path", ctypes.c_int32), ("outer", ctypes.c_int32),
                ("s_schedule", ctypes.c_int32 * 8), ("n_s", ctypes.c_int32), ("compress_tau", ctypes.c_double),
                ("omega", ctypes.c_double), ("nu_pre", ctypes.c_int32), ("nu_post", ctypes.c_int32),
                ("rtol", ctypes.c_double), ("max_cycles", ctypes.c_int32), ("chunks", ctypes.c_int32),
                ("u0", ctypes.POINTER(ctypes.c_double)), ("adapt_C", ctypes.c_double), ("cycle", ctypes.c_int32),
                ("adapt_keep", ctypes.c_int32), ("coarse_tau", ctypes.c_double)]


class mg_solve_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("cycles", ctypes.c_int32), ("publishes", ctypes.c_int32),
                ("final_s", ctypes.c_int32), ("rel_residual", ctypes.c_double), ("time_ms", ctypes.c_double),
                ("assembly_ms", ctypes.c_double), ("cells_by_class", ctypes.c_int64 * 4),
                ("payload_bytes", ctypes.c_int64)]


class mg_trace_entry(ctypes.Structure):
    _fields_ = [("cycle", ctypes.c_int32), ("pending_jobs", ctypes.c_int32), ("publishes", ctypes.c_int32),
                ("restarted", ctypes.c_int32), ("rel_residual_est", ctypes.c_double), ("time_ms", ctypes.c_double)]


class mg_paper_format_stats(ctypes.Structure):
    _fields_ = [("cells_by_p3", ctypes.c_int64 * 9), ("bytes_full", ctypes.c_double), ("bytes_paper", ctypes.c_double),
                ("compression", ctypes.c_double), ("max_abs_error", ctypes.c_double)]


class mg_server_desc(ctypes.Structure):
    _fields_ = [("max_active", ctypes.c_int32), ("use_graphs", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_double), ("inject_fail_every", ctypes.c_int32),
                ("pad0", ctypes.c_int32)]


class mg_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("cycles", ctypes.c_int32), ("publishes", ctypes.c_int32),
                ("pad0", ctypes.c_int32), ("rel_residual", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("total_ms", ctypes.c_double)]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libmg.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        st = ctypes.c_int
        sig = {
            "mg_create_problem": (st, [ctypes.POINTER(mg_problem_desc), _VP, ctypes.POINTER(_VP)]),
            "mg_destroy_problem": (st, [_VP]),
            "mg_assemble_level": (st, [_VP, ctypes.c_int, ctypes.c_int]),
            "mg_vcycle": (st, [_VP, ctypes.c_int, _D]),
            "mg_solve": (st, [_VP, ctypes.POINTER(mg_solve_info)]),
            "mg_get_solution": (st, [_VP, _D, ctypes.c_size_t]),
            "mg_get_element_matrices": (st, [_VP, ctypes.c_int, _D, ctypes.c_size_t]),
            "mg_get_cell_data": (st, [_VP, ctypes.POINTER(ctypes.c_uint8), _D, ctypes.c_size_t]),
            "mg_get_cell_accuracy": (st, [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.c_size_t]),
            "mg_export_state": (st, [_VP, ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
            "mg_import_state": (st, [_VP, ctypes.c_void_p, ctypes.c_size_t]),
            "mg_get_coarse_classes": (st, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_uint8), ctypes.c_size_t]),
            "mg_get_trace": (st, [_VP, ctypes.POINTER(mg_trace_entry), ctypes.c_size_t,
                                  ctypes.POINTER(ctypes.c_size_t)]),
            "mg_paper_format": (st, [_VP, ctypes.c_double, ctypes.POINTER(ctypes.c_uint8), _D, ctypes.c_size_t,
                                     ctypes.POINTER(mg_paper_format_stats)]),
            "mg_get_cell_matrices": (st, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_size_t, _D]),
            "mg_apply_level": (st, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D]),
            "mg_vcycle_apply": (st, [_VP, _D, _D]),
            "mg_apply_transfer": (st, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]),
            "mg_server_create": (st, [ctypes.POINTER(mg_server_desc), ctypes.POINTER(_VP)]),
            "mg_submit": (st, [_VP, ctypes.POINTER(mg_problem_desc), _D, ctypes.POINTER(ctypes.c_uint64)]),
            "mg_poll": (st, [_VP, ctypes.c_uint64, ctypes.POINTER(mg_result)]),
            "mg_server_drain": (st, [_VP, ctypes.c_double]),
            "mg_server_destroy": (st, [_VP]),
            "mg_last_error": (ctypes.c_char_p, []),
            "mg_version": (ctypes.c_char_p, []),
            "mg_profile_kernel": (st, [_VP, ctypes.c_int, ctypes.c_int, _D]),
            "mg_launch_count": (ctypes.c_uint64, []),
            "mg_inject_assembly_failure": (st, [_VP, ctypes.c_int]),
            "mg_measure_peak": (st, [ctypes.c_int, _D]),
            "mg_assemble_surplus_noalloc": (st, [ctypes.POINTER(mg_eps_desc), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_double, ctypes.c_int64, ctypes.c_int64, _VP, _VP, _VP,
                                                 _VP]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class MGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(status: int) -> int:
    if status != MG_OK:
        raise MGError(status, load().mg_last_error().decode())
    return status


def last_error() -> str:
    return load().mg_last_error().decode()


def eps_desc(field: "_inputs.EpsField") -> mg_eps_desc:
    e = mg_eps_desc()
    e.kind = int(field.kind)
    e.n_modes = int(field.n_modes)
    e.n_boxes = int(field.n_boxes)
    e.v_out, e.v_in = float(field.v_out), float(field.v_in)
    for a in range(3):
        e.center[a] = float(field.center[a]) if a < len(field.center) else 0.0
    e.radius, e.sigma, e.theta = float(field.radius), float(field.sigma), float(field.theta)
    e.jump_x, e.jump_factor = float(field.jump_x), float(field.jump_factor)
    for m in range(field.n_modes):
        for a in range(3):
            e.k[m][a] = int(field.k[m, a])
        e.phase[m] = float(field.phase[m])
    for b in range(field.n_boxes):
        for a in range(3):
            e.box_lo[b][a] = float(field.box_lo[b, a])
            e.box_hi[b][a] = float(field.box_hi[b, a])
    return e


def problem_desc(dim: int, n_cells: int, field, path: int = PATH_FP64_PLAIN, s_schedule=(8,),
                 f_const: float = 1.0, outer: int = OUTER_FCG, tau: float = 1e-6, omega: float = 0.6,
                 nu_pre: int = 2, nu_post: int = 2, rtol: float = 1e-8, max_cycles: int = 500,
                 chunks: int = 0, u0: Optional[np.ndarray] = None, adapt_C: float = 0.0,
                 cycle: int = 0, coarse_tau: float = 0.0, adapt_keep: int = 0) -> mg_problem_desc:
    d = mg_problem_desc()
    d.dim, d.n_cells = dim, n_cells
    d.eps = eps_desc(field)
    d.f_const = f_const
    d.path, d.outer = path, outer
    for i, s in enumerate(s_schedule):
        d.s_schedule[i] = int(s)
    d.n_s = len(s_schedule)
    d.compress_tau, d.omega = tau, omega
    d.nu_pre, d.nu_post = nu_pre, nu_post
    d.rtol, d.max_cycles, d.chunks = rtol, max_cycles, chunks
    d.adapt_C = adapt_C
    d.cycle = cycle
    d.coarse_tau = coarse_tau
    d.adapt_keep = adapt_keep
    if u0 is not None:
        u0 = np.ascontiguousarray(u0, np.float64)
        d.u0 = u0.ctypes.data_as(_D)
        d._u0_keep = u0
    return d


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


class Problem:
    """One solve: owns an mg_problem handle."""

    def __init__(self, desc: mg_problem_desc, stream: Optional[int] = None):
        self.desc = desc
        self.dim, self.n = desc.dim, desc.n_cells
        h = _VP()
        _check(load().mg_create_problem(ctypes.byref(desc), stream, ctypes.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            load().mg_destroy_problem(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def nvert(self) -> int:
        return (self.n + 1) ** self.dim

    def level_cells(self, level: int) -> int:
        return (self.n // 3 ** level) ** self.dim

    def assemble(self, s: int, async_: bool = False):
        _check(load().mg_assemble_level(self.h, int(s), 1 if async_ else 0))

    def vcycle(self, n: int) -> float:
        rel = ctypes.c_double()
        _check(load().mg_vcycle(self.h, int(n), ctypes.byref(rel)))
        return rel.value

    def solve(self, check: bool = True) -> mg_solve_info:
        info = mg_solve_info()
        st = load().mg_solve(self.h, ctypes.byref(info))
        if check:
            _check(st)
        return info

    def inject_assembly_failure(self, s: int) -> None:
        """Test hook: side-stream assembly jobs of accuracy s fail on the host."""
        _check(load().mg_inject_assembly_failure(self.h, int(s)))

    def solution(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        """u on the (N+1)^d vertex grid (FP64); `out`, if given, is filled
        instead (e.g. a view of pinned host memory for fast copies)."""
        u = np.zeros(self.nvert) if out is None else out
        if u.dtype != np.float64 or u.size != self.nvert or not u.flags.c_contiguous:
            raise ValueError("out must be a contiguous float64 array of (N+1)^d entries")
        _check(load().mg_get_solution(self.h, _p(u), u.size))
        return u

    def element_matrices(self, level: int = 0) -> np.ndarray:
        nv = 1 << self.dim
        A = np.zeros((self.level_cells(level), nv, nv))
        _check(load().mg_get_element_matrices(self.h, level, _p(A), A.size))
        return A

    def cell_matrices(self, cells, level: int = 0) -> np.ndarray:
        nv = 1 << self.dim
        cells = np.ascontiguousarray(np.asarray(cells, np.int64))
        A = np.zeros((cells.shape[0], nv, nv))
        _check(load().mg_get_cell_matrices(self.h, level, cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                           cells.shape[0], _p(A)))
        return A

    def cell_data(self):
        n = self.level_cells(0)
        cls = np.zeros(n, np.uint8)
        ec = np.zeros(n)
        _check(load().mg_get_cell_data(self.h, cls.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _p(ec), n))
        return cls, ec

    def trace(self) -> list:
        """Per-iteration records of the last solve, as dicts."""
        n = ctypes.c_size_t(0)
        _check(load().mg_get_trace(self.h, None, 0, ctypes.byref(n)))
        buf = (mg_trace_entry * max(n.value, 1))()
        _check(load().mg_get_trace(self.h, buf, n.value, ctypes.byref(n)))
        return [{f: getattr(buf[i], f) for f, _ in mg_trace_entry._fields_} for i in range(n.value)]

    def paper_format(self, delta: float = 1e-8, decoded: bool = False):
        """The paper's truncated storage of the finest level's surplus:
        (p3 per cell, decoded matrices or None, statistics as a dict)."""
        n = self.level_cells(0)
        nv = 1 << self.dim
        p3 = np.zeros(n, np.uint8)
        At = np.zeros((n, nv, nv)) if decoded else None
        st = mg_paper_format_stats()
        _check(load().mg_paper_format(self.h, float(delta), p3.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                      _p(At) if decoded else None, n, ctypes.byref(st)))
        stats = {"cells_by_p3": list(st.cells_by_p3), "bytes_full": st.bytes_full, "bytes_paper": st.bytes_paper,
                 "compression": st.compression, "max_abs_error": st.max_abs_error}
        return p3, At, stats

    def export_state(self) -> bytes:
        """Checkpoint of the problem's state (solution, stored operator, accuracies)."""
        n = ctypes.c_size_t(0)
        _check(load().mg_export_state(self.h, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(load().mg_export_state(self.h, buf, n.value, ctypes.byref(n)))
        return buf.raw[:n.value]

    def import_state(self, state: bytes) -> None:
        buf = ctypes.create_string_buffer(bytes(state), len(state))
        _check(load().mg_import_state(self.h, buf, len(state)))

    def coarse_classes(self, level: int) -> np.ndarray:
        n = self.level_cells(level)
        cls = np.zeros(n, np.uint8)
        _check(load().mg_get_coarse_classes(self.h, level, cls.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), n))
        return cls

    def cell_accuracy(self) -> np.ndarray:
        n = self.level_cells(0)
        sc = np.zeros(n, np.int32)
        _check(load().mg_get_cell_accuracy(self.h, sc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n))
        return sc

    def apply(self, level: int, op: int, x: np.ndarray, b: Optional[np.ndarray] = None, inner: bool = False):
        x = np.ascontiguousarray(x, np.float64)
        y = np.zeros_like(x)
        bp = _p(np.ascontiguousarray(b, np.float64)) if b is not None else None
        _check(load().mg_apply_level(self.h, level, op, 1 if inner else 0, _p(x), bp, _p(y)))
        return y

    def restrict_residual(self, level: int, x: np.ndarray, b: np.ndarray, inner: bool = False) -> np.ndarray:
        """R (b - A x) onto level + 1 (mg_apply_transfer, op 0)."""
        x = np.ascontiguousarray(x, np.float64)
        b = np.ascontiguousarray(b, np.float64)
        nc = self.n // 3 ** (level + 1)
        out = np.zeros((nc + 1) ** self.dim)
        _check(load().mg_apply_transfer(self.h, level, 0, 1 if inner else 0, _p(x), _p(b), None, _p(out)))
        return out

    def prolong_smooth(self, level: int, x: np.ndarray, b: np.ndarray, c: np.ndarray, inner: bool = False) -> np.ndarray:
        """S(x + P c) on the level (mg_apply_transfer, op 1)."""
        x = np.ascontiguousarray(x, np.float64)
        b = np.ascontiguousarray(b, np.float64)
        c = np.ascontiguousarray(c, np.float64)
        out = np.zeros_like(x)
        _check(load().mg_apply_transfer(self.h, level, 1, 1 if inner else 0, _p(x), _p(b), _p(c), _p(out)))
        return out

    def profile(self, which: int, reps: int = 20) -> float:
        ms = ctypes.c_double()
        _check(load().mg_profile_kernel(self.h, which, reps, ctypes.byref(ms)))
        return ms.value

    def vcycle_apply(self, b: np.ndarray) -> np.ndarray:
        b = np.ascontiguousarray(b, np.float64)
        e = np.zeros_like(b)
        _check(load().mg_vcycle_apply(self.h, _p(b), _p(e)))
        return e


def measure_peak(kind: int) -> float:
    """Operations per second of one arithmetic pipe (0 FP32 FMA, 1 FP64 FMA,
    2 FP32 exp); see mg_measure_peak in include/mg.h."""
    v = np.zeros(1)
    _check(load().mg_measure_peak(int(kind), _p(v)))
    return float(v[0])


def assemble_surplus_noalloc(field, dim: int, n_cells: int, s: int, cell0: int, ncell: int, eps_c_ptr: int,
                             cls_ptr: int, surplus_ptr: int, tau: float = 1e-6, stream: Optional[int] = None) -> None:
    """Allocation-free assembly of the stored mixed-precision cell data into
    caller-owned device buffers (raw device pointers, e.g. torch tensors'
    data_ptr()); see mg_assemble_surplus_noalloc in include/mg.h."""
    e = eps_desc(field)
    _check(load().mg_assemble_surplus_noalloc(ctypes.byref(e), dim, n_cells, s, float(tau), int(cell0), int(ncell),
                                              eps_c_ptr, cls_ptr, surplus_ptr, stream))


class Server:
    def __init__(self, max_active: int = 8, budget_bytes: float = 0.0, inject_fail_every: int = 0,
                 use_graphs: bool = True):
        d = mg_server_desc()
        d.max_active, d.hbm_budget_bytes = max_active, budget_bytes
        d.inject_fail_every, d.use_graphs = inject_fail_every, 1 if use_graphs else 0
        h = _VP()
        _check(load().mg_server_create(ctypes.byref(d), ctypes.byref(h)))
        self.h = h
        self._keep = {}

    def submit(self, desc: mg_problem_desc, want_solution: bool = False) -> int:
        t = ctypes.c_uint64()
        dst = None
        if want_solution:
            dst = np.zeros((desc.n_cells + 1) ** desc.dim)
        _check(load().mg_submit(self.h, ctypes.byref(desc), _p(dst) if dst is not None else None, ctypes.byref(t)))
        self._keep[t.value] = (desc, dst)
        return t.value

    def poll(self, ticket: int):
        r = mg_result()
        st = load().mg_poll(self.h, ticket, ctypes.byref(r))
        return st, r

    def solution(self, ticket: int) -> Optional[np.ndarray]:
        return self._keep[ticket][1]

    def drain(self, timeout_ms: float = 0.0) -> int:
        return load().mg_server_drain(self.h, float(timeout_ms))

    def close(self):
        if self.h:
            load().mg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
