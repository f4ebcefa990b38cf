"""CPU oracle (test infrastructure only).

Plain FP64 C (``oracle.c``) plus a NumPy dense brute force (``dense.py``).
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it; the CUDA library never does, and the two share no code.

Every function is pinned by ``tests/test_oracle.py`` against closed forms,
invariants, exact rational integration and library routines.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (FP64, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


class _Field(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dim", ctypes.c_int), ("n_modes", ctypes.c_int),
                ("n_boxes", ctypes.c_int), ("v_out", ctypes.c_double), ("v_in", ctypes.c_double),
                ("center", ctypes.c_double * 3), ("radius", ctypes.c_double),
                ("sigma", ctypes.c_double), ("theta", ctypes.c_double),
                ("jump_x", ctypes.c_double), ("jump_factor", ctypes.c_double),
                ("k", ctypes.POINTER(ctypes.c_int32)), ("phase", ctypes.POINTER(ctypes.c_double)),
                ("box_lo", ctypes.POINTER(ctypes.c_double)),
                ("box_hi", ctypes.POINTER(ctypes.c_double))]


_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        FP = ctypes.POINTER(_Field)
        lib.oc_eps.argtypes = [FP, _D]
        lib.oc_eps.restype = ctypes.c_double
        lib.oc_sample_coord.argtypes = [ctypes.c_int] * 4
        lib.oc_sample_coord.restype = ctypes.c_double
        lib.oc_element_matrix.argtypes = [FP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, _D]
        lib.oc_assemble.argtypes = [FP, ctypes.c_int, ctypes.c_int, _D]
        lib.oc_assemble_cells.argtypes = [FP, ctypes.c_int, ctypes.c_int, _I64, ctypes.c_int64, _D]
        lib.oc_assemble_adaptive.argtypes = [FP, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_int,
                                             ctypes.c_double, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_int32)]
        lib.oc_round_format.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double]
        lib.oc_round_format.restype = ctypes.c_double
        lib.oc_round_e4m3.argtypes = [ctypes.c_double]
        lib.oc_round_e4m3.restype = ctypes.c_double
        lib.oc_round_f16.argtypes = [ctypes.c_double]
        lib.oc_round_f16.restype = ctypes.c_double
        lib.oc_compress_cell.argtypes = [ctypes.c_int, _D, ctypes.c_double, _D, ctypes.c_double, _D, _D]
        lib.oc_compress_cell.restype = ctypes.c_int
        lib.oc_kref.argtypes = [ctypes.c_int, ctypes.c_int, _D]
        lib.oc_compress.argtypes = [FP, ctypes.c_int, _D, ctypes.c_double, _D,
                                    ctypes.POINTER(ctypes.c_uint8), _D]
        lib.oc_pf_roundtrip.argtypes = [ctypes.c_double, ctypes.c_int]
        lib.oc_pf_roundtrip.restype = ctypes.c_double
        lib.oc_pf_choose.argtypes = [_D, ctypes.c_int, ctypes.c_double]
        lib.oc_pf_choose.restype = ctypes.c_int
        lib.oc_paper_format.argtypes = [ctypes.c_int, ctypes.c_int64, _D, _D, _D, ctypes.c_double,
                                        ctypes.POINTER(ctypes.c_int32), _D]
        lib.oc_apply.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D]
        lib.oc_diag.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        lib.oc_residual.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]
        lib.oc_jacobi.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, ctypes.c_double, _D]
        lib.oc_prolong_add.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        lib.oc_restrict.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        lib.oc_galerkin.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        lib.oc_solve.argtypes = [ctypes.c_int, ctypes.c_int, _D, ctypes.c_double, _D, ctypes.c_double,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                 _D, _D]
        lib.oc_solve.restype = ctypes.c_int
        lib.oc_vcycle_once.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_int, _D]
        lib.oc_vcycle_once.restype = ctypes.c_int
        lib.oc_inject.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        lib.oc_additive_once.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_int, _D]
        lib.oc_additive_once.restype = ctypes.c_int
        lib.oc_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(_D)


class Field:
    """Holds an eps field (from ``paper_2005_03606_gb300.inputs``) in the oracle's layout."""

    def __init__(self, eps):
        self.eps = eps
        self._k = np.ascontiguousarray(np.asarray(eps.k, np.int32).reshape(-1, 3))
        self._phase = np.ascontiguousarray(np.asarray(eps.phase, np.float64))
        self._lo = np.ascontiguousarray(np.asarray(eps.box_lo, np.float64).reshape(-1, 3))
        self._hi = np.ascontiguousarray(np.asarray(eps.box_hi, np.float64).reshape(-1, 3))
        f = _Field()
        f.kind, f.dim = int(eps.kind), int(eps.dim)
        f.n_modes, f.n_boxes = int(self._k.shape[0]), int(self._lo.shape[0])
        f.v_out, f.v_in = float(eps.v_out), float(eps.v_in)
        for a in range(3):
            f.center[a] = float(eps.center[a]) if a < len(eps.center) else 0.0
        f.radius, f.sigma, f.theta = float(eps.radius), float(eps.sigma), float(eps.theta)
        f.jump_x, f.jump_factor = float(eps.jump_x), float(eps.jump_factor)
        f.k = self._k.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        f.phase = _p(self._phase)
        f.box_lo = _p(self._lo)
        f.box_hi = _p(self._hi)
        self.c = f

    @property
    def dim(self):
        return self.eps.dim


def eps_at(field: Field, x) -> float:
    x = np.ascontiguousarray(np.asarray(x, np.float64))
    return _load().oc_eps(ctypes.byref(field.c), _p(x))


def sample_coord(n_cells: int, s: int, i: int, j: int) -> float:
    return _load().oc_sample_coord(n_cells, s, i, j)


def element_matrix(field: Field, n_cells: int, cell, s: int) -> np.ndarray:
    d = field.dim
    nv = 1 << d
    A = np.zeros((nv, nv))
    cc = (ctypes.c_int * 3)(*(list(cell) + [0] * (3 - len(cell))))
    _load().oc_element_matrix(ctypes.byref(field.c), n_cells, cc, s, _p(A))
    return A


def assemble(field: Field, n_cells: int, s: int) -> np.ndarray:
    """Element matrices of all cells, shape (n_cells^d, 2^d, 2^d)."""
    d = field.dim
    nv = 1 << d
    A = np.zeros((n_cells ** d, nv, nv))
    _load().oc_assemble(ctypes.byref(field.c), n_cells, s, _p(A))
    return A


def assemble_cells(field: Field, n_cells: int, s: int, cells) -> np.ndarray:
    d = field.dim
    nv = 1 << d
    cells = np.ascontiguousarray(np.asarray(cells, np.int64))
    A = np.zeros((cells.shape[0], nv, nv))
    _load().oc_assemble_cells(ctypes.byref(field.c), n_cells, s,
                              cells.ctypes.data_as(_I64), cells.shape[0], _p(A))
    return A


def assemble_adaptive(field: Field, n_cells: int, schedule, C: float, keep_old: bool = False):
    """Adaptive per-cell accuracy (Section "Adaptive stencil integration"):
    (element matrices of every cell, accuracy s of each stored matrix).
    keep_old: a cell that passes the test keeps the older matrix (the
    reading of Table "memory-footprint") instead of the newer one."""
    nv = 1 << field.dim
    ncell = n_cells ** field.dim
    A = np.zeros((ncell, nv, nv))
    sc = np.zeros(ncell, np.int32)
    sched = np.ascontiguousarray(np.asarray(schedule, np.int32))
    _load().oc_assemble_adaptive(ctypes.byref(field.c), n_cells, sched.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 len(sched), float(C), 1 if keep_old else 0, _p(A),
                                 sc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return A, sc


def kref(dim: int, n_cells: int) -> np.ndarray:
    nv = 1 << dim
    K = np.zeros((nv, nv))
    _load().oc_kref(dim, n_cells, _p(K))
    return K


def round_e4m3(x: float) -> float:
    return _load().oc_round_e4m3(float(x))


def round_f16(x: float) -> float:
    return _load().oc_round_f16(float(x))


def round_format(x: float, mbits: int, emin: int, maxval: float) -> float:
    return _load().oc_round_format(float(x), mbits, emin, maxval)


def compress_cell(dim: int, A: np.ndarray, eps_c: float, K: np.ndarray, tau: float):
    """Returns (class, decoded stored matrix, scale) for one cell."""
    A = np.ascontiguousarray(A, np.float64)
    K = np.ascontiguousarray(K, np.float64)
    At = np.zeros_like(A)
    sc = np.zeros(1)
    c = _load().oc_compress_cell(dim, _p(A), float(eps_c), _p(K), float(tau), _p(At), _p(sc))
    return c, At, float(sc[0])


def compress(field: Field, n_cells: int, A_all: np.ndarray, tau: float):
    """Mixed-path stored operator: (decoded matrices, classes, scales)."""
    A_all = np.ascontiguousarray(A_all, np.float64)
    At = np.zeros_like(A_all)
    cls = np.zeros(A_all.shape[0], np.uint8)
    sc = np.zeros(A_all.shape[0])
    _load().oc_compress(ctypes.byref(field.c), n_cells, _p(A_all), float(tau), _p(At),
                        cls.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _p(sc))
    return At, cls, sc


def pf_roundtrip(x: float, p3: int) -> float:
    """Value of x after storage in the paper's format with p3 bytes
    (Section "Precision toggling and information density")."""
    return _load().oc_pf_roundtrip(float(x), int(p3))


def pf_choose(dA, delta: float) -> int:
    """Bytes per entry of a cell's surplus entries dA at absolute threshold delta."""
    a = np.ascontiguousarray(np.ravel(dA), np.float64)
    return _load().oc_pf_choose(_p(a), a.size, float(delta))


def paper_format(dim: int, A_all: np.ndarray, eps_c: np.ndarray, K: np.ndarray, delta: float):
    """(p3 per cell, decoded stored matrices) of the paper's format on the
    surplus A - eps_c K of every cell."""
    A_all = np.ascontiguousarray(A_all, np.float64)
    ncell = A_all.shape[0]
    p3 = np.zeros(ncell, np.int32)
    At = np.zeros_like(A_all)
    _load().oc_paper_format(dim, ncell, _p(A_all), _p(np.ascontiguousarray(eps_c, np.float64)),
                            _p(np.ascontiguousarray(K, np.float64)), float(delta),
                            p3.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _p(At))
    return p3, At


def paper_compression(dim: int, p3: np.ndarray) -> float:
    """Compression factor of the paper's accounting: a full element matrix is
    4^d doubles; a cell stores one marker byte plus p3 bytes per entry."""
    ne = 4 ** dim
    return float(p3.size * ne * 8) / float(np.sum(1 + ne * p3.astype(np.int64)))


def apply(dim: int, n_cells: int, A_all: np.ndarray, u: np.ndarray) -> np.ndarray:
    y = np.zeros((n_cells + 1) ** dim)
    _load().oc_apply(dim, n_cells, _p(np.ascontiguousarray(A_all)), _p(np.ascontiguousarray(u, np.float64)), _p(y))
    return y


def diag(dim: int, n_cells: int, A_all: np.ndarray) -> np.ndarray:
    y = np.zeros((n_cells + 1) ** dim)
    _load().oc_diag(dim, n_cells, _p(np.ascontiguousarray(A_all)), _p(y))
    return y


def residual(dim, n_cells, A_all, b, u):
    r = np.zeros((n_cells + 1) ** dim)
    _load().oc_residual(dim, n_cells, _p(np.ascontiguousarray(A_all)), _p(np.ascontiguousarray(b, np.float64)),
                        _p(np.ascontiguousarray(u, np.float64)), _p(r))
    return r


def jacobi(dim, n_cells, A_all, b, u, omega):
    out = np.zeros((n_cells + 1) ** dim)
    _load().oc_jacobi(dim, n_cells, _p(np.ascontiguousarray(A_all)), _p(np.ascontiguousarray(b, np.float64)),
                      _p(np.ascontiguousarray(u, np.float64)), float(omega), _p(out))
    return out


def prolong_add(dim, nc, ec, ef):
    ef = np.array(ef, np.float64, copy=True)
    _load().oc_prolong_add(dim, nc, _p(np.ascontiguousarray(ec, np.float64)), _p(ef))
    return ef


def restrict(dim, nc, rf):
    bc = np.zeros((nc + 1) ** dim)
    _load().oc_restrict(dim, nc, _p(np.ascontiguousarray(rf, np.float64)), _p(bc))
    return bc


def galerkin(dim, nc, A_fine):
    nv = 1 << dim
    Ac = np.zeros((nc ** dim, nv, nv))
    _load().oc_galerkin(dim, nc, _p(np.ascontiguousarray(A_fine)), _p(Ac))
    return Ac


OUTER_RICHARDSON, OUTER_FCG = 0, 1


def solve(dim, n_cells, A_fine, f_const=1.0, u0=None, omega=0.6, nu_pre=2, nu_post=2,
          rtol=1e-8, max_cycles=200, outer=OUTER_FCG):
    """Returns (u on the vertex grid, residual history, cycles)."""
    u = np.zeros((n_cells + 1) ** dim)
    hist = np.zeros(max_cycles + 1)
    u0p = _p(np.ascontiguousarray(u0, np.float64)) if u0 is not None else None
    k = _load().oc_solve(dim, n_cells, _p(np.ascontiguousarray(A_fine)), float(f_const), u0p,
                         float(omega), nu_pre, nu_post, float(rtol), max_cycles, int(outer), _p(u), _p(hist))
    if k < 0:
        raise ValueError("bad grid size")
    return u, hist[: k + 1], k


def vcycle_once(dim, n_cells, A_fine, b, omega=0.6, nu_pre=2, nu_post=2):
    e = np.zeros((n_cells + 1) ** dim)
    rc = _load().oc_vcycle_once(dim, n_cells, _p(np.ascontiguousarray(A_fine)),
                                _p(np.ascontiguousarray(b, np.float64)), float(omega), nu_pre, nu_post, _p(e))
    if rc < 0:
        raise ValueError("bad grid size")
    return e


def inject(dim, nc, rf):
    bc = np.zeros((nc + 1) ** dim)
    _load().oc_inject(dim, nc, _p(np.ascontiguousarray(rf, np.float64)), _p(bc))
    return bc


ADDITIVE, ADAFAC_PI, ADAFAC_JAC = 0, 1, 2


def additive_once(dim, n_cells, A_fine, b, omega=0.6, variant=ADAFAC_JAC):
    """One additive cycle (plain, adaFAC-PI or adaFAC-Jac) for A e = b from e = 0."""
    e = np.zeros((n_cells + 1) ** dim)
    rc = _load().oc_additive_once(dim, n_cells, _p(np.ascontiguousarray(A_fine, np.float64)),
                                  _p(np.ascontiguousarray(b, np.float64)), float(omega), int(variant), _p(e))
    if rc != 0:
        raise ValueError("n_cells must be a power of 3")
    return e


def load_vector(dim: int, n_cells: int, f_const: float = 1.0) -> np.ndarray:
    """f_v = integral of f_const * phi_v = f_const h^d on interior vertices."""
    n1 = n_cells + 1
    f = np.full((n1,) * dim, f_const * (1.0 / n_cells) ** dim)
    for a in range(dim):
        idx = [slice(None)] * dim
        for e in (0, n1 - 1):
            idx[a] = e
            f[tuple(idx)] = 0.0
    return f.reshape(-1)


def num_threads() -> int:
    return _load().oc_num_threads()
