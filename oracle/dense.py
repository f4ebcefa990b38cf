"""Dense brute force for tiny grids (test infrastructure only).

Scatters element matrices into one dense global matrix on the interior
vertices (Eq. "weak-form-of-assembly": the global operator is the sum of
the element contributions; Dirichlet rows and columns are removed) and
solves with ``numpy.linalg.solve``.  Written independently of ``oracle.c``.
"""
from __future__ import annotations

import itertools

import numpy as np


def vertex_index(dim: int, n_cells: int, v) -> int:
    r, m = 0, 1
    for a in range(dim):
        r += v[a] * m
        m *= n_cells + 1
    return r


def interior_mask(dim: int, n_cells: int) -> np.ndarray:
    n1 = n_cells + 1
    grid = np.indices((n1,) * dim).reshape(dim, -1)[::-1]  # x fastest
    inside = np.ones(grid.shape[1], bool)
    for a in range(dim):
        inside &= (grid[a] > 0) & (grid[a] < n_cells)
    return inside


def global_matrix(dim: int, n_cells: int, A_all: np.ndarray) -> np.ndarray:
    """Full (n+1)^d x (n+1)^d matrix of the element sum (boundary rows kept)."""
    n1 = n_cells + 1
    nv = 1 << dim
    M = np.zeros((n1 ** dim, n1 ** dim))
    for c, cc in enumerate(itertools.product(range(n_cells), repeat=dim)):
        cc = cc[::-1]  # itertools gives the slowest axis first; cell index has x fastest
        gv = [vertex_index(dim, n_cells, [cc[a] + ((i >> a) & 1) for a in range(dim)]) for i in range(nv)]
        M[np.ix_(gv, gv)] += A_all[c]
    return M


def dense_solve(dim: int, n_cells: int, A_all: np.ndarray, f: np.ndarray) -> np.ndarray:
    """u with u = 0 on the boundary and A_int u_int = f_int."""
    M = global_matrix(dim, n_cells, A_all)
    m = interior_mask(dim, n_cells)
    u = np.zeros(M.shape[0])
    u[m] = np.linalg.solve(M[np.ix_(m, m)], f[m])
    return u
