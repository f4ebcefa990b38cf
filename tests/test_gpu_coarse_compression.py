"""Compressed coarse-level operators on the GPU against the oracle.

With desc.coarse_tau > 0 every coarse level stores its Galerkin operator as
the lossy hierarchical surplus over its one-sample rediscretisation (Section
"Precision toggling and information density"), decoded before any use.  For
each coarse level the oracle takes the GPU's stored operator of the level
above (read back through the C ABI), forms the Galerkin product in FP64 and
applies the same storage rule (oracle.compress at that level's cell count:
eps at the coarse cell centres, rounded to FP32).  Classes are integers
decided in FP32 on the GPU and FP64 in the oracle: they must agree except
within 1% (plus the FP32 noise band) of a threshold.  The decoded matrices
agree within 1e-5 of each cell's largest entry plus the storage bound (2 tau
relative: each side's own lossy step), since the GPU's Galerkin product runs
in FP32.
"""
import numpy as np
import pytest

import oracle
from paper_2005_03606_gb300 import inputs, mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2005_03606_gb300 import build
    build.build()
    return mg.load()


def _near_threshold(A_ref, eps_c32, K, tau, dim):
    nv = 1 << dim
    iu = np.triu_indices(nv, 1)
    D = A_ref - eps_c32[:, None, None] * K[None]
    Dm = np.abs(D[:, iu[0], iu[1]]).max(axis=1)
    An = np.abs(A_ref).max(axis=(1, 2))
    x = (nv - 1) * Dm / np.maximum(tau * An, 1e-300)
    band = (nv - 1) * 2e-7 / tau
    near = np.zeros(len(x), bool)
    for thr in (1.0, 448.0 / 16.0, 65504.0 / 16.0):
        near |= np.abs(x - thr) < 0.01 * thr + band
    return near


CASES = [
    (3, 81, inputs.boxes_field(3, 14), 4, 1e-6),
    (3, 81, inputs.boxes_field(3, 14), 4, 1e-3),
    (2, 243, inputs.disc_field(2, v_in=100.0), 8, 1e-6),
    (3, 27, inputs.fourier_field(3, 15, sigma=2.0, jump_x=0.37, jump_factor=1e4), 4, 1e-4),
]


@pytest.mark.parametrize("dim,n,fld,s,tau", CASES)
def test_coarse_operators_match_oracle(dim, n, fld, s, tau):
    F = oracle.Field(fld)
    with mg.Problem(mg.problem_desc(dim, n, fld, path=mg.PATH_MIXED_PLAIN, s_schedule=(s,), coarse_tau=tau)) as P:
        P.assemble(s)
        levels, classes = [P.element_matrices(0)], [None]
        nl, l = n // 3, 1
        while nl >= 3:
            levels.append(P.element_matrices(l))
            classes.append(P.coarse_classes(l))
            nl //= 3
            l += 1
    nl = n
    for l in range(1, len(levels)):
        nl //= 3
        A_gal = oracle.galerkin(dim, nl, levels[l - 1])
        At, cls, _ = oracle.compress(F, nl, A_gal, tau)
        ec32 = np.array([np.float32(oracle.eps_at(F, [(c + 0.5) / nl for c in cc]))
                         for cc in _cell_coords(dim, nl)], np.float64)
        near = _near_threshold(A_gal, ec32, oracle.kref(dim, nl), tau, dim)
        bad = (classes[l] != cls) & ~near
        assert not bad.any(), (l, np.flatnonzero(bad)[:5])
        den = np.abs(At).max(axis=(1, 2))
        err = np.abs(levels[l] - At).max(axis=(1, 2)) / den
        assert err.max() <= 1e-5 + 2 * tau, (l, err.max())
    # the piecewise-constant fields leave most coarse cells without a surplus
    if fld.kind in (inputs.KIND_BOXES, inputs.KIND_DISC):
        assert (classes[1] == 0).mean() > 0.5


def _cell_coords(dim, n):
    for c in range(n ** dim):
        out, t = [], c
        for _ in range(dim):
            out.append(t % n)
            t //= n
        yield out


def test_coarse_compression_keeps_the_solve():
    w = inputs.workload("boxes3d", 81)
    base = dict(path=mg.PATH_MIXED_PLAIN, s_schedule=(8,), rtol=1e-8)
    with mg.Problem(mg.problem_desc(w.dim, w.n_cells, w.eps, **base)) as P:
        i0 = P.solve()
        u0 = P.solution()
    with mg.Problem(mg.problem_desc(w.dim, w.n_cells, w.eps, coarse_tau=1e-6, **base)) as P:
        i1 = P.solve()
        u1 = P.solution()
    assert i1.status == mg.MG_OK and i1.rel_residual <= 2e-8
    assert abs(i1.cycles - i0.cycles) <= 3
    assert np.abs(u1 - u0).max() <= 1e-6 * np.abs(u0).max()


def test_coarse_compression_arguments():
    f = inputs.const_field(2)
    for kw in ({"coarse_tau": -1.0}, {"coarse_tau": float("nan")},
               {"coarse_tau": 1e-6, "path": mg.PATH_FP64_PLAIN}):
        with pytest.raises(mg.MGError) as ei:
            mg.Problem(mg.problem_desc(2, 27, f, **kw))
        assert ei.value.status == mg.MG_ERR_INVALID
    with mg.Problem(mg.problem_desc(2, 27, f, path=mg.PATH_MIXED_PLAIN)) as P:
        with pytest.raises(mg.MGError):
            P.coarse_classes(1)
