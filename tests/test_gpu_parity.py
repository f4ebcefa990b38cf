"""Parity of the CUDA path (through the C ABI) against the CPU oracle.

Tolerances:
  * FP64 assembly: per cell max|A_gpu - A_oracle| <= 1e-12 max|A_oracle|.
  * FP32 (mixed) assembly incl. lossy storage: <= 1e-5 max|A_oracle| per cell
    (compression bound tau = 1e-6 plus FP32 integration error).
  * Operators, transfers, V-cycle in FP64: 1e-11 relative; in FP32: 1e-5.
  * Solutions: both sides converge to rtol; the difference is bounded by the
    conditioning times the residual gap and checked at the stated factors.
Storage classes are integers decided in FP32 on the GPU and FP64 in the
oracle: they must agree except for cells whose oracle size ratio lies within
1% of a class threshold.
"""
import numpy as np
import pytest

import oracle
from oracle import dense
from paper_2005_03606_gb300 import inputs, mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2005_03606_gb300 import build
    build.build()
    return mg.load()


def cellwise_err(A, B):
    den = np.abs(B).max(axis=(1, 2))
    return (np.abs(A - B).max(axis=(1, 2)) / den).max()


ASM_CASES = [
    (2, 27, inputs.disc_field(2), 8),
    (2, 81, inputs.theta_field(2, 16.0), 5),
    (2, 729, inputs.fourier_field(2, 12, sigma=1.0), 2),
    (3, 9, inputs.fourier_field(3, 13, sigma=1.0), 4),
    (3, 27, inputs.boxes_field(3, 14), 4),
    (3, 9, inputs.disc_field(3), 3),
    (3, 27, inputs.fourier_field(3, 15, sigma=2.0, jump_x=0.37, jump_factor=1e4), 6),
    (3, 9, inputs.const_field(3, 2.5), 16),
    (3, 81, inputs.theta_field(3, 4.0), 2),
]


@pytest.mark.parametrize("dim,n,fld,s", ASM_CASES)
def test_fp64_assembly_matches_oracle(dim, n, fld, s):
    with mg.Problem(mg.problem_desc(dim, n, fld, path=mg.PATH_FP64_PLAIN, s_schedule=(s,))) as P:
        P.assemble(s)
        if n ** dim <= 30000:
            A = P.element_matrices(0)
            ref = oracle.assemble(oracle.Field(fld), n, s)
        else:
            cells = np.random.default_rng(0).choice(n ** dim, 3000, replace=False)
            cells = np.concatenate([cells, [0, n ** dim - 1, n - 1]])
            A = P.cell_matrices(cells)
            ref = oracle.assemble_cells(oracle.Field(fld), n, s, cells)
    assert cellwise_err(A, ref) <= 1e-12


def test_fp64_geometric_stencil_is_cell_centre_sample():
    fld = inputs.fourier_field(3, 16)
    with mg.Problem(mg.problem_desc(3, 27, fld, path=mg.PATH_FP64_DELAYED, s_schedule=(1, 2))) as P:
        A = P.element_matrices(0)
    ref = oracle.assemble(oracle.Field(fld), 27, 1)
    assert cellwise_err(A, ref) <= 1e-12


def _class_ratio_near_threshold(A_ref, eps_c32, K, tau, dim):
    """True where the oracle's class decision lies within 1% of a threshold."""
    nv = 1 << dim
    iu = np.triu_indices(nv, 1)
    D = A_ref - eps_c32[:, None, None] * K[None]
    Dm = np.abs(D[:, iu[0], iu[1]]).max(axis=1)
    An = np.abs(A_ref).max(axis=(1, 2))
    F = nv - 1
    x = F * Dm / np.maximum(tau * An, 1e-300)
    # FP32 evaluation of eps and of the surplus sums carries an absolute noise of
    # about 2e-7 max|A| per entry; decisions within that band (plus 1%) may differ
    band = F * 2e-7 / tau
    near = np.zeros(len(x), bool)
    for thr in (1.0, 448.0 / 16.0, 65504.0 / 16.0):
        near |= np.abs(x - thr) < 0.01 * thr + band
    return near


MIXED_CASES = [
    (3, 27, inputs.boxes_field(3, 21), 4),
    (3, 27, inputs.fourier_field(3, 22, sigma=1.0), 4),
    (3, 27, inputs.fourier_field(3, 23, sigma=2e-5), 4),
    (3, 9, inputs.fourier_field(3, 24, sigma=2.0, jump_x=0.37, jump_factor=1e4), 8),
    (2, 81, inputs.disc_field(2), 8),
    (2, 243, inputs.fourier_field(2, 25, sigma=1e-4), 3),
]


@pytest.mark.parametrize("dim,n,fld,s", MIXED_CASES)
def test_mixed_assembly_and_storage_match_oracle(dim, n, fld, s):
    tau = 1e-6
    with mg.Problem(mg.problem_desc(dim, n, fld, path=mg.PATH_MIXED_PLAIN, s_schedule=(s,), tau=tau)) as P:
        P.assemble(s)
        A = P.element_matrices(0)
        cls, ec = P.cell_data()
    f = oracle.Field(fld)
    ref = oracle.assemble(f, n, s)
    At_ref, cls_ref, _ = oracle.compress(f, n, ref, tau)
    # assembly error of the stored FP32 operator against the exact FP64 one
    assert cellwise_err(A, ref) <= 1e-5
    # stored operator symmetric with zero row sums
    assert np.abs(A - A.transpose(0, 2, 1)).max() == 0.0
    assert (np.abs(A.sum(axis=2)).max(axis=1) <= 1e-6 * np.abs(A).max(axis=(1, 2))).all()
    # storage classes: equal except near a threshold
    K = oracle.kref(dim, n)
    near = _class_ratio_near_threshold(ref, ec.astype(np.float32).astype(np.float64), K, tau, dim)
    mism = (cls != cls_ref) & ~near
    assert mism.sum() == 0, (np.unique(cls, return_counts=True), np.unique(cls_ref, return_counts=True))
    # class-0 cells store exactly the geometric stencil
    z = cls == 0
    if z.any():
        np.testing.assert_allclose(A[z], ec[z, None, None] * K[None], rtol=0, atol=1e-7 * np.abs(ref).max())
    # where classes agree, the decoded surplus agrees within the storage bound
    same = cls == cls_ref
    err = np.abs(A[same] - At_ref[same]).max(axis=(1, 2)) / np.abs(ref[same]).max(axis=(1, 2))
    assert (err <= 2.5e-6 + 1e-5).all()


def test_mixed_storage_classes_cover_all_formats():
    fld = inputs.fourier_field(3, 41, sigma=2e-5)
    with mg.Problem(mg.problem_desc(3, 27, fld, path=mg.PATH_MIXED_PLAIN, s_schedule=(4,))) as P:
        P.assemble(4)
        cls, _ = P.cell_data()
    assert set(np.unique(cls)) >= {1, 2}


def _stored_operator(path, fld, n, s):
    """The oracle's stored operator of a path: A(s) in FP64, or the decoded
    lossy surplus storage for the mixed paths."""
    f = oracle.Field(fld)
    A = oracle.assemble(f, n, s)
    if path in (mg.PATH_MIXED_PLAIN, mg.PATH_MIXED_DELAYED):
        A, _, _ = oracle.compress(f, n, A, 1e-6)
    return A


@pytest.mark.parametrize("path,s,opdiff", [(mg.PATH_FP64_PLAIN, 4, 0.0), (mg.PATH_MIXED_PLAIN, 1, 0.0),
                                           (mg.PATH_MIXED_PLAIN, 4, 1e-5)])
@pytest.mark.parametrize("dim,n,fld", [(2, 81, inputs.disc_field(2)), (3, 27, inputs.boxes_field(3, 31)),
                                       (3, 81, inputs.disc_field(3, v_in=100.0))])
def test_operator_apply_and_jacobi_match_oracle(path, s, opdiff, dim, n, fld):
    # opdiff bounds max|A_gpu - A_oracle| / max|A| per cell of the FP32 stored
    # operator (0: both sides store the same numbers, e.g. the geometric stencils
    # of a piecewise-constant field).  These fields are piecewise constant: the
    # FP64 applications of the mixed path use the exact FP64 operator (the
    # oracle's A(s)), the FP32 inner ones the lossy stored operator.
    stored = _stored_operator(path, fld, n, s)
    exact = oracle.assemble(oracle.Field(fld), n, s)
    with mg.Problem(mg.problem_desc(dim, n, fld, path=path, s_schedule=(s,))) as P:
        if s > 1:
            P.assemble(s)
        rng = np.random.default_rng(5)
        m = dense.interior_mask(dim, n)
        x = rng.standard_normal((n + 1) ** dim) * m
        b = rng.standard_normal((n + 1) ** dim) * m
        # the 2^d cells around a vertex each contribute up to 7 |A| |x| terms
        scale = np.abs(stored).max() * np.abs(x).max() * (1 << dim) * 8
        y_ref = oracle.apply(dim, n, exact, x)
        j_ref = oracle.jacobi(dim, n, exact, b, x, 0.6)
        r_ref = oracle.residual(dim, n, exact, b, x)
        tol = 1e-13 * scale
        y = P.apply(0, 0, x, b)
        assert np.abs(y - y_ref).max() <= tol
        assert np.abs(P.apply(0, 2, x, b) - r_ref).max() <= tol
        dmin = np.abs(oracle.diag(dim, n, exact)[m]).min()
        assert np.abs(P.apply(0, 1, x, b) - j_ref).max() <= 0.6 * (tol / dmin) * 4 + 1e-12 * np.abs(j_ref).max()
        if path == mg.PATH_MIXED_PLAIN:
            # FP32 inner arithmetic of the V-cycle on the lossy stored operator
            y_ref = oracle.apply(dim, n, stored, x)
            j_ref = oracle.jacobi(dim, n, stored, b, x, 0.6)
            dmin = np.abs(oracle.diag(dim, n, stored)[m]).min()
            tol32 = 1e-6 * scale + opdiff * scale
            assert np.abs(P.apply(0, 0, x, b, inner=True) - y_ref).max() <= tol32
            assert np.abs(P.apply(0, 1, x, b, inner=True) - j_ref).max() <= 0.6 * (tol32 / dmin) * 4 + 1e-6 * np.abs(j_ref).max()


def test_lossy_residual_switch_applies_the_stored_operator(monkeypatch):
    # MG_LOSSY_RESIDUAL: the FP64 applications of the mixed path use the lossy
    # stored operator, as they do on fields that are not piecewise constant
    dim, n, s, fld = 3, 27, 4, inputs.boxes_field(3, 31)
    stored = _stored_operator(mg.PATH_MIXED_PLAIN, fld, n, s)
    monkeypatch.setenv("MG_LOSSY_RESIDUAL", "1")
    with mg.Problem(mg.problem_desc(dim, n, fld, path=mg.PATH_MIXED_PLAIN, s_schedule=(s,))) as P:
        P.assemble(s)
        rng = np.random.default_rng(5)
        m = dense.interior_mask(dim, n)
        x = rng.standard_normal((n + 1) ** dim) * m
        b = rng.standard_normal((n + 1) ** dim) * m
        y = P.apply(0, 0, x, b)
    scale = np.abs(stored).max() * np.abs(x).max() * (1 << dim) * 8
    assert np.abs(y - oracle.apply(dim, n, stored, x)).max() <= (1e-13 + 1e-5) * scale


@pytest.mark.parametrize("path", [mg.PATH_FP64_PLAIN, mg.PATH_MIXED_PLAIN])
@pytest.mark.parametrize("dim,n,fld,s", [(2, 243, inputs.disc_field(2), 2), (3, 81, inputs.boxes_field(3, 33), 2),
                                         (3, 27, inputs.fourier_field(3, 34, sigma=1.0), 4)])
def test_galerkin_levels_match_oracle(path, dim, n, fld, s):
    with mg.Problem(mg.problem_desc(dim, n, fld, path=path, s_schedule=(s,))) as P:
        P.assemble(s)
        levels = [P.element_matrices(l) for l in range(1, 3)]
    Af = _stored_operator(path, fld, n, s)
    tol = 1e-12 if path == mg.PATH_FP64_PLAIN else 2e-5
    nc = n // 3
    for Ac in levels:
        ref = oracle.galerkin(dim, nc, Af)
        assert cellwise_err(Ac, ref) <= tol
        Af = ref
        nc //= 3


@pytest.mark.parametrize("thread", [False, True])
def test_galerkin_forms_agree(monkeypatch, thread):
    # the Galerkin product of a compressed 3D FP32 level: the surplus
    # children's pair products through a per-warp queue (default) or in their
    # coarse cell's thread (MG_GALERKIN_THREAD=1), each against the oracle
    if thread:
        monkeypatch.setenv("MG_GALERKIN_THREAD", "1")
    else:
        monkeypatch.delenv("MG_GALERKIN_THREAD", raising=False)
    dim, n, s, fld = 3, 81, 2, inputs.boxes_field(3, 33)
    with mg.Problem(mg.problem_desc(dim, n, fld, path=mg.PATH_MIXED_PLAIN, s_schedule=(s,))) as P:
        P.assemble(s)
        Ac = P.element_matrices(1)
    Af = _stored_operator(mg.PATH_MIXED_PLAIN, fld, n, s)
    assert cellwise_err(Ac, oracle.galerkin(dim, n // 3, Af)) <= 2e-5


@pytest.mark.parametrize("path", [mg.PATH_FP64_PLAIN, mg.PATH_MIXED_PLAIN])
@pytest.mark.parametrize("dim,n,fld", [(2, 81, inputs.disc_field(2)), (3, 27, inputs.fourier_field(3, 35, sigma=1.0)),
                                       (3, 27, inputs.boxes_field(3, 31))])
def test_vcycle_matches_oracle(path, dim, n, fld):
    A = _stored_operator(path, fld, n, 4)
    with mg.Problem(mg.problem_desc(dim, n, fld, path=path, s_schedule=(4,))) as P:
        P.assemble(4)
        rng = np.random.default_rng(6)
        b = rng.standard_normal((n + 1) ** dim) * dense.interior_mask(dim, n)
        e = P.vcycle_apply(b)
    e_ref = oracle.vcycle_once(dim, n, A, b)
    tol = 1e-11 if path == mg.PATH_FP64_PLAIN else 1e-4
    assert np.abs(e - e_ref).max() <= tol * np.abs(e_ref).max()


@pytest.mark.parametrize("outer", [mg.OUTER_FCG, mg.OUTER_RICHARDSON])
def test_fp64_plain_solve_matches_oracle_2d_disc(outer):
    # 2D 81^2, eps = 10 in the disc r = 0.3, s = 8, V(2,2), omega = 0.6
    w = inputs.workload("disc2d")
    d = mg.problem_desc(2, 81, w.eps, path=mg.PATH_FP64_PLAIN, s_schedule=(8,), rtol=1e-10, outer=outer)
    with mg.Problem(d) as P:
        info = P.solve()
        u = P.solution()
    A = oracle.assemble(oracle.Field(w.eps), 81, 8)
    o_outer = oracle.OUTER_FCG if outer == mg.OUTER_FCG else oracle.OUTER_RICHARDSON
    u_ref, hist, k = oracle.solve(2, 81, A, rtol=1e-10, outer=o_outer)
    assert info.rel_residual <= 2e-10
    assert np.abs(u - u_ref).max() <= 1e-8 * np.abs(u_ref).max()
    assert abs(info.cycles - k) <= 2
    # residual of the GPU solution under the oracle's operator, in FP64 on the host
    r = oracle.residual(2, 81, A, oracle.load_vector(2, 81), u)
    assert np.linalg.norm(r) <= 3e-10 * np.linalg.norm(oracle.load_vector(2, 81))


@pytest.mark.parametrize("lossy", [False, True])
def test_mixed_solve_matches_oracle_operator(monkeypatch, lossy):
    # boxes (piecewise constant): the mixed path's FP64 outer residual uses the
    # exact operator, so its solution is the FP64 oracle operator's; with
    # MG_LOSSY_RESIDUAL it is the lossy stored operator's
    fld = inputs.boxes_field(3, 2003)
    n, s = 27, 4
    if lossy:
        monkeypatch.setenv("MG_LOSSY_RESIDUAL", "1")
    d = mg.problem_desc(3, n, fld, path=mg.PATH_MIXED_PLAIN, s_schedule=(s,), rtol=1e-9)
    with mg.Problem(d) as P:
        info = P.solve()
        u = P.solution()
    f = oracle.Field(fld)
    A = oracle.assemble(f, n, s)
    At, _, _ = oracle.compress(f, n, A, 1e-6)
    u_ref, _, _ = oracle.solve(3, n, At, rtol=1e-9)
    u_exact_op, _, _ = oracle.solve(3, n, A, rtol=1e-9)
    assert info.rel_residual <= 2e-9
    fv = oracle.load_vector(3, n)
    if lossy:
        assert np.abs(u - u_ref).max() <= 1e-5 * np.abs(u_ref).max()
        assert np.abs(u - u_exact_op).max() <= 1e-4 * np.abs(u_exact_op).max()
    else:
        assert np.abs(u - u_exact_op).max() <= 1e-7 * np.abs(u_exact_op).max()
        # the residual under the oracle's FP64 operator, recomputed on the host
        assert np.linalg.norm(oracle.residual(3, n, A, fv, u)) <= 2e-9 * np.linalg.norm(fv)


@pytest.mark.parametrize("path", [mg.PATH_FP64_DELAYED, mg.PATH_MIXED_DELAYED])
def test_delayed_path_reaches_plain_solution(path):
    fld = inputs.fourier_field(3, 2002, sigma=1.0)
    n = 27
    plain = mg.PATH_FP64_PLAIN if path == mg.PATH_FP64_DELAYED else mg.PATH_MIXED_PLAIN
    with mg.Problem(mg.problem_desc(3, n, fld, path=plain, s_schedule=(8,), rtol=1e-9)) as P:
        P.solve()
        u_plain = P.solution()
    with mg.Problem(mg.problem_desc(3, n, fld, path=path, s_schedule=(1, 2, 4, 8), rtol=1e-9)) as P:
        info = P.solve()
        u_del = P.solution()
        A_del = P.element_matrices(0)
    assert info.final_s == 8 and info.publishes >= 9
    assert info.rel_residual <= 2e-9
    assert np.abs(u_del - u_plain).max() <= 1e-6 * np.abs(u_plain).max()
    ref = oracle.assemble(oracle.Field(fld), n, 8)
    assert cellwise_err(A_del, ref) <= (1e-12 if path == mg.PATH_FP64_DELAYED else 1e-5)


def test_async_assembly_published_at_cycle_boundaries():
    fld = inputs.boxes_field(3, 2003)
    with mg.Problem(mg.problem_desc(3, 81, fld, path=mg.PATH_MIXED_DELAYED, s_schedule=(1, 8))) as P:
        r0 = P.vcycle(1)
        P.assemble(8, async_=True)
        rels = [P.vcycle(2) for _ in range(40)]
        info = P.solve()
        A = P.cell_matrices(np.arange(0, 81 ** 3, 997))
    ref = oracle.assemble_cells(oracle.Field(fld), 81, 8, np.arange(0, 81 ** 3, 997))
    assert cellwise_err(A, ref) <= 1e-5
    assert info.status == mg.MG_OK and info.rel_residual <= 2e-8
    assert r0 > rels[-1]


def test_theta_setup_with_zero_rhs_converges_to_zero():
    # Eq. "theta-setup": f = 0 has the solution u = 0; start from noise in [0, 4/3]
    fld = inputs.theta_field(2, 8.0)
    n = 81
    u0 = inputs.noise_vector(2, n, 11)
    d = mg.problem_desc(2, n, fld, path=mg.PATH_MIXED_DELAYED, s_schedule=(1, 2, 4), f_const=0.0, rtol=1e-10, u0=u0)
    with mg.Problem(d) as P:
        info = P.solve()
        u = P.solution()
    assert info.status == mg.MG_OK
    assert np.abs(u).max() <= 1e-7


def test_full_size_mixed_assembly_sampled():
    # 243^3 cells, 64 boxes of contrast 1e3, s = 8, at the benchmark's size and chunking
    w = inputs.workload("boxes3d")
    n = w.n_cells
    with mg.Problem(mg.problem_desc(3, n, w.eps, path=mg.PATH_MIXED_PLAIN, s_schedule=(8,))) as P:
        P.assemble(8)
        rng = np.random.default_rng(7)
        cls_all, _ = P.cell_data()
        nz = np.flatnonzero(cls_all)
        cells = np.concatenate([rng.choice(n ** 3, 400, replace=False), rng.choice(nz, 400, replace=False),
                                [0, n - 1, n ** 3 - 1, n ** 3 - n]])
        A = P.cell_matrices(cells)
    ref = oracle.assemble_cells(oracle.Field(w.eps), n, 8, cells)
    assert cellwise_err(A, ref) <= 1e-5
    assert 0.0 < (cls_all > 0).mean() < 0.5


def _oracle_vertex_rows(fld, n, s, verts, x, lossy=True):
    """(A x)_v and diag_v of the oracle's stored mixed operator (lossy) or
    of its FP64 A(s) (not lossy) at vertices `verts` (flat indices), from the
    2^3 cells around each vertex only."""
    f = oracle.Field(fld)
    n1 = n + 1
    K = oracle.kref(3, n)
    vi, vj, vk = verts % n1, (verts // n1) % n1, verts // (n1 * n1)
    cells, where = [], []
    for ox in range(2):
        for oy in range(2):
            for oz in range(2):
                cx, cy, cz = vi - 1 + ox, vj - 1 + oy, vk - 1 + oz
                cells.append((cz * n + cy) * n + cx)
                where.append((ox, oy, oz))
    uniq, inv = np.unique(np.concatenate(cells), return_inverse=True)
    A = oracle.assemble_cells(f, n, s, uniq)
    At = np.empty_like(A)
    for t, c in enumerate(uniq):
        cc = (c % n, (c // n) % n, c // (n * n))
        ec = oracle.eps_at(f, [oracle.sample_coord(n, 1, cc[a], 0) for a in range(3)])
        if lossy:
            _, At[t], _ = oracle.compress_cell(3, A[t], ec, K, 1e-6)
        else:
            At[t] = A[t]
    inv = inv.reshape(8, -1)
    Ax = np.zeros(len(verts))
    dg = np.zeros(len(verts))
    scale = np.zeros(len(verts))
    for w, (ox, oy, oz) in enumerate(where):
        a = (1 - ox) | ((1 - oy) << 1) | ((1 - oz) << 2)
        cx, cy, cz = vi - 1 + ox, vj - 1 + oy, vk - 1 + oz
        M = At[inv[w]]
        for bb in range(8):
            xb = x[((cz + (bb >> 2)) * n1 + cy + ((bb >> 1) & 1)) * n1 + cx + (bb & 1)]
            Ax += M[:, a, bb] * xb
            scale += np.abs(M[:, a, bb] * xb)
        dg += M[:, a, a]
    return Ax, dg, scale


def test_full_size_split_sweep_sampled():
    # 243^3 boxes at s = 8: the FP32 geometric bulk pass + fix-up pass against
    # the oracle's stored operator at sampled vertices (random ones and ones
    # at a corner of a cell with a surplus record)
    w = inputs.workload("boxes3d")
    n = w.n_cells
    n1 = n + 1
    line = np.zeros(n1, bool)
    line[1:n] = True
    mask = (line[:, None, None] & line[None, :, None] & line[None, None, :]).reshape(-1)
    rng = np.random.default_rng(11)
    x = rng.standard_normal(n1 ** 3) * mask
    b = rng.standard_normal(n1 ** 3) * mask
    with mg.Problem(mg.problem_desc(3, n, w.eps, path=mg.PATH_MIXED_PLAIN, s_schedule=(8,))) as P:
        P.assemble(8)
        y = P.apply(0, 0, x, b, inner=True)
        jac = P.apply(0, 1, x, b, inner=True)
        res = P.apply(0, 2, x, b, inner=True)
        y64 = P.apply(0, 0, x, b)          # FP64 outer operator (split bulk + surplus fix-up)
        res64 = P.apply(0, 2, x, b)
        cls_all, _ = P.cell_data()
    nz = np.flatnonzero(cls_all)
    cz = rng.choice(nz, 150, replace=False)
    near = ((cz // (n * n) + 1) * n1 + (cz // n) % n + 1) * n1 + cz % n + 1   # upper corner of the cell
    verts = np.concatenate([rng.choice(np.flatnonzero(mask), 150, replace=False), near])
    verts = verts[mask[verts]]
    Ax, dg, scale = _oracle_vertex_rows(w.eps, n, 8, verts, x)
    tol = 2e-5 * scale + 1e-7 * np.abs(Ax).max()
    assert np.all(np.abs(y[verts] - Ax) <= tol)
    assert np.all(np.abs(res[verts] - (b[verts] - Ax)) <= tol + 1e-6 * np.abs(b[verts]))
    # the FP64 outer operator: the exact A(8) (FP64 eps_c K_ref h + FP64 surplus)
    Ax64, _, scale64 = _oracle_vertex_rows(w.eps, n, 8, verts, x, lossy=False)
    tol64 = 1e-13 * scale64
    assert np.all(np.abs(y64[verts] - Ax64) <= tol64)
    assert np.all(np.abs(res64[verts] - (b[verts] - Ax64)) <= tol64 + 1e-15 * np.abs(b[verts]))
    j_ref = x[verts] + 0.6 * (b[verts] - Ax) / dg
    assert np.all(np.abs(jac[verts] - j_ref) <= 0.6 * (tol + 1e-6 * np.abs(b[verts])) / dg * 2 + 1e-6 * np.abs(j_ref))


@pytest.mark.parametrize("env", [{"MG_STENCIL_CAP": "64"}, {"MG_NO_SPLIT_SWEEP": "1"}, {}])
def test_split_sweep_variants_match_oracle(monkeypatch, env):
    # the split FP32 sweep with a stencil table smaller than the touched list
    # (the fix-up pass rebuilds the vertices beyond it from their cell records),
    # without the split (one pass over the cell records), and as built
    dim, n, fld, s = 3, 27, inputs.boxes_field(3, 31), 4
    stored = _stored_operator(mg.PATH_MIXED_PLAIN, fld, n, s)
    rng = np.random.default_rng(5)
    m = dense.interior_mask(dim, n)
    x = rng.standard_normal((n + 1) ** dim) * m
    b = rng.standard_normal((n + 1) ** dim) * m
    y_ref = oracle.apply(dim, n, stored, x)
    j_ref = oracle.jacobi(dim, n, stored, b, x, 0.6)
    r_ref = oracle.residual(dim, n, stored, b, x)
    scale = np.abs(stored).max() * np.abs(x).max() * (1 << dim) * 8
    tol32 = 1e-6 * scale + 1e-5 * scale
    dmin = np.abs(oracle.diag(dim, n, stored)[m]).min()
    for k in ("MG_STENCIL_CAP", "MG_NO_SPLIT_SWEEP"):
        monkeypatch.delenv(k, raising=False)
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    with mg.Problem(mg.problem_desc(dim, n, fld, path=mg.PATH_MIXED_PLAIN, s_schedule=(s,))) as P:
        P.assemble(s)
        y = P.apply(0, 0, x, b, inner=True)
        jac = P.apply(0, 1, x, b, inner=True)
        res = P.apply(0, 2, x, b, inner=True)
    assert np.abs(y - y_ref).max() <= tol32
    assert np.abs(res - r_ref).max() <= tol32 + 1e-6 * np.abs(b).max()
    assert np.abs(jac - j_ref).max() <= 0.6 * (tol32 / dmin) * 4 + 1e-6 * np.abs(j_ref).max()


@pytest.mark.parametrize("graphs", [True, False])
def test_serving_results_alone_and_in_mix_agree(graphs):
    reqs = [(3, 27, inputs.fourier_field(3, 101, sigma=0.7)), (2, 243, inputs.fourier_field(2, 102, sigma=1.5)),
            (3, 81, inputs.fourier_field(3, 103, sigma=1.0)), (2, 81, inputs.fourier_field(2, 104, sigma=2.0)),
            (3, 27, inputs.fourier_field(3, 105, sigma=2.0))]
    descs = [mg.problem_desc(d, n, f, path=mg.PATH_MIXED_DELAYED, s_schedule=(1, 2, 4, 8), rtol=1e-8)
             for d, n, f in reqs]
    alone = []
    for d in descs:
        with mg.Problem(d) as P:
            P.solve()
            alone.append(P.solution())
    S = mg.Server(max_active=4, use_graphs=graphs)
    ts = [S.submit(d, want_solution=True) for d in descs for _ in range(2)]
    assert S.drain(120000) == mg.MG_OK
    for i, t in enumerate(ts):
        st, r = S.poll(t)
        assert st == mg.MG_OK, mg.STATUS_NAMES[st]
        assert r.rel_residual <= 2e-8
        u = S.solution(t)
        ua = alone[i // 2]
        assert np.abs(u - ua).max() <= 1e-6 * np.abs(ua).max()
    S.close()


def test_edge_cases_smallest_grid_and_errors():
    fld = inputs.disc_field(3)
    with mg.Problem(mg.problem_desc(3, 9, fld, path=mg.PATH_FP64_PLAIN, s_schedule=(2,), rtol=1e-12)) as P:
        info = P.solve()
        u = P.solution()
        with pytest.raises(mg.MGError):
            P.element_matrices(5)
        with pytest.raises(mg.MGError):
            P.cell_matrices([9 ** 3])
    A = oracle.assemble(oracle.Field(fld), 9, 2)
    u_ref = dense.dense_solve(3, 9, A, oracle.load_vector(3, 9))
    assert np.abs(u - u_ref).max() <= 1e-9 * np.abs(u_ref).max()


@pytest.mark.parametrize("dim,n,fld,s,path", [
    (3, 27, inputs.boxes_field(3, 2003), 8, mg.PATH_MIXED_PLAIN),
    (3, 27, inputs.boxes_field(3, 14), 4, mg.PATH_FP64_PLAIN),
    (2, 81, inputs.disc_field(2), 8, mg.PATH_FP64_PLAIN),
    (3, 9, inputs.disc_field(3), 4, mg.PATH_MIXED_PLAIN),
])
def test_interface_cell_list_matches_full_assembly(monkeypatch, dim, n, fld, s, path):
    # piecewise-constant fields integrate only the cells a discontinuity
    # crosses; every other cell must come out exactly as the full pass has it
    # (on the mixed paths the interface list also turns on the FP64 integration
    # of the exact operator; MG_LOSSY_RESIDUAL keeps the FP32 one, as without it)
    mixed = path == mg.PATH_MIXED_PLAIN
    out = []
    for env in ({"MG_NO_INTERFACE_LIST": "1"}, {"MG_LOSSY_RESIDUAL": "1"} if mixed else {}, {}):
        monkeypatch.delenv("MG_NO_INTERFACE_LIST", raising=False)
        monkeypatch.delenv("MG_LOSSY_RESIDUAL", raising=False)
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        with mg.Problem(mg.problem_desc(dim, n, fld, path=path, s_schedule=(s,))) as P:
            P.assemble(s)
            A = P.element_matrices(0)
            cls, _ = P.cell_data()
        out.append((A, cls))
    (A0, c0), (A1, c1), (A2, c2) = out
    assert np.array_equal(c0, c1)
    assert cellwise_err(A1, A0) <= 1e-14
    ref = oracle.assemble(oracle.Field(fld), n, s)
    tol = 1e-12 if path == mg.PATH_FP64_PLAIN else 1e-5
    assert cellwise_err(A1, ref) <= tol
    assert cellwise_err(A2, ref) <= tol


@pytest.mark.parametrize("env", [{}, {"MG_NO_DENSE_STENCIL": "1"}])
def test_dense_surplus_field_sweeps_match_oracle(monkeypatch, env):
    # lognormal field with a jump: every cell carries a surplus, the finest
    # FP32 level is swept from assembled stencils (or, without them, by the
    # split pass with every vertex touched); FP64 operator through the split
    # bulk + surplus fix-up either way
    monkeypatch.delenv("MG_NO_DENSE_STENCIL", raising=False)
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    dim, n, s = 3, 27, 4
    fld = inputs.fourier_field(3, 15, sigma=2.0, jump_x=0.37, jump_factor=1e4)
    stored = _stored_operator(mg.PATH_MIXED_PLAIN, fld, n, s)
    rng = np.random.default_rng(9)
    m = dense.interior_mask(dim, n)
    x = rng.standard_normal((n + 1) ** dim) * m
    b = rng.standard_normal((n + 1) ** dim) * m
    y_ref = oracle.apply(dim, n, stored, x)
    j_ref = oracle.jacobi(dim, n, stored, b, x, 0.6)
    scale = np.abs(stored).max() * np.abs(x).max() * (1 << dim) * 8
    tol = 1e-5 * scale
    dmin = np.abs(oracle.diag(dim, n, stored)[m]).min()
    with mg.Problem(mg.problem_desc(dim, n, fld, path=mg.PATH_MIXED_PLAIN, s_schedule=(s,))) as P:
        P.assemble(s)
        assert np.abs(P.apply(0, 0, x, b, inner=True) - y_ref).max() <= tol + 1e-6 * scale
        assert np.abs(P.apply(0, 1, x, b, inner=True) - j_ref).max() <= 0.6 * (tol / dmin) * 4 + 1e-6 * np.abs(j_ref).max()
        assert np.abs(P.apply(0, 0, x, b) - y_ref).max() <= tol
        assert np.abs(P.apply(0, 2, x, b) - (b - y_ref) * m).max() <= tol
        info = P.solve()
        assert info.status == mg.MG_OK


# ---------------------------------------------------------------- degenerate and limit cases

@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("path", [mg.PATH_FP64_PLAIN, mg.PATH_FP64_DELAYED, mg.PATH_MIXED_DELAYED,
                                  mg.PATH_MIXED_PLAIN])
def test_smallest_grids(dim, path):
    # N = 3 has no coarser level: rejected (L >= 2 is required).  N = 9, the
    # smallest accepted grid, is one smoothing level over the 3^d coarse solve.
    fld = inputs.fourier_field(dim, 41, sigma=1.0)
    s = 4
    sched = (1, s) if path in (mg.PATH_FP64_DELAYED, mg.PATH_MIXED_DELAYED) else (s,)
    with pytest.raises(mg.MGError) as ei:
        mg.Problem(mg.problem_desc(dim, 3, fld, path=path, s_schedule=sched))
    assert ei.value.status == mg.MG_ERR_INVALID
    with mg.Problem(mg.problem_desc(dim, 9, fld, path=path, s_schedule=sched, rtol=1e-10)) as P:
        info = P.solve()
        u = P.solution()
    A = _stored_operator(path, fld, 9, s)
    u_ref = dense.dense_solve(dim, 9, A, oracle.load_vector(dim, 9))
    assert info.status == mg.MG_OK
    tol = 1e-8 if path in (mg.PATH_FP64_PLAIN, mg.PATH_FP64_DELAYED) else 1e-4
    assert np.abs(u - u_ref).max() <= tol * np.abs(u_ref).max()


@pytest.mark.parametrize("path", [mg.PATH_MIXED_DELAYED, mg.PATH_FP64_PLAIN])
def test_zero_right_hand_side_gives_zero(path):
    fld = inputs.boxes_field(3, 2003)
    with mg.Problem(mg.problem_desc(3, 27, fld, path=path, s_schedule=(1, 2) if path == mg.PATH_MIXED_DELAYED
                                    else (2,), f_const=0.0)) as P:
        info = P.solve()
        u = P.solution()
    assert info.status == mg.MG_OK
    assert np.abs(u).max() == 0.0


def test_constant_field_has_no_surplus_and_matches_geometric_solve():
    # constant eps: A(s) = eps K_ref at every s, so every cell is class 0 and
    # the mixed solve equals the s = 1 (geometric) FP64 solve
    fld = inputs.const_field(3, 2.5)
    with mg.Problem(mg.problem_desc(3, 27, fld, path=mg.PATH_MIXED_DELAYED, s_schedule=(1, 2, 4, 8))) as P:
        info = P.solve()
        u = P.solution()
    assert info.status == mg.MG_OK
    assert list(info.cells_by_class)[1:] == [0, 0, 0]
    with mg.Problem(mg.problem_desc(3, 27, fld, path=mg.PATH_FP64_PLAIN, s_schedule=(1,), rtol=1e-12)) as P:
        P.solve()
        u64 = P.solution()
    assert np.abs(u - u64).max() <= 1e-7 * np.abs(u64).max()


def test_initial_guess_and_cycle_limit():
    fld = inputs.disc_field(2)
    base = mg.problem_desc(2, 81, fld, path=mg.PATH_MIXED_PLAIN, s_schedule=(8,), rtol=1e-9)
    with mg.Problem(base) as P:
        P.solve()
        u_ref = P.solution()
    u0 = np.ascontiguousarray(inputs.noise_vector(2, 81, 7))
    with mg.Problem(mg.problem_desc(2, 81, fld, path=mg.PATH_MIXED_PLAIN, s_schedule=(8,), rtol=1e-9,
                                    u0=u0)) as P:
        info = P.solve()
        u = P.solution()
    assert info.status == mg.MG_OK
    assert np.abs(u - u_ref).max() <= 1e-6 * np.abs(u_ref).max()
    with mg.Problem(mg.problem_desc(2, 81, fld, path=mg.PATH_MIXED_PLAIN, s_schedule=(8,), rtol=1e-12,
                                    max_cycles=2)) as P:
        info = P.solve(check=False)
    assert info.status == mg.MG_ERR_NOT_CONVERGED
    assert info.cycles <= 3


def test_largest_2d_grid_residual_checked_on_the_host():
    # 729^2 cells (the largest 2D serving size), mixed delayed path: the final
    # residual of the oracle's stored operator, recomputed on the host
    n = 729
    fld = inputs.fourier_field(2, 12, sigma=1.5)
    with mg.Problem(mg.problem_desc(2, n, fld, path=mg.PATH_MIXED_DELAYED, s_schedule=(1, 2, 4, 8),
                                    rtol=1e-8)) as P:
        info = P.solve()
        u = P.solution()
        own = P.cell_matrices(np.arange(n * n, dtype=np.int64))
    assert info.status == mg.MG_OK
    f = oracle.load_vector(2, n)
    m = dense.interior_mask(2, n)
    # a lognormal field is not piecewise constant: the path solves its own
    # stored operator (FP32 integration, lossy storage), read back and applied
    # on the host in FP64: the residual target 1e-8 holds for it (x 2 for the
    # host's summation order)
    r_own = (f - oracle.apply(2, n, own, u)) * m
    assert np.linalg.norm(r_own) <= 2e-8 * np.linalg.norm(f * m)
    # under the oracle's stored operator it is bounded by the FP32 integration
    # (per cell within 1e-5 of the FP64 matrix)
    stored = _stored_operator(mg.PATH_MIXED_PLAIN, fld, n, 8)
    r = (f - oracle.apply(2, n, stored, u)) * m
    assert np.linalg.norm(r) <= 1e-4 * np.linalg.norm(f * m)


@pytest.mark.parametrize("dim,n,fld,sched", [
    (3, 81, inputs.boxes_field(3, 2003), (1, 2, 4)),
    (2, 243, inputs.disc_field(2), (1, 2, 4, 8)),
])
def test_mixed_delayed_residual_under_the_fp64_operator(dim, n, fld, sched):
    # piecewise-constant fields: the mixed delayed solution meets 1e-8 under the
    # oracle's FP64 operator A(s_final), recomputed on the host (x 2 for the
    # host's summation order)
    with mg.Problem(mg.problem_desc(dim, n, fld, path=mg.PATH_MIXED_DELAYED, s_schedule=sched, rtol=1e-8)) as P:
        info = P.solve()
        u = P.solution()
    assert info.status == mg.MG_OK
    A = oracle.assemble(oracle.Field(fld), n, sched[-1])
    fv = oracle.load_vector(dim, n)
    assert np.linalg.norm(oracle.residual(dim, n, A, fv, u)) <= 2e-8 * np.linalg.norm(fv)


@pytest.mark.parametrize("switch", ["MG_NO_VTAIL", "MG_NO_GRAPHS", "MG_NO_PDL", "MG_FUSED_RESTRICT",
                                    "MG_NO_SPECULATE", "MG_NO_U1", "MG_CELL_FORM64"])
def test_alternative_cycle_implementations_agree(switch, monkeypatch):
    # the one-block tail of the V-cycle (levels 9 and 3), the CUDA-graph replay
    # of an iteration, the programmatic-dependent launches, the fused
    # residual + restriction, the inner iterations enqueued ahead of the host's
    # test and the first smoothing step formed by the kernel that writes the
    # right-hand side and the cell form of the FP64 bulk pass (instead of its
    # vertex form) are implementation choices: switching any of them must
    # give the same solution.  They change the rounding order of FP32 sums,
    # and on this coarse 27^3 grid (boxes of 0.5 to 4 cells, 83 cycles) the
    # inner iteration count moves by a few cycles with it (so does the
    # speculation, by the extra steps it takes).
    w = inputs.workload("boxes3d", 27)
    d = mg.problem_desc(3, 27, w.eps, path=mg.PATH_MIXED_PLAIN, s_schedule=(8,), rtol=1e-8)
    with mg.Problem(d) as P:
        i0 = P.solve()
        u0 = P.solution()
    monkeypatch.setenv(switch, "1")
    with mg.Problem(d) as P:
        i1 = P.solve()
        u1 = P.solution()
    assert i1.status == mg.MG_OK and abs(i1.cycles - i0.cycles) <= max(1, round(0.04 * i0.cycles))
    assert np.abs(u1 - u0).max() <= 1e-6 * np.abs(u0).max()


# ------------------------------------------------------------ transfers fused with sweeps
TRANSFER_CASES = [
    (2, 81, inputs.disc_field(2), mg.PATH_FP64_PLAIN, {}),
    (2, 81, inputs.disc_field(2), mg.PATH_MIXED_PLAIN, {}),
    (3, 27, inputs.boxes_field(3, 31), mg.PATH_FP64_PLAIN, {}),
    (3, 27, inputs.boxes_field(3, 31), mg.PATH_MIXED_PLAIN, {}),
    (3, 27, inputs.boxes_field(3, 31), mg.PATH_MIXED_PLAIN, {"MG_FUSED_RESTRICT": "1"}),   # fused (split level)
    (3, 27, inputs.boxes_field(3, 31), mg.PATH_MIXED_PLAIN, {"MG_FUSED_RESTRICT": "1", "MG_STENCIL_CAP": "64"}),
    (3, 81, inputs.disc_field(3, v_in=100.0), mg.PATH_MIXED_PLAIN, {}),
]


@pytest.mark.parametrize("dim,n,fld,path,env", TRANSFER_CASES)
def test_restricted_residual_matches_oracle(monkeypatch, dim, n, fld, path, env):
    # R (b - A x) onto the next coarser level in the V-cycle arithmetic: the
    # fused residual + restriction on split 3D levels (its z-restricted bulk
    # pass, the touched vertices' fix-up residuals and the x-y pass), the tiled
    # restriction after a residual sweep elsewhere
    for k in ("MG_FUSED_RESTRICT", "MG_STENCIL_CAP"):
        monkeypatch.delenv(k, raising=False)
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    s = 4
    stored = _stored_operator(path, fld, n, s)
    rng = np.random.default_rng(21)
    m = dense.interior_mask(dim, n)
    x = rng.standard_normal((n + 1) ** dim) * m
    b = rng.standard_normal((n + 1) ** dim) * m
    inner = path == mg.PATH_MIXED_PLAIN
    with mg.Problem(mg.problem_desc(dim, n, fld, path=path, s_schedule=(s,))) as P:
        P.assemble(s)
        out = P.restrict_residual(0, x, b, inner=inner)
        out2 = P.restrict_residual(0, x, b, inner=inner)
    nc = n // 3
    ref = oracle.restrict(dim, nc, oracle.residual(dim, n, stored, b, x))
    mc = dense.interior_mask(dim, nc)
    assert np.all(out[~mc] == 0.0)
    # the restriction weights sum to 3^d per coarse vertex
    rscale = (np.abs(stored).max() * np.abs(x).max() * (1 << dim) * 8 + np.abs(b).max()) * 3 ** dim
    tol = (1e-11 if not inner else 2e-6) * rscale
    assert np.abs(out - ref).max() <= tol
    assert np.array_equal(out, out2)   # deterministic: no atomics in the sums


@pytest.mark.parametrize("dim,n,fld,path,env", [c for c in TRANSFER_CASES if not c[4]])
def test_prolonged_smoothing_matches_oracle(dim, n, fld, path, env):
    # S(x + P c): prolongation of a coarse correction, then one damped Jacobi sweep
    s = 4
    stored = _stored_operator(path, fld, n, s)
    rng = np.random.default_rng(22)
    m = dense.interior_mask(dim, n)
    nc = n // 3
    x = rng.standard_normal((n + 1) ** dim) * m
    b = rng.standard_normal((n + 1) ** dim) * m
    c = rng.standard_normal((nc + 1) ** dim) * dense.interior_mask(dim, nc)
    inner = path == mg.PATH_MIXED_PLAIN
    with mg.Problem(mg.problem_desc(dim, n, fld, path=path, s_schedule=(s,))) as P:
        P.assemble(s)
        out = P.prolong_smooth(0, x, b, c, inner=inner)
    xp = oracle.prolong_add(dim, nc, c, x)
    ref = oracle.jacobi(dim, n, stored, b, xp, 0.6)
    dmin = np.abs(oracle.diag(dim, n, stored)[m]).min()
    scale = np.abs(stored).max() * np.abs(xp).max() * (1 << dim) * 8 + np.abs(b).max()
    tol = (1e-11 if not inner else 2e-5) * (scale / dmin + np.abs(xp).max())
    assert np.all(out[~m] == 0.0)
    assert np.abs(out - ref).max() <= tol


@pytest.mark.parametrize("cell_form", [False, True])
def test_full_size_fp64_residual_sampled(monkeypatch, cell_form):
    # 243^3 boxes at s = 8: the outer FP64 residual b - A x of the mixed path
    # (the exact FP64 operator) in the launch configuration of the benchmark,
    # at sampled vertices (random ones and ones next to a cell with a surplus
    # record) against the oracle's FP64 A(8) rows.  The vertex form (eps sums
    # per vertex and per edge built once) is the default; MG_CELL_FORM64=1
    # forms them in every application.
    if cell_form:
        monkeypatch.setenv("MG_CELL_FORM64", "1")
    else:
        monkeypatch.delenv("MG_CELL_FORM64", raising=False)
    w = inputs.workload("boxes3d")
    n = w.n_cells
    n1 = n + 1
    line = np.zeros(n1, bool)
    line[1:n] = True
    mask = (line[:, None, None] & line[None, :, None] & line[None, None, :]).reshape(-1)
    rng = np.random.default_rng(13)
    x = rng.standard_normal(n1 ** 3) * mask
    b = rng.standard_normal(n1 ** 3) * mask
    with mg.Problem(mg.problem_desc(3, n, w.eps, path=mg.PATH_MIXED_PLAIN, s_schedule=(8,))) as P:
        P.assemble(8)
        r = P.apply(0, 2, x, b)
        cls_all, _ = P.cell_data()
    nz = rng.choice(np.flatnonzero(cls_all), 32, replace=False)
    # the upper corner vertex of each cell (interior, so that the row is a full one)
    near = [(min(n - 1, c % n + 1), min(n - 1, (c // n) % n + 1), min(n - 1, c // (n * n) + 1)) for c in nz]
    rand = [tuple(int(t) for t in rng.integers(1, n, 3)) for _ in range(32)]
    verts = np.array([(k * n1 + j) * n1 + i for (i, j, k) in near + rand])
    Ax, _, scale = _oracle_vertex_rows(w.eps, n, 8, verts, x, lossy=False)
    ref = b[verts] - Ax
    assert np.all(np.abs(r[verts] - ref) <= 1e-12 * (scale + np.abs(b[verts])))
    assert np.all(r.reshape(n1, n1, n1)[0] == 0) and np.all(r.reshape(n1, n1, n1)[:, :, n] == 0)


@pytest.mark.parametrize("fused", [False, True])
def test_full_size_fused_restriction_sampled(monkeypatch, fused):
    # 243^3 boxes at s = 8, the launch configuration of the benchmark's
    # V-cycle (the separate residual sweep and tiled restriction) and the fused
    # residual + restriction: R (b - A x) at sampled coarse vertices (random
    # ones and ones above a cell with a surplus record), each from the
    # oracle's residual at its 5^3 fine vertices
    if fused:
        monkeypatch.setenv("MG_FUSED_RESTRICT", "1")
    else:
        monkeypatch.delenv("MG_FUSED_RESTRICT", raising=False)
    w = inputs.workload("boxes3d")
    n = w.n_cells
    n1, nc = n + 1, n // 3
    nc1 = nc + 1
    line = np.zeros(n1, bool)
    line[1:n] = True
    mask = (line[:, None, None] & line[None, :, None] & line[None, None, :]).reshape(-1)
    rng = np.random.default_rng(12)
    x = rng.standard_normal(n1 ** 3) * mask
    b = rng.standard_normal(n1 ** 3) * mask
    with mg.Problem(mg.problem_desc(3, n, w.eps, path=mg.PATH_MIXED_PLAIN, s_schedule=(8,))) as P:
        P.assemble(8)
        out = P.restrict_residual(0, x, b, inner=True)
        cls_all, _ = P.cell_data()
    nz = np.flatnonzero(cls_all)
    cz = rng.choice(nz, 24, replace=False)
    # the coarse vertex nearest to the cell's upper corner
    near = [tuple(min(nc - 1, max(1, (int(v) + 1 + 1) // 3)) for v in (c % n, (c // n) % n, c // (n * n))) for c in cz]
    rand = [tuple(int(t) for t in rng.integers(1, nc, 3)) for _ in range(24)]
    w1 = np.array([1.0 / 3.0, 2.0 / 3.0, 1.0, 2.0 / 3.0, 1.0 / 3.0])
    d = np.arange(-2, 3)
    for (I, J, K) in near + rand:
        fi, fj, fk = np.meshgrid(3 * I + d, 3 * J + d, 3 * K + d, indexing="ij")
        verts = ((fk * n1 + fj) * n1 + fi).reshape(-1)
        wts = (w1[:, None, None] * w1[None, :, None] * w1[None, None, :]).reshape(-1)
        Ax, _, scale = _oracle_vertex_rows(w.eps, n, 8, verts, x)
        ref = np.sum(wts * (b[verts] - Ax))
        got = out[(K * nc1 + J) * nc1 + I]
        tol = 2e-5 * np.sum(wts * (scale + np.abs(b[verts]))) + 1e-7 * np.abs(ref)
        assert abs(got - ref) <= tol, (I, J, K, got, ref)
