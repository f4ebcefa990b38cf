"""The allocation-free assembly entry point against the regular one.

mg_assemble_surplus_noalloc computes, into caller-owned device buffers and
with a fixed scratch array inside the library, the same cell data that the
mixed-precision paths store (cell-centre eps, storage class, decoded surplus).
The regular path is a MIXED_PLAIN problem assembled with mg_assemble_level and
read back with mg_get_cell_data / mg_get_cell_matrices.  Both are called
through the C ABI; the element matrices rebuilt from the allocation-free
output must match the regular ones within the mixed-assembly tolerance
(1e-5 of each cell's largest entry), the classes and eps exactly.  Two calls
run back to back on different cell ranges (the scratch array is shared by
every call).  This file is collected last on purpose: it must pass both alone
in a fresh process and after every other test.
"""
import numpy as np
import pytest

from paper_2005_03606_gb300 import inputs, mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_03606_gb300 import build
    build.build()
    return mg.load()


def _kref_off(dim, ham):
    if dim == 2:
        return -1.0 / 6.0 if ham == 1 else -1.0 / 3.0
    return 0.0 if ham == 1 else -1.0 / 12.0


def _rebuild(dim, n, eps_c, surplus):
    """Element matrices of the cells from eps_c (their own) and the surplus."""
    nv = 1 << dim
    hfac = 1.0 / n if dim == 3 else 1.0
    A = np.zeros((eps_c.shape[0], nv, nv))
    p = 0
    for a in range(nv):
        for b in range(a + 1, nv):
            v = eps_c * hfac * _kref_off(dim, bin(a ^ b).count("1")) + surplus[:, p]
            A[:, a, b] = v
            A[:, b, a] = v
            p += 1
    A[:, np.arange(nv), np.arange(nv)] = -A.sum(axis=2)
    return A


def _noalloc(fld, dim, n, s, cell0, ncell, stream):
    npairs = 6 if dim == 2 else 28
    eps_c = torch.empty(n ** dim, dtype=torch.float32, device="cuda")
    cls = torch.empty(ncell, dtype=torch.uint8, device="cuda")
    sur = torch.empty(ncell * npairs, dtype=torch.float32, device="cuda")
    mg.assemble_surplus_noalloc(fld, dim, n, s, cell0, ncell, eps_c.data_ptr(), cls.data_ptr(), sur.data_ptr(),
                                stream=stream)
    return eps_c, cls, sur.view(ncell, npairs)


def _regular(fld, dim, n, s, cells):
    with mg.Problem(mg.problem_desc(dim, n, fld, path=mg.PATH_MIXED_PLAIN, s_schedule=(s,))) as P:
        P.assemble(s)
        cls, ec = P.cell_data()
        A = P.cell_matrices(cells)
    return cls, ec, A


CASES = [
    # dim, n, field, s, (cell0_rows, nrows) of the two back-to-back calls
    (3, 27, inputs.boxes_field(3, 2003), 8, [(0, 27 * 27), (9 * 27 + 5, 300)]),
    (2, 81, inputs.disc_field(2), 8, [(0, 81), (17, 40)]),
    (3, 27, inputs.fourier_field(3, 15, sigma=2.0, jump_x=0.37, jump_factor=1e4), 4, [(27 * 10, 27 * 7), (0, 1)]),
    # one sample per cell: the surplus is zero by definition (the early-return branch)
    (3, 27, inputs.boxes_field(3, 2003), 1, [(0, 27 * 27), (5 * 27, 27)]),
]


@pytest.mark.parametrize("dim,n,fld,s,ranges", CASES)
def test_noalloc_matches_regular_assembly(dim, n, fld, s, ranges):
    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for row0, nrows in ranges:            # two calls in a row, nothing in between
        outs.append((row0 * n, nrows * n, _noalloc(fld, dim, n, s, row0 * n, nrows * n, stream)))
    torch.cuda.synchronize()
    ref_cls, ref_ec, _ = _regular(fld, dim, n, s, np.zeros(1, np.int64))
    for cell0, ncell, (eps_c, cls, sur) in outs:
        ec = eps_c.cpu().numpy().astype(np.float64)
        assert np.array_equal(ec, ref_ec)
        c = cls.cpu().numpy()
        assert np.array_equal(c, ref_cls[cell0:cell0 + ncell])
        cells = np.arange(cell0, cell0 + ncell, dtype=np.int64)
        _, _, A_ref = _regular(fld, dim, n, s, cells)
        A = _rebuild(dim, n, ec[cells], sur.cpu().numpy().astype(np.float64))
        den = np.abs(A_ref).max(axis=(1, 2))
        err = (np.abs(A - A_ref).max(axis=(1, 2)) / den).max()
        assert err <= TOL, err
        s_np = sur.cpu().numpy()
        assert np.all(s_np[c == 0] == 0.0)
        if s == 1:
            assert not c.any() and not s_np.any()


def test_noalloc_rejects_ranges_beyond_scratch():
    n = 243
    fld = inputs.boxes_field(3, 2003)
    dummy = torch.empty(16, dtype=torch.uint8, device="cuda")
    p = dummy.data_ptr()
    with pytest.raises(mg.MGError) as ei:    # 243^3 cells need far more than the 64 MiB scratch
        mg.assemble_surplus_noalloc(fld, 3, n, 8, 0, n ** 3, p, p, p)
    assert ei.value.status == mg.MG_ERR_INVALID
    assert "scratch" in str(ei.value)
    with pytest.raises(mg.MGError) as ei:    # not whole x-rows
        mg.assemble_surplus_noalloc(fld, 3, 27, 8, 5, 27, p, p, p)
    assert ei.value.status == mg.MG_ERR_INVALID
    with pytest.raises(mg.MGError) as ei:    # row-aligned start, ragged length
        mg.assemble_surplus_noalloc(fld, 3, 27, 8, 27, 40, p, p, p)
    assert ei.value.status == mg.MG_ERR_INVALID
    with pytest.raises(mg.MGError) as ei:    # accuracy beyond 64 samples per axis
        mg.assemble_surplus_noalloc(fld, 3, 27, 65, 0, 27, p, p, p)
    assert ei.value.status == mg.MG_ERR_INVALID
