"""The paper's truncated storage format on the GPU against the oracle.

mg_paper_format encodes the surplus A - eps_c K of every finest-level cell of
a problem's stored operator with the paper's format (Section "Precision
toggling and information density"; sign bit, truncated mantissa, signed-char
exponent, p3 bytes per entry chosen against an absolute threshold delta).
The oracle (oracle.paper_format) is given the same A (read back through the
C ABI), the same eps_c and the same K: K_ref h^(d-2) from its closed form,
entry by entry rounded to FP64 (2/3, -1/6, -1/3 in 2D; 1/3, 0, -1/12 times 1/N
in 3D), which the test checks against the oracle's integrated K_ref.  The
choice of p3 is then decided on identical FP64 numbers on both sides, and it
must be: truncation toward zero makes it hinge on the last bit (a surplus
that is a short dyadic fraction fits two bytes, the same value one ulp lower
needs five), so p3 and the decoded matrices are compared exactly, together
with the statistics and the error bound |stored - A| <= delta.
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


def _kref_closed(dim, n):
    nv = 1 << dim
    K = np.zeros((nv, nv))
    for a in range(nv):
        for b in range(nv):
            ham = bin(a ^ b).count("1")
            if dim == 2:
                k = 2.0 / 3.0 if ham == 0 else (-1.0 / 6.0 if ham == 1 else -1.0 / 3.0)
                K[a, b] = k
            else:
                k = 1.0 / 3.0 if ham == 0 else (0.0 if ham == 1 else -1.0 / 12.0)
                K[a, b] = k * (1.0 / n)
    return K


def _check(dim, n, fld, path, s, delta):
    with mg.Problem(mg.problem_desc(dim, n, fld, path=path, s_schedule=(s,))) as P:
        P.assemble(s)
        A = P.element_matrices(0)
        _, ec = P.cell_data()
        p3, At, st = P.paper_format(delta, decoded=True)
    K = _kref_closed(dim, n)
    assert np.abs(K - oracle.kref(dim, n)).max() <= 1e-15 * np.abs(K).max()
    p_or, At_or = oracle.paper_format(dim, A, ec, K, delta)
    assert np.array_equal(p3.astype(np.int32), p_or)
    assert np.array_equal(At, At_or)
    assert np.abs(At - A).max() <= delta
    assert st["max_abs_error"] == np.abs(At - A).max()
    assert st["cells_by_p3"] == [int((p3 == k).sum()) for k in range(9)]
    assert st["cells_by_p3"][1] == 0
    assert st["compression"] == pytest.approx(oracle.paper_compression(dim, p_or), rel=1e-14)
    return p3, st


CASES = [
    (2, 27, inputs.theta_field(2, 16.0), mg.PATH_FP64_PLAIN, 4, 1e-8),
    (2, 81, inputs.disc_field(2), mg.PATH_FP64_PLAIN, 8, 1e-8),
    (3, 9, inputs.fourier_field(3, 13, sigma=1.0), mg.PATH_FP64_PLAIN, 4, 1e-8),
    (3, 27, inputs.boxes_field(3, 14), mg.PATH_MIXED_PLAIN, 4, 1e-8),
    (2, 27, inputs.theta_field(2, 64.0), mg.PATH_FP64_PLAIN, 8, 1e-12),
    (3, 9, inputs.fourier_field(3, 13, sigma=1.0), mg.PATH_FP64_PLAIN, 4, 1e-4),
]


@pytest.mark.parametrize("dim,n,fld,path,s,delta", CASES)
def test_paper_format_matches_oracle(dim, n, fld, path, s, delta):
    p3, st = _check(dim, n, fld, path, s, delta)
    assert len(np.unique(p3)) >= 2      # the cases exercise more than one width


def test_paper_format_constant_field_is_all_markers():
    for dim, n, full in ((2, 27, 128.0), (3, 9, 512.0)):
        with mg.Problem(mg.problem_desc(dim, n, inputs.const_field(dim, 2.5), path=mg.PATH_FP64_PLAIN,
                                        s_schedule=(4,))) as P:
            P.assemble(4)
            p3, _, st = P.paper_format(1e-8)
        assert np.all(p3 == 0) and st["compression"] == full


def test_paper_format_widths_shrink_with_the_threshold():
    fld = inputs.theta_field(2, 16.0)
    with mg.Problem(mg.problem_desc(2, 27, fld, path=mg.PATH_FP64_PLAIN, s_schedule=(8,))) as P:
        P.assemble(8)
        widths = [P.paper_format(d)[0].astype(int) for d in (1e-14, 1e-10, 1e-6, 1e-2)]
    for a, b in zip(widths, widths[1:]):
        assert np.all(b <= a)
    assert widths[0].sum() > widths[-1].sum()


def test_paper_format_rejects_bad_threshold():
    with mg.Problem(mg.problem_desc(2, 27, inputs.const_field(2), path=mg.PATH_FP64_PLAIN)) as P:
        for bad in (-1.0, float("nan"), float("inf")):
            with pytest.raises(mg.MGError) as ei:
                P.paper_format(bad)
            assert ei.value.status == mg.MG_ERR_INVALID


E2E_CASES = [
    (2, 27, inputs.theta_field(2, 16.0), 4, 1e-8),
    (2, 81, inputs.disc_field(2), 8, 1e-8),
    (3, 9, inputs.fourier_field(3, 13, sigma=1.0), 4, 1e-8),
    (2, 27, inputs.theta_field(2, 64.0), 8, 1e-12),
]


@pytest.mark.parametrize("dim,n,fld,s,delta", E2E_CASES)
def test_paper_format_end_to_end_from_oracle_matrices(dim, n, fld, s, delta):
    """The whole chain against the oracle alone: the oracle assembles the FP64
    element matrices, takes eps at the cell centres and encodes them; the GPU
    assembles, encodes and decodes its own.  The decoded GPU matrices must
    represent the oracle's exact matrices within delta plus the FP64 assembly
    tolerance, and the byte choices may differ only in cells whose choice
    flips within that tolerance (truncation makes it hinge on the last bit):
    there the GPU's choice must be the oracle's choice for the GPU's own A."""
    with mg.Problem(mg.problem_desc(dim, n, fld, path=mg.PATH_FP64_PLAIN, s_schedule=(s,))) as P:
        P.assemble(s)
        A_gpu = P.element_matrices(0)
        p3, At, _ = P.paper_format(delta, decoded=True)
    f = oracle.Field(fld)
    A_or = oracle.assemble(f, n, s)
    cc = np.indices((n,) * dim).reshape(dim, -1)[::-1].T          # cell index, x fastest
    ec = np.array([oracle.eps_at(f, [oracle.sample_coord(n, 1, int(i), 0) for i in c]) for c in cc])
    K = _kref_closed(dim, n)
    p_or, At_or = oracle.paper_format(dim, A_or, ec, K, delta)
    scale = np.abs(A_or).max()
    assert np.abs(A_gpu - A_or).max() <= 1e-12 * scale
    assert np.abs(At - A_or).max() <= delta + 2e-12 * scale
    assert np.abs(At_or - A_or).max() <= delta
    diff = np.nonzero(p3.astype(np.int32) != p_or)[0]
    assert diff.size <= max(2, 0.02 * p3.size), diff.size
    if diff.size:
        p_own, _ = oracle.paper_format(dim, A_gpu[diff], ec[diff], K, delta)
        assert np.array_equal(p3[diff].astype(np.int32), p_own)


def test_memory_footprint_table_theta1_column_under_keep_old():
    # Table "memory-footprint", theta = 1: one accuracy step n -> n + 1 per
    # cycle with C = 1%; under the keep-old reading every cell keeps n = 1 and
    # only its one-byte marker: max n 1, average 1.00, compression 128.00 in all
    # ten cycles, as printed
    # (the descriptor's schedule holds at most 8 levels; mg_assemble_level takes any s)
    d = mg.problem_desc(2, 27, inputs.theta_field(2, 1.0), path=mg.PATH_FP64_PLAIN, s_schedule=tuple(range(1, 9)),
                        adapt_C=0.01, adapt_keep=1)
    with mg.Problem(d) as P:
        for s in range(1, 11):
            if s > 1:
                P.assemble(s)
            acc = P.cell_accuracy()
            _, _, st = P.paper_format(1e-8)
            assert acc.max() == 1 and st["compression"] == 128.0
