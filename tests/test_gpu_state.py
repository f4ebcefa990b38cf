"""Checkpoint export and import of a problem's state through the C ABI.

A state exported from one problem and imported into a fresh problem of the
same descriptor must reproduce the stored operator (decoded element matrices
equal bit for bit), the solution, the per-cell accuracies, and the rest of
the solve (the same cycles and the same solution within round-off of the
restart).  Buffers that do not belong to a compatible problem are rejected
before anything changes.
"""
import numpy as np
import pytest

from paper_2005_03606_gb300 import inputs, mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2005_03606_gb300 import build
    build.build()
    return mg.load()


CASES = [
    dict(dim=3, n=27, fld=inputs.fourier_field(3, 15, sigma=1.0), path=mg.PATH_FP64_DELAYED, sched=(1, 2, 4)),
    dict(dim=3, n=27, fld=inputs.boxes_field(3, 14), path=mg.PATH_MIXED_DELAYED, sched=(1, 2, 4, 8), adapt=1e-2),
    dict(dim=2, n=243, fld=inputs.disc_field(2), path=mg.PATH_MIXED_PLAIN, sched=(8,)),
]


def _desc(c, **kw):
    return mg.problem_desc(c["dim"], c["n"], c["fld"], path=c["path"], s_schedule=c["sched"],
                           adapt_C=c.get("adapt", 0.0), chunks=3, **kw)


@pytest.mark.parametrize("c", CASES)
def test_state_round_trip_after_a_solve(c):
    with mg.Problem(_desc(c)) as P:
        P.solve()
        st = P.export_state()
        A1, u1, s1 = P.element_matrices(0), P.solution(), P.cell_accuracy()
    with mg.Problem(_desc(c)) as Q:
        Q.import_state(st)
        assert np.array_equal(Q.element_matrices(0), A1)
        assert np.array_equal(Q.solution(), u1)
        assert np.array_equal(Q.cell_accuracy(), s1)
        info = Q.solve()    # already converged on the imported operator
        assert info.status == mg.MG_OK and info.cycles <= 1
        assert np.abs(Q.solution() - u1).max() <= 1e-7 * np.abs(u1).max()


@pytest.mark.parametrize("c", CASES[2:])
def test_resume_in_the_middle_of_a_solve(c):
    with mg.Problem(_desc(c, rtol=1e-9)) as P:
        P.assemble(c["sched"][-1])
        P.vcycle(4)
        st = P.export_state()
        ref = P.solve()
        u_ref = P.solution()
    with mg.Problem(_desc(c, rtol=1e-9)) as Q:
        Q.import_state(st)
        info = Q.solve()
        u = Q.solution()
    assert info.status == mg.MG_OK
    assert abs(info.cycles - ref.cycles) <= 1
    assert np.abs(u - u_ref).max() <= 1e-8 * np.abs(u_ref).max()


def test_incompatible_states_are_rejected():
    c = CASES[2]
    with mg.Problem(_desc(c)) as P:
        P.assemble(8)
        st = P.export_state()
        with pytest.raises(mg.MGError) as ei:     # too small a buffer for export
            n = mg.ctypes.c_size_t(0)
            buf = mg.ctypes.create_string_buffer(16)
            mg._check(mg.load().mg_export_state(P.h, buf, 16, mg.ctypes.byref(n)))
        assert ei.value.status == mg.MG_ERR_INVALID
        A = P.element_matrices(0)
        for bad in (st[:-1], st + b"\\0", b"XX" + st[2:]):
            with pytest.raises(mg.MGError) as ei:
                P.import_state(bad)
            assert ei.value.status == mg.MG_ERR_INVALID
        assert np.array_equal(P.element_matrices(0), A)     # nothing changed
    other = dict(c, n=81)
    with mg.Problem(_desc(other)) as Q:
        with pytest.raises(mg.MGError) as ei:
            Q.import_state(st)
        assert ei.value.status == mg.MG_ERR_INVALID
