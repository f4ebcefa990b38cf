"""Adaptive per-cell accuracy on the GPU against the oracle.

Section "Adaptive stencil integration": each cell walks the accuracy schedule
and keeps the first matrix whose relative change against the previous level's
matrix (element-wise maximum norm) is below C.  The oracle
(oracle.assemble_adaptive) compares exact FP64 matrices; the GPU compares
against the matrix it stored at the previous level (FP64 on the FP64 paths,
the decoded lossy record on the mixed paths), computed in the kernel's
precision.  So a cell's accuracy is unique only where no change ratio on its
path lies near C: cells with |ratio - C| within the comparison's error band
(1e-10 FP64, 1% of C mixed) may stop one level apart, and there the GPU's choice
must be a level of the schedule whose oracle matrix it holds.  Everywhere
else the accuracies agree exactly and the stored matrices match the oracle's
adaptive matrices within the assembly tolerances (1e-12 FP64, 1e-5 mixed,
relative to each cell's largest entry).
"""
import numpy as np
import pytest

import oracle
from paper_2005_03606_gb300 import inputs, mg

pytestmark = pytest.mark.gpu

C = 1e-2


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2005_03606_gb300 import build
    build.build()
    return mg.load()


def _ratios(F, n, sched):
    """Oracle change ratio of every cell at every judged level, and the
    matrices of every level."""
    mats = [oracle.assemble(F, n, s) for s in sched]
    r = []
    for k in range(1, len(sched)):
        num = np.abs(mats[k] - mats[k - 1]).max(axis=(1, 2))
        den = np.abs(mats[k - 1]).max(axis=(1, 2))
        r.append(num / den)
    return np.stack(r, axis=1), mats


def _check(dim, n, fld, path, sched, chunks, run, C=C, keep=0):
    F = oracle.Field(fld)
    A_ref, s_ref = oracle.assemble_adaptive(F, n, sched, C, keep_old=bool(keep))
    r, mats = _ratios(F, n, sched)
    mixed = path in (mg.PATH_MIXED_PLAIN, mg.PATH_MIXED_DELAYED)
    band, tol = (1e-4 * C / 1e-2, 1e-5) if mixed else (1e-10, 1e-12)
    with mg.Problem(mg.problem_desc(dim, n, fld, path=path, s_schedule=sched, chunks=chunks, adapt_C=C,
                                    adapt_keep=keep)) as P:
        run(P)
        s_gpu = P.cell_accuracy()
        A = P.cell_matrices(np.arange(n ** dim, dtype=np.int64))
    # the oracle's path for each cell: the judged levels up to its stop (under
    # keep-old the stored level is the one before the test that stopped it)
    k_stop = np.searchsorted(np.asarray(sched), s_ref)
    if keep:
        k_stop = np.minimum(k_stop + 1, len(sched) - 1)
    judged = np.arange(1, len(sched))[None, :] <= k_stop[:, None]
    near = (np.abs(r - C) <= band) & judged
    amb = near.any(axis=1)
    assert amb.mean() < 0.05, amb.mean()
    ok = ~amb
    assert np.array_equal(s_gpu[ok], s_ref[ok])
    den = np.abs(A_ref).max(axis=(1, 2))
    err = np.abs(A - A_ref).max(axis=(1, 2)) / den
    assert err[ok].max() <= tol, err[ok].max()
    for c in np.flatnonzero(amb):
        assert s_gpu[c] in sched
        ref = mats[list(sched).index(s_gpu[c])][c]
        assert np.abs(A[c] - ref).max() <= tol * np.abs(ref).max()
    # more than one accuracy in use: the rule did something
    assert len(np.unique(s_ref)) >= 2
    return s_gpu, s_ref


def _assemble_all(sched):
    def run(P):
        for s in sched:
            if s > 1:
                P.assemble(s)
    return run


def _solve(P):
    P.solve()


CASES = [
    # dim, n, field, path, schedule, chunks, how, C
    (2, 81, inputs.disc_field(2), mg.PATH_FP64_PLAIN, (1, 2, 4, 8), 3, "assemble", C),
    (2, 81, inputs.theta_field(2, 16.0), mg.PATH_FP64_DELAYED, (1, 2, 4, 8), 1, "solve", 1e-3),
    (3, 27, inputs.fourier_field(3, 15, sigma=2.0, jump_x=0.37, jump_factor=1e4), mg.PATH_MIXED_PLAIN,
     (1, 2, 3, 4, 6), 3, "assemble", C),
    (3, 27, inputs.boxes_field(3, 14), mg.PATH_MIXED_DELAYED, (2, 4, 8), 0, "solve", C),
    (3, 27, inputs.fourier_field(3, 13, sigma=1.0), mg.PATH_FP64_PLAIN, (2, 4, 8, 16), 0, "solve", C),
    (3, 27, inputs.fourier_field(3, 13, sigma=1.0), mg.PATH_MIXED_DELAYED, (1, 2, 4, 8), 2, "solve", 0.1),
    (3, 27, inputs.disc_field(3), mg.PATH_MIXED_PLAIN, (1, 2, 4), 3, "solve", C),
]


@pytest.mark.parametrize("dim,n,fld,path,sched,chunks,how,c", CASES)
def test_adaptive_accuracy_matches_oracle(dim, n, fld, path, sched, chunks, how, c):
    run = _solve if how == "solve" else _assemble_all(sched)
    _check(dim, n, fld, path, sched, chunks, run, c)


KEEP_CASES = [
    (2, 81, inputs.disc_field(2), mg.PATH_FP64_PLAIN, (1, 2, 4, 8), 3, "assemble", C),
    (2, 81, inputs.theta_field(2, 16.0), mg.PATH_FP64_DELAYED, (1, 2, 4, 8), 1, "solve", 1e-3),
    (3, 27, inputs.fourier_field(3, 15, sigma=2.0, jump_x=0.37, jump_factor=1e4), mg.PATH_MIXED_PLAIN,
     (1, 2, 3, 4, 6), 3, "assemble", C),
    (3, 27, inputs.boxes_field(3, 14), mg.PATH_MIXED_DELAYED, (2, 4, 8), 0, "solve", C),
]


@pytest.mark.parametrize("dim,n,fld,path,sched,chunks,how,c", KEEP_CASES)
def test_adaptive_keep_old_reading_matches_oracle(dim, n, fld, path, sched, chunks, how, c):
    # adapt_keep = 1: a cell that passes the test keeps the matrix it was tested against
    run = _solve if how == "solve" else _assemble_all(sched)
    _check(dim, n, fld, path, sched, chunks, run, c, keep=1)


def test_adaptive_keep_flag_rejected_outside_0_1():
    with pytest.raises(mg.MGError) as ei:
        mg.Problem(mg.problem_desc(2, 27, inputs.disc_field(2), s_schedule=(1, 2), adapt_C=0.01, adapt_keep=2))
    assert ei.value.status == mg.MG_ERR_INVALID


def test_adaptive_off_reports_chunk_accuracy():
    fld = inputs.disc_field(2)
    with mg.Problem(mg.problem_desc(2, 27, fld, path=mg.PATH_FP64_PLAIN, s_schedule=(1, 4))) as P:
        assert np.all(P.cell_accuracy() == 1)
        P.assemble(4)
        assert np.all(P.cell_accuracy() == 4)


def test_adaptive_constant_field_stops_at_first_judged_level():
    fld = inputs.const_field(3, 2.5)
    for path, sched, first in ((mg.PATH_FP64_PLAIN, (1, 2, 4), 2), (mg.PATH_MIXED_PLAIN, (2, 4, 8), 4)):
        with mg.Problem(mg.problem_desc(3, 27, fld, path=path, s_schedule=sched, adapt_C=C)) as P:
            _assemble_all(sched)(P)
            assert np.all(P.cell_accuracy() == first)


def test_adaptive_rejects_bad_C():
    fld = inputs.const_field(2)
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(mg.MGError) as ei:
            mg.Problem(mg.problem_desc(2, 27, fld, s_schedule=(1, 2), adapt_C=bad))
        assert ei.value.status == mg.MG_ERR_INVALID


@pytest.mark.parametrize("path", [mg.PATH_FP64_DELAYED, mg.PATH_MIXED_DELAYED, mg.PATH_FP64_PLAIN])
def test_solve_trace_records_every_iteration(path):
    """Per-iteration telemetry (residual and pending background jobs, the two
    quantities of the paper's starvation experiment)."""
    fld = inputs.disc_field(2, v_in=1e-3, v_out=1.0)
    sched = (1, 2, 4, 8) if path != mg.PATH_FP64_PLAIN else (8,)
    with mg.Problem(mg.problem_desc(2, 81, fld, path=path, s_schedule=sched, chunks=3)) as P:
        info = P.solve()
        tr = P.trace()
        # a second solve replaces the record
        info2 = P.solve()
        tr2 = P.trace()
    assert len(tr) == info.cycles and len(tr2) == info2.cycles
    assert [t["cycle"] for t in tr] == list(range(1, info.cycles + 1))
    pend = [t["pending_jobs"] for t in tr]
    assert all(a >= b for a, b in zip(pend, pend[1:]))          # no job is added during a solve
    assert pend[-1] == 0 and tr[-1]["publishes"] == info.publishes
    if path == mg.PATH_FP64_PLAIN:
        assert max(pend) == 0 and info.publishes == 0
    times = [t["time_ms"] for t in tr]
    assert all(a <= b for a, b in zip(times, times[1:]))
    assert tr[0]["restarted"] == 1
    assert tr[-1]["rel_residual_est"] <= 1e-6
