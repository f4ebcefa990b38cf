"""Additive cycles (Section "adaFAC-x") on the GPU against the oracle.

One application of the plain additive cycle, adaFAC-PI and adaFAC-Jac to a
random fine residual, through mg_vcycle_apply, against oracle.additive_once
on the same stored fine operator (the oracle recomputes the Galerkin levels).
Tolerances as for the V-cycle: 1e-11 relative on the FP64 path, 1e-4 on the
mixed path (FP32 vectors and operators; the oracle gets the decoded stored
operator).  Then whole solves with each cycle under flexible CG and
Richardson reach the residual target on their own operator.
"""
import numpy as np
import pytest

import oracle
from oracle import dense
from paper_2005_03606_gb300 import inputs, mg

pytestmark = pytest.mark.gpu

VARIANTS = [(mg.CYCLE_ADDITIVE, oracle.ADDITIVE), (mg.CYCLE_ADAFAC_PI, oracle.ADAFAC_PI),
            (mg.CYCLE_ADAFAC_JAC, oracle.ADAFAC_JAC)]


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2005_03606_gb300 import build
    build.build()
    return mg.load()


def _stored_operator(path, fld, n, s):
    f = oracle.Field(fld)
    A = oracle.assemble(f, n, s)
    if path in (mg.PATH_MIXED_PLAIN, mg.PATH_MIXED_DELAYED):
        A, _, _ = oracle.compress(f, n, A, 1e-6)
    return A


@pytest.mark.parametrize("cycle,variant", VARIANTS)
@pytest.mark.parametrize("path", [mg.PATH_FP64_PLAIN, mg.PATH_MIXED_PLAIN])
@pytest.mark.parametrize("dim,n,fld", [(2, 81, inputs.disc_field(2)), (3, 27, inputs.fourier_field(3, 35, sigma=1.0)),
                                       (3, 27, inputs.boxes_field(3, 31))])
def test_additive_cycle_matches_oracle(cycle, variant, path, dim, n, fld):
    A = _stored_operator(path, fld, n, 4)
    with mg.Problem(mg.problem_desc(dim, n, fld, path=path, s_schedule=(4,), cycle=cycle)) as P:
        P.assemble(4)
        b = np.random.default_rng(8).standard_normal((n + 1) ** dim) * dense.interior_mask(dim, n)
        e = P.vcycle_apply(b)
    e_ref = oracle.additive_once(dim, n, A, b, 0.6, variant)
    tol = 1e-11 if path == mg.PATH_FP64_PLAIN else 1e-4
    assert np.abs(e - e_ref).max() <= tol * np.abs(e_ref).max()


@pytest.mark.parametrize("cycle", [mg.CYCLE_ADDITIVE, mg.CYCLE_ADAFAC_PI, mg.CYCLE_ADAFAC_JAC])
@pytest.mark.parametrize("path", [mg.PATH_FP64_PLAIN, mg.PATH_MIXED_DELAYED])
def test_additive_solves_converge(cycle, path):
    w = inputs.workload("disc2d")
    sched = (8,) if path == mg.PATH_FP64_PLAIN else (1, 2, 4, 8)
    d = mg.problem_desc(2, 81, w.eps, path=path, s_schedule=sched, rtol=1e-8, cycle=cycle, max_cycles=2000)
    with mg.Problem(d) as P:
        info = P.solve()
        u = P.solution()
    assert info.status == mg.MG_OK and info.rel_residual <= 2e-8
    if path == mg.PATH_FP64_PLAIN:
        A = oracle.assemble(oracle.Field(w.eps), 81, 8)
        f = oracle.load_vector(2, 81)
        assert np.linalg.norm(oracle.residual(2, 81, A, f, u)) <= 3e-8 * np.linalg.norm(f)


def test_adafac_richardson_converges():
    # the damped additive schemes as stationary solvers (u += B (f - A u)), the
    # paper's use of them
    w = inputs.workload("disc2d")
    for cycle in (mg.CYCLE_ADAFAC_PI, mg.CYCLE_ADAFAC_JAC):
        d = mg.problem_desc(2, 81, w.eps, path=mg.PATH_FP64_PLAIN, s_schedule=(8,), rtol=1e-8, cycle=cycle,
                            outer=mg.OUTER_RICHARDSON, max_cycles=3000)
        with mg.Problem(d) as P:
            info = P.solve(check=False)
        assert info.status == mg.MG_OK, (cycle, info.status, info.cycles, info.rel_residual)


def test_unknown_cycle_rejected():
    with pytest.raises(mg.MGError) as ei:
        mg.Problem(mg.problem_desc(2, 27, inputs.const_field(2), cycle=7))
    assert ei.value.status == mg.MG_ERR_INVALID
