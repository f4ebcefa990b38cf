"""Failure paths of a solve, made on the host (no device fault, trap or hang).

* A side-stream assembly job that fails (injected on the host before any
  device work for its chunk, mg_inject_assembly_failure) is reported by
  mg_solve as MG_ERR_INJECTED at the next cycle boundary; the problem can
  still be destroyed and the device keeps working.
* A stationary iteration whose smoother amplifies error (damped Jacobi with
  omega = 2.5, beyond the stable range 0 < omega < 2 / lambda_max(D^-1 A))
  trips the divergence guard: MG_ERR_DIVERGED on the FP64 and mixed paths,
  long before the values leave the FP64 range.
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


@pytest.mark.parametrize("path", [mg.PATH_MIXED_DELAYED, mg.PATH_FP64_DELAYED])
@pytest.mark.parametrize("s_fail", [2, 8])
def test_injected_assembly_failure_is_reported(path, s_fail):
    d = mg.problem_desc(3, 27, inputs.boxes_field(3, 2003), path=path, s_schedule=(1, 2, 4, 8))
    with mg.Problem(d) as P:
        P.inject_assembly_failure(s_fail)
        info = P.solve(check=False)
        assert info.status == mg.MG_ERR_INJECTED
        assert "injected" in mg.last_error()
    # the device and the library keep working: the same problem without injection converges
    with mg.Problem(d) as P:
        info = P.solve()
        assert info.status == mg.MG_OK and info.rel_residual <= 2e-8


def test_injection_hook_rejects_bad_arguments():
    d = mg.problem_desc(2, 27, inputs.disc_field(2), path=mg.PATH_MIXED_DELAYED, s_schedule=(1, 2, 4))
    with mg.Problem(d) as P:
        with pytest.raises(mg.MGError) as ei:
            P.inject_assembly_failure(-1)
        assert ei.value.status == mg.MG_ERR_INVALID
        P.inject_assembly_failure(4)
        P.inject_assembly_failure(0)         # off again: the solve converges
        assert P.solve().status == mg.MG_OK


@pytest.mark.parametrize("path", [mg.PATH_FP64_PLAIN, mg.PATH_MIXED_PLAIN])
def test_unstable_smoother_is_reported_as_diverged(path):
    d = mg.problem_desc(2, 81, inputs.disc_field(2), path=path, s_schedule=(8,), omega=2.5,
                        outer=mg.OUTER_RICHARDSON, max_cycles=200)
    with mg.Problem(d) as P:
        info = P.solve(check=False)
        assert info.status == mg.MG_ERR_DIVERGED, (info.status, mg.last_error())
        assert info.cycles < 60
        u = P.solution()
        assert np.isfinite(u).all()
    # a stable omega on the same problem converges
    d.omega = 0.6
    with mg.Problem(d) as P:
        assert P.solve().status == mg.MG_OK
