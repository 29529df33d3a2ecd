"""Failure detection on the GPU without a GPU fault: every failure here is one the
kernels or the host report as a status, and the context stays usable after each.

  * a bounded wait that runs out: the stage kernel's wait for its bulk copies is
    given a limit of zero spins, so every CTA gives up at once, flags the instance,
    lets its copies land and leaves; the next status check returns LBS_ERR_TIMEOUT,
    and after lbs_clear_status and lbs_set_state the solver steps exactly as a fresh one;
  * a residual target that is not reached within max_steps: LBS_ERR_NO_CONVERGENCE;
  * arithmetic blow-up: a time step far above the RK-3 / WENO-5 stability limit drives
    the state to infinity and NaN, and the finalisation flags it (LBS_ERR_NONFINITE).
"""
import numpy as np
import pytest

import workloads as W
from tests._pair import oracle_of, solver_of

pytestmark = pytest.mark.gpu


def _lbs():
    import paper_1702_01335_gb300 as P
    return P


def test_bounded_wait_runs_out_and_reports_timeout():
    P = _lbs()
    p = W.C1  # Q = 128: rows 16-byte aligned, staged by bulk copies
    dt = oracle_of(p, None).dt
    s = solver_of(p, dt, P.LBS_FP32)
    ref = solver_of(p, dt, P.LBS_FP32)
    s.step(5)
    ref.step(5)
    saved = s.get_state(0)
    s.set_wait_limit(0)
    s.step(1)
    with pytest.raises(P.LbsError) as e:
        s.residual()
    assert e.value.status == P.LBS_ERR_TIMEOUT
    assert "bounded wait" in str(e.value)
    # the context and the handle stay usable: restore the limit, the status and the state
    s.set_wait_limit(1 << 26)
    s.clear_status()
    s.set_state(0, saved)
    s.step(7)
    ref.step(7)
    # the resumed run starts from records of the state's own moments (the analysis pass,
    # FP32 sums) instead of the moments the last step took about the cell velocities,
    # equal to FP32 rounding: the states agree to that, not bit for bit
    a, b = s.populations(), ref.populations()
    assert np.abs(a - b).max() < 1e-6 * np.abs(b).max()
    assert abs(s.residual() / ref.residual() - 1.0) < 1e-3


def test_run_to_steady_reports_no_convergence():
    P = _lbs()
    p = W.C1
    s = solver_of(p, oracle_of(p, None).dt, P.LBS_FP64)
    with pytest.raises(P.LbsError) as e:
        s.run_to_steady(1e-8, max_steps=50, check_every=10)
    assert e.value.status == P.LBS_ERR_NO_CONVERGENCE
    steps = s.run_to_steady(1e-8, max_steps=50, check_every=10, raise_on_fail=False)
    assert steps[0] == 50
    assert s.steps_taken() == 100


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_unstable_time_step_reports_nonfinite(precision):
    """dt = 20 x the CFL step of C1: the upwind scheme's amplification factor exceeds 1
    on the shortest waves, which grow until the state overflows; the finalisation
    flags the cell and the next status check returns LBS_ERR_NONFINITE."""
    P = _lbs()
    p = W.C1
    dt = 20.0 * oracle_of(p, None).dt
    s = solver_of(p, dt, P.LBS_FP64 if precision == "fp64" else P.LBS_FP32)
    blew_up = False
    for _ in range(200):
        s.step(10)
        try:
            s.residual()
        except P.LbsError as e:
            assert e.status == P.LBS_ERR_NONFINITE
            blew_up = True
            break
    assert blew_up
    # a fresh solver on the same device still works
    t = solver_of(p, dt / 20.0, P.LBS_FP64)
    t.step(3)
    assert np.isfinite(t.residual())
