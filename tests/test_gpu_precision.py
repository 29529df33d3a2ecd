"""FP32 storage with FP64 moment sums: the error of every macroscopic profile against
the FP64 oracle, stated as a number and bounded by 1e-5 relative to the profile's
scale: its own maximum, except velocities (the Couette scale max(max |u_x|, u_w)) and
heat fluxes (n T^(3/2)).  Both the bounded numbers and the errors relative to each
profile's own maximum are printed for the record."""
import numpy as np
import pytest

import workloads as W
from tests._pair import oracle_of, profile_errors, solver_of

pytestmark = pytest.mark.gpu

BOUND = 1e-5
PROFILES8 = ("n", "ux", "T", "qx", "qz", "Pxx", "Pxz", "Pzz")


def _report(name, errs, s=None, o=None, own=None):
    worst = max(errs[k] for k in PROFILES8)
    if own is not None:
        print("\n[fp32 vs fp64 oracle, own-maximum scale] %s: %s" % (
            name, ", ".join("%s %.1e" % (k, own[k]) for k in PROFILES8)))
    extra = ""
    if s is not None:
        dz = np.diff(o.xf)
        extra = "; mass drift fp32 %.1e, oracle %.1e" % (np.sum(s.profiles()["n"] * dz) - 1.0,
                                                          np.sum(o.profiles()["n"] * dz) - 1.0)
    print("\n[fp32 vs fp64 oracle] %s: %s; worst %.2e%s" % (
        name, ", ".join("%s %.1e" % (k, errs[k]) for k in PROFILES8), worst, extra))
    return worst


def test_fp32_error_c1_steady_state():
    """C1 marched to the oracle's steady state (R < 1e-8)."""
    import paper_1702_01335_gb300 as P
    o = oracle_of(W.C1, None)
    steps, R = o.run_to_steady(1e-8, chunk=100)
    s = solver_of(W.C1, o.dt, P.LBS_FP32)
    s.step(steps)
    gp, op = s.profiles(), o.profiles()
    worst = _report("C1 steady (%d steps)" % steps, profile_errors(gp, op, W.C1["u_w"]), s, o,
                    profile_errors(gp, op))
    assert worst < BOUND


def test_fp32_error_c2_2000_steps():
    import paper_1702_01335_gb300 as P
    o = oracle_of(W.C2, None)
    o.step(2000)
    s = solver_of(W.C2, o.dt, P.LBS_FP32)
    s.step(2000)
    gp, op = s.profiles(), o.profiles()
    worst = _report("C2 after 2000 steps", profile_errors(gp, op, W.C2["u_w"]), s, o, profile_errors(gp, op))
    assert worst < BOUND


def test_fp32_error_c3_60_steps():
    import paper_1702_01335_gb300 as P
    o = oracle_of(W.C3, None)
    o.step(60)
    s = solver_of(W.C3, o.dt, P.LBS_FP32)
    s.step(60)
    gp, op = s.profiles(), o.profiles()
    worst = _report("C3 after 60 steps", profile_errors(gp, op, W.C3["u_w"]), s, o, profile_errors(gp, op))
    assert worst < BOUND
