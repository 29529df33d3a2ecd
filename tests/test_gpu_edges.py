"""Edge cases of the CUDA path against the oracle: the largest velocity set
(Q = 32768), the largest grid (Nz = 4096), the largest expansion order (N = 8),
a zero-step call, and the degenerate Couette problem with resting walls at the
gas temperature, whose rest state is a fixed point of the scheme."""
import numpy as np
import pytest

import workloads as W
from tests._pair import gpu_f, oracle_of, profile_errors, rel_err, same_state, solver_of

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2e-5


def _lbs():
    import paper_1702_01335_gb300 as P
    return P


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_largest_velocity_set(prec):
    """Q = 2 * 16 * 16 * 64 = 32768, the limit: 16384 velocities per half range, so
    dozens of chunks per sign for every V."""
    P = _lbs()
    p = dict(Qx=16, Qy=16, Qz=64, N_eq=4, Nz=7, A=0.5, Kn=0.5, u_w=0.3, T_w=1.0, Pr=2.0 / 3.0,
             visc_law=0, visc_param=1.0)
    o = oracle_of(p, None)
    assert o.Q == 32768
    s = solver_of(p, o.dt, P.LBS_FP64 if prec == "fp64" else P.LBS_FP32)
    o.step(3)
    s.step(3)
    if prec == "fp64":
        assert rel_err(gpu_f(s, o), o.f[3:3 + o.Nz]) < FP64_TOL
    else:
        errs = profile_errors(s.profiles(), o.profiles(), uw=p["u_w"])
        assert max(errs.values()) < FP32_TOL, errs


def test_largest_grid():
    """Nz = 4096 cells (the limit), stretched: thousands of z-tiles per instance."""
    P = _lbs()
    p = dict(W.C1, Nz=4096, A=0.9)
    o = oracle_of(p, None)
    s = solver_of(p, o.dt, P.LBS_FP64)
    o.step(3)
    s.step(3)
    assert rel_err(gpu_f(s, o), o.f[3:3 + o.Nz]) < FP64_TOL


def test_largest_expansion_order():
    """N_eq = 8 on every axis (9 nodes each): the longest coefficient recurrences and
    half-range tables of the finalisation, in both finalisation layouts."""
    P = _lbs()
    p = dict(Qx=9, Qy=9, Qz=9, N_eq=8, Nz=10, A=0.7, Kn=0.2, u_w=0.5, T_w=1.2, Pr=2.0 / 3.0,
             visc_law=1, visc_param=0.3101)
    o = oracle_of(p, None)
    o.step(10)
    for fin in (1, 2):
        s = solver_of(p, o.dt, P.LBS_FP64)
        s.set_finalize(fin)
        s.step(10)
        assert rel_err(gpu_f(s, o), o.f[3:3 + o.Nz]) < FP64_TOL, fin


def test_zero_steps_and_resting_walls():
    """lbs_step(0) changes nothing; with u_w = 0 and T_w = 1 the rest state stays at
    rest (n = 1, u = 0, T = 1) to rounding: the stored deviations stay at the level of
    the FP64 rounding of the equilibrium coefficients.  (The residual is a relative
    change; with u_x zero up to rounding in every cell its u_x part compares rounding
    with rounding, so it is not a measure here.)"""
    P = _lbs()
    p = dict(W.C1, u_w=0.0, A=0.9)
    s = solver_of(p, 0.003, P.LBS_FP64)
    before = s.get_state(0)
    s.step(0)
    assert same_state(s.get_state(0), before)
    s.step(200)
    prof = s.profiles()
    assert np.abs(prof["n"] - 1).max() < 1e-13
    assert np.abs(prof["ux"]).max() < 1e-13
    assert np.abs(prof["T"] - 1).max() < 1e-13
    assert np.abs(s.get_state(0).d).max() < 1e-12
