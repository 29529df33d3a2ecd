"""GPU parity of the reduced phi / chi model (Sec. III, Eqs. reduced_def, boltz_red,
phieq, sred_def; lbs_orders.Qy = 0) against the oracle's reduced model, which is
pinned to the y-integrals of the full model (tests/test_oracle_pins.py)."""
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from tests._pair import gpu_f, oracle_of, profile_errors, rel_err, solver_of

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2e-5
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# several velocity chunks per half range (Q = 4 * 6 * 7 = 168 at V = 1), ragged
# z-tiles, stretched grid, Sutherland viscosity, Shakhov Pr = 2/3
RED = dict(Qx=6, Qy=0, Qz=7, N_eq=4, Nz=37, A=0.9, Kn=0.3, u_w=0.4, T_w=1.1, Pr=2.0 / 3.0,
           visc_law=1, visc_param=0.5239)
# the largest normal order and a uniform grid; Q = 4 * 16 * 64 = 4096
RED_WIDE = dict(Qx=16, Qy=0, Qz=64, N_eq=4, Nz=24, A=0.0, Kn=2.0, u_w=0.2, T_w=1.0, Pr=2.0 / 3.0,
                visc_law=0, visc_param=0.5)


def _lbs():
    import paper_1702_01335_gb300 as P
    return P


@pytest.mark.parametrize("params,steps", [(RED, 30), (RED_WIDE, 12)])
def test_fp64_reduced_state_matches_oracle(params, steps):
    P = _lbs()
    o = oracle_of(params, dt=None)
    assert o.reduced
    s = solver_of(params, o.dt, P.LBS_FP64)
    assert s.info()["Q"] == o.Q
    o.step(steps)
    s.step(steps)
    assert rel_err(gpu_f(s, o), o.f[3:3 + o.Nz]) < FP64_TOL
    errs = profile_errors(s.profiles(), o.profiles())
    assert max(errs.values()) < FP64_TOL, sorted(errs.items(), key=lambda kv: -kv[1])
    p = s.profiles()
    for k in ("uy", "qy", "Pxy", "Pyz"):
        assert np.all(p[k] == 0.0), k


def test_fp32_reduced_profiles_match_oracle():
    P = _lbs()
    o = oracle_of(RED, dt=None)
    s = solver_of(RED, o.dt, P.LBS_FP32)
    o.step(40)
    s.step(40)
    errs = profile_errors(s.profiles(), o.profiles(), uw=RED["u_w"])
    assert max(errs.values()) < FP32_TOL, sorted(errs.items(), key=lambda kv: -kv[1])
    dz = np.diff(o.xf)
    assert abs(np.sum(s.profiles()["n"] * dz) - 1.0) < 1e-6


@pytest.mark.parametrize("fin", [1, 2])
@pytest.mark.parametrize("V,ZT,fuse", [(1, 3, 1), (2, 7, 0), (4, 12, 2)])
def test_reduced_tilings_and_finalisation_layouts(V, ZT, fuse, fin):
    """Every work decomposition gives the oracle's reduced state; a batch of three
    instances so that split stepping has two halves."""
    P = _lbs()
    o = oracle_of(RED, dt=None)
    s = solver_of([RED] * 3, o.dt, P.LBS_FP64)
    s.set_tiling(V, ZT, fuse)
    s.set_finalize(fin)
    o.step(15)
    s.step(15)
    for b in (0, 2):
        assert rel_err(gpu_f(s, o, b), o.f[3:3 + o.Nz]) < FP64_TOL, b


def test_reduced_half_channel_is_upper_half_of_full_channel():
    """Bounce-back on the centre line with phi and chi: each field mirrors onto itself."""
    P = _lbs()
    from paper_1702_01335_gb300 import Instance, Solver
    S = 19
    o = oracle_of(dict(RED, Nz=2 * S), dt=None)
    s = Solver([Instance(dt=o.dt, half=1, **dict(RED, Nz=S))], precision=P.LBS_FP64)
    o.step(40)
    s.step(40)
    f_gpu = s.populations() * o.weights()[None, :]
    assert rel_err(f_gpu, o.f[3 + S:3 + 2 * S]) < FP64_TOL
    p_ora = {k: v[S:] for k, v in o.profiles().items()}
    errs = profile_errors(s.profiles(), p_ora)
    assert max(errs.values()) < FP64_TOL, errs


def test_reduced_warm_start_and_static_moments():
    """lbs_init_from_profiles seeds phi_eq (1 + S_phi) and T phi_eq (1 + S_chi) as the
    oracle does, and the allocation-free moments of a reduced state equal lbs_profiles."""
    P = _lbs()
    import torch
    o = oracle_of(RED, dt=None)
    s = solver_of(RED, o.dt, P.LBS_FP64)
    z = o.xc[3:3 + o.Nz]
    prof = np.zeros((8, o.Nz))
    prof[0] = 1.0 + 0.05 * np.cos(np.pi * z)
    prof[1] = 0.8 * RED["u_w"] * 2 * z
    prof[2] = 1.0 + 0.1 * (0.25 - z ** 2)
    prof[3] = 0.01 * z
    prof[4] = -0.02 * z
    s.init_from_profiles(0, prof)
    u = np.zeros((3, o.Nz)); u[0] = prof[1]
    q = np.zeros((3, o.Nz)); q[0] = prof[3]; q[2] = prof[4]
    o.init_from_moments(prof[0], u, prof[2], q)
    assert rel_err(gpu_f(s, o), o.f[3:3 + o.Nz]) < FP64_TOL
    o.step(10)
    s.step(10)
    assert rel_err(gpu_f(s, o), o.f[3:3 + o.Nz]) < FP64_TOL
    ref = s.profiles()
    f_dev = torch.empty((RED["Nz"], s.instances[0].Q), dtype=torch.float64, device="cuda")
    s.get_state_device(0, f_dev.data_ptr())
    out = torch.zeros((14, RED["Nz"]), dtype=torch.float64, device="cuda")
    s.moments_static(0, f_dev.data_ptr(), out.data_ptr())
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for a, k in enumerate(P.PROFILE_NAMES):
        assert np.allclose(got[a], ref[k], rtol=1e-12, atol=1e-14), k


def _printed(label):
    rows = json.load(open(os.path.join(GOLDEN, "paper_tables.json")))["table"]
    hit = [r for r in rows if r["gas"] == label["gas"] and r["delta"] == label["delta"]
           and abs(r["uw"] - label["uw"]) < 1e-12]
    assert len(hit) == 1, label
    return hit[0]


def test_reduced_paper_tables_lb_columns():
    """The paper's own model reproduces every LB entry of Tables gradu, shear and temp
    with delta >= 0.1 (44 printed numbers): one FP32 batch of the 20 half channels,
    120000 steps, the bars of tests/test_gpu_half_channel.py."""
    P = _lbs()
    from paper_1702_01335_gb300 import Instance, Solver
    runs = W.paper_tables(reduced=True)
    s = Solver([Instance(**p) for _, p in runs], precision=P.LBS_FP32)
    assert s.instances[0].Q == 4 * 7 * 30 and s.instances[2].Q == 4 * 7 * 7
    s.step(120000)
    bad = []
    for b, (label, _) in enumerate(runs):
        r, d = _printed(label), s.diagnostics(b)
        if "nu" in r and abs(d["nu"] - r["nu"]) > 1.0e-3 + 5e-4:
            bad.append((label, "nu", d["nu"], r["nu"]))
        half_digit = 0.5 * 10.0 ** (math.floor(math.log10(r["Pi"])) - 3)
        if abs(d["Pi"] - r["Pi"]) > 1e-3 * r["Pi"] + half_digit:
            bad.append((label, "Pi", d["Pi"], r["Pi"]))
        if "T0" in r and abs(d["T0"] - r["T0"]) > 1e-3 * r["T0"] + 5e-4:
            bad.append((label, "T0", d["T0"], r["T0"]))
    assert not bad, bad
