"""The low-Mach workload of Sec. IV (Table luo): the phi / chi model on the half
channel with u_w = 1e-5, BGK, tau = k / sqrt 2, HLB(1;2) along the flow.  Its
comparison data (linearised-Boltzmann benchmarks) are not available, so the
checks are parity with the oracle and the linear scaling that defines the regime.
The deviations from the rest state are 1e-5 of the populations, below what FP32
storage resolves, so these runs are FP64."""
import numpy as np
import pytest

import workloads as W
from tests._pair import oracle_of, profile_errors, rel_err

pytestmark = pytest.mark.gpu


def _run(k):
    return [p for lab, p in W.luo_runs() if lab["k"] == k][0]


def test_lowmach_half_channel_matches_oracle():
    """k = 0.1 (Q = 4 * 2 * 7, S = 32): the FP64 half channel against the upper half of
    the oracle's full channel.  Velocities and stresses are compared on the scale of
    u_w, i.e. on the deviations themselves."""
    import paper_1702_01335_gb300 as P
    from paper_1702_01335_gb300 import Instance, Solver
    p = _run(0.1)
    S = p["Nz"]
    full = {k: v for k, v in p.items() if k != "half"}
    o = oracle_of(dict(full, Nz=2 * S), dt=None)
    s = Solver([Instance(dt=o.dt, **p)], precision=P.LBS_FP64)
    o.step(300)
    s.step(300)
    f_gpu = s.populations() * o.weights()[None, :]
    f_ora = o.f[3 + S:3 + 2 * S]
    assert rel_err(f_gpu, f_ora) < 1e-13
    po = {k: v[S:] for k, v in o.profiles().items()}
    pg = s.profiles()
    uw = p["u_w"]
    for k in ("ux", "Pxz", "qx"):
        assert np.abs(pg[k] - po[k]).max() < 1e-9 * uw, (k, np.abs(pg[k] - po[k]).max())
    for k in ("n", "T", "Pxx", "Pzz"):
        assert np.abs(pg[k] - po[k]).max() < 1e-13, k


def test_lowmach_response_is_linear_in_the_wall_speed():
    """The regime of Sec. IV: u_x / u_w and P_xz / u_w do not depend on u_w to
    O(u_w), while T - T_w and n - 1 grow as u_w^2."""
    import paper_1702_01335_gb300 as P
    from paper_1702_01335_gb300 import Instance, Solver
    p = _run(0.1)
    s = Solver([Instance(**dict(p, u_w=1e-5)), Instance(**dict(p, u_w=2e-5))], precision=P.LBS_FP64)
    s.step(3000)
    a, b = s.profiles(0), s.profiles(1)
    for k in ("ux", "Pxz"):
        ra, rb = a[k] / 1e-5, b[k] / 2e-5
        assert np.abs(ra - rb).max() < 1e-4 * np.abs(ra).max(), k
    dT_a, dT_b = a["T"] - 1.0, b["T"] - 1.0
    assert np.abs(dT_a).max() < 1e-9
    ratio = dT_b[np.argmax(np.abs(dT_a))] / dT_a[np.argmax(np.abs(dT_a))]
    assert abs(ratio - 4.0) < 0.05, ratio
