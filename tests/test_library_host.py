"""Host-side checks of the solver library that need no GPU: it builds and loads,
exports every entry point include/lbs.h declares, its quadrature (an algorithm
independent of the oracle's) agrees with the oracle's, and bad arguments are
rejected before any device work."""
import ctypes as C
import math
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import quadrature as oq
from oracle.oracle import Oracle, mass_flow, nu_center, pi_stress, t_center, txy_average, u_nonlinear, u_wall
from paper_1702_01335_gb300 import lbs as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(lbs_\w+)\s*\(", txt))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = L.load()
    names = declared_symbols()
    assert "lbs_create" in names and "lbs_step" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(L.EXPORTS) >= set(names) - {"lbs_last_error"} | set()


@pytest.mark.parametrize("Q", [1, 2, 4, 7, 16])
def test_full_range_rule_matches_oracle(Q):
    x, w = L.quadrature(0, Q)
    xo, wo = oq.full_range_rule(Q)
    assert np.allclose(x, xo, rtol=0, atol=1e-13)
    assert np.allclose(w, wo, rtol=1e-12, atol=0)


@pytest.mark.parametrize("Q", [1, 4, 7, 16, 32, 48, 64, 80, 100])
def test_half_range_rule_matches_oracle(Q):
    x, w = L.quadrature(1, Q)
    xo, wo = oq.half_range_rule(Q)
    assert np.allclose(x, xo, rtol=1e-12, atol=0)
    assert np.allclose(w, wo, rtol=1e-11, atol=0)


def test_bad_arguments_are_rejected():
    lib = L.load()
    h = C.c_void_p()
    bad = [
        L.Instance(Qx=0), L.Instance(Qz=101), L.Instance(N_eq=9), L.Instance(Nz=5),
        L.Instance(Kn=0.0), L.Instance(T_w=-1.0), L.Instance(Pr=0.0), L.Instance(A=1.0),
        L.Instance(cfl=0.0, dt=0.0), L.Instance(visc_law=1, visc_param=0.0),
        L.Instance(Qx=64, Qy=64, Qz=64), L.Instance(half=2), L.Instance(Qy=-1),
    ]
    for inst in bad:
        d = (L._Desc * 1)(inst.desc())
        st = lib.lbs_batch_create(C.byref(h), d, 1, 0, None)
        assert st == 1, inst
        assert lib.lbs_last_error().decode()
    mixed = (L._Desc * 2)(L.Instance(Qy=0).desc(), L.Instance().desc())
    assert lib.lbs_batch_create(C.byref(h), mixed, 2, 0, None) == 1
    assert "mix" in lib.lbs_last_error().decode()
    assert L.Instance(Qy=0, Qx=5, Qz=6).Q == 4 * 5 * 6
    assert lib.lbs_quadrature(2, 4, None, None) == 1
    assert lib.lbs_step(None, 1) == 1
    prof = np.zeros((14, 12))
    for Nz, A, half in ((11, 0.5, 0), (12, 1.0, 0), (5, 0.5, 1), (12, 0.5, 3)):
        with pytest.raises(L.LbsError):
            L.couette_diagnostics(np.zeros((14, Nz)), Nz, A, half, 0.1)
    assert lib.lbs_couette_diagnostics(None, 12, 0.5, 0, 0.1, 1.0, None) == 1
    assert lib.lbs_couette_nonlinear_velocity(None, 12, 0.5, 0, None, None) == 1
    for Nz, A, half in ((11, 0.5, 0), (5, 0.5, 1), (12, -0.1, 0)):
        with pytest.raises(L.LbsError):
            L.couette_nonlinear_velocity(np.ones((14, Nz)), Nz, A, half)
    assert lib.lbs_set_finalize(None, 1, None) == 1
    assert L.couette_diagnostics(prof, 12, 0.5, 0, 0.1)["Txy"] == 0.0


def _smooth_profiles(Nz, x, rng):
    """Smooth profiles with the Couette symmetry on cell centres x (n, T, P_xz even; u_x odd)."""
    prof = np.zeros((14, Nz))
    c = rng.uniform(0.5, 1.5, 8)
    prof[0] = c[0] + 0.3 * c[1] * x ** 2
    prof[1] = 0.2 * c[2] * x + 0.5 * c[3] * x ** 3 + np.sin(c[4] * x) * 0.1
    prof[4] = c[5] + 0.4 * x ** 2 - c[6] * x ** 4 + 0.05 * np.cos(3 * x)
    prof[12] = -0.3 * c[7] + 0.01 * x ** 2
    prof[[2, 3, 5, 6, 7, 8, 9, 10, 11, 13]] = rng.standard_normal((10, Nz))  # not read
    return prof


@pytest.mark.parametrize("A", [0.0, 0.7, 0.98])
@pytest.mark.parametrize("S", [8, 16, 33])
def test_diagnostics_match_oracle(A, S):
    """lbs_couette_diagnostics (its own code) against the oracle's post-processing on the
    upper half of a full channel of 2S cells, and on the same cells given as a half channel."""
    rng = np.random.default_rng(S)
    o = Oracle(2, 2, 2, 1, 2 * S, A=A)
    x = o.xc[3:3 + o.Nz]
    prof = _smooth_profiles(2 * S, x, rng)
    uw, Tw = 0.37, 1.3
    for half, p in ((0, prof), (1, prof[:, S:])):
        d = L.couette_diagnostics(p, p.shape[1], A, half, uw, Tw)
        assert abs(d["nu"] - nu_center(o, prof[1], uw)) < 1e-11
        assert abs(d["dudz0"] - 2 * uw * nu_center(o, prof[1], uw)) < 1e-11
        assert abs(d["T0"] - t_center(o, prof[4])) < 1e-11
        assert abs(d["u_wall"] - u_wall(o, prof[1])) < 1e-12
        assert abs(d["u_slip"] - (uw - u_wall(o, prof[1]))) < 1e-12
        if A > 0:
            assert abs(d["Txy"] - txy_average(o, prof[12], A)) < 1e-13
            assert abs(d["Pi"] - pi_stress(o, prof[12], uw, A)) < 1e-13
            assert abs(d["mflow"] - mass_flow(o, prof[0], prof[1], A)) < 1e-13
        else:  # the A -> 0 limit of the rectangle rule: the midpoint rule on uniform cells
            assert abs(d["Txy"] - np.mean(prof[12][S:])) < 1e-13
            assert abs(d["mflow"] - 0.5 * np.mean(prof[0][S:] * prof[1][S:])) < 1e-13
        assert d["mflow_hydro"] == uw / 4
        assert abs(d["Txy_bal"] + uw * np.sqrt(2 * Tw / np.pi)) < 1e-15
        z, unl = L.couette_nonlinear_velocity(p, p.shape[1], A, half)
        assert np.abs(z - x[S:]).max() < 1e-14
        assert np.abs(unl - u_nonlinear(o, prof[1])).max() < 1e-11


def test_erfc_series_against_libm():
    """erfc_nonneg (lbs_internal.h: the Maclaurin series of erf below 1/2, the library
    erfc above) against the C library's erfc on [0, 3], built on the host from the same
    header the kernels include."""
    src = r"""
#include <cstdio>
#include <cmath>
#include "lbs_internal.h"
int main() {
    double worst = 0.0;
    for (int i = 0; i <= 300000; ++i) {
        const double x = 3.0 * i / 300000.0, a = lbs::erfc_nonneg(x), b = std::erfc(x);
        worst = std::fmax(worst, std::fabs(a - b) / b);
    }
    std::printf("%.6e\n", worst);
    return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        cpp, exe = os.path.join(d, "e.cpp"), os.path.join(d, "e")
        open(cpp, "w").write(src)
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1702_01335_gb300", "csrc"),
                               cpp, "-o", exe])
        worst = float(subprocess.check_output([exe]).decode())
    assert worst < 5e-16, worst


def _rk3_upwind5_cfl_limit():
    """Largest CFL number nu = |p| dt / dz for which RK-3 (Eq. rk3) with the linear
    fifth-order upwind flux (WENO-5 at its ideal weights d = 1/10, 6/10, 3/10 of the
    three third-order candidates) is stable for every Fourier mode (von Neumann)."""
    th = np.linspace(0.0, 2 * np.pi, 4001)
    # interface value at j+1/2 from f_{j-2..j+2}: the three candidates of Eq. (weno5_flux)
    c1 = np.array([2, -7, 11, 0, 0]) / 6.0
    c2 = np.array([0, -1, 5, 2, 0]) / 6.0
    c3 = np.array([0, 0, 2, 5, -1]) / 6.0
    coef = 0.1 * c1 + 0.6 * c2 + 0.3 * c3
    R = sum(coef[m] * np.exp(1j * (m - 2) * th) for m in range(5))
    sym = -(R - R * np.exp(-1j * th))          # -(F_{j+1/2} - F_{j-1/2}) per unit CFL
    def stable(nu):
        z = nu * sym
        return np.max(np.abs(1 + z + z * z / 2 + z ** 3 / 6)) <= 1 + 1e-12
    lo, hi = 0.1, 3.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if stable(mid) else (lo, mid)
    return lo


def test_time_step_stability_of_the_table_runs():
    """The paper's printed time steps against the scheme's linear stability limit
    (about 1.43): dt = 5e-4 at Q_n = 7 and 2.5e-4 at Q_n = 30 are stable on the 16-cell
    half channel with A = 0.98; 2.5e-4 at Q_n = 100 (delta = 0.01) is not, and 1e-4 is."""
    from oracle.oracle import grid
    nu = _rk3_upwind5_cfl_limit()
    assert 1.3 < nu < 1.6, nu
    _, xf = grid(32, 0.98)
    dz = float(np.min(np.diff(xf)))
    for Qn, dt, ok in ((7, 5e-4, True), (30, 2.5e-4, True), (100, 2.5e-4, False), (100, 1e-4, True)):
        x, _ = L.quadrature(1, Qn)
        assert (x.max() * dt / dz < nu) == ok, (Qn, dt, x.max() * dt / dz, nu)


def test_diagnostics_of_the_ballistic_state():
    """The free-molecular state (the oracle without collisions) has closed-form
    diagnostics: u = 0 inside, so u_slip = u_w and the mass flow vanishes, and
    T_xy / T_xy^bal = 1 (Eq. Txy_bal) -- for a full channel and its upper half."""
    uw, Tw = 0.3, 1.0
    o = Oracle(4, 4, 4, 3, 16, A=0.5, uw=uw, Tw=Tw, collisions=False)
    o.step(2500)
    p = o.profiles()
    prof = np.stack([p[k] for k in L.PROFILE_NAMES])
    # the rectangle rule of Eq. (Txy) applied to a constant: 1 up to its O(d_eta^2) error
    E = math.atanh(0.5)
    rule = E / (0.5 * 8) * sum(1 / math.cosh((s + 0.5) * E / 8) ** 2 for s in range(8))
    assert 0 < abs(rule - 1) < 1e-3
    for half, pr in ((0, prof), (1, prof[:, 8:])):
        d = L.couette_diagnostics(pr, pr.shape[1], 0.5, half, uw, Tw)
        assert abs(d["u_slip"] - uw) < 1e-11 and abs(d["mflow"]) < 1e-12
        assert abs(d["Txy"] / d["Txy_bal"] - rule) < 1e-11
        assert abs(d["Pi"] - rule / math.sqrt(math.pi)) < 1e-11  # -T_xy / (u_w sqrt 2) at T_w = 1
        assert abs(d["T0"] - (Tw + uw ** 2 / 3)) < 1e-11


def test_autotuner_host_logic(monkeypatch, tmp_path):
    """autotune.py without a GPU (timings from a stand-in solver): it keeps the fastest
    valid candidate, skips rejected ones, writes the choice under the kernel hash and the
    batch signature, drops entries of other kernel versions, and answers a repeated call
    from the cache without timing again."""
    import json
    from paper_1702_01335_gb300 import autotune as AT

    made = []

    class FakeSolver:
        def __init__(self, instances, precision=1):
            self.instances, self.precision, self.t = instances, precision, None
            made.append(self)

        def set_tiling(self, V, ZT, F):
            if ZT > 64:
                raise L.LbsError(1, "tiling")
            self.t = (V, ZT, F)

        def profile_steps(self, n):
            V, ZT, F = self.t
            ms = (1.0 + abs(V - 2) + abs(ZT - 12) / 10 + F) * n  # fastest: V = 2, ZT = 12, F = 0
            return 0.9 * ms, 0.1 * ms, ms

        def tiling(self):
            return {"ctas": 1}

        def set_finalize(self, mode):
            self.fin = mode
            return mode == 2

        def close(self):
            pass

    monkeypatch.setattr(AT, "Solver", FakeSolver)
    monkeypatch.setattr(AT, "_cache", {})
    cache = tmp_path / "cache.json"
    cache.write_text(json.dumps({"0000000000000000:p1:9x9": {"V": 1, "ZT": 4, "fuse": 0}}))
    target = FakeSolver([L.Instance(Nz=16), L.Instance(Nz=16), L.Instance(Nz=24)], precision=1)
    made.clear()
    r = AT.autotune(target, candidates=((1, 8, 0), (2, 12, 0), (2, 12, 1), (4, 99, 0)), steps=3,
                    cache_file=str(cache))
    assert (r["V"], r["ZT"], r["fuse"]) == (2, 12, 0) and target.t == (2, 12, 0)
    assert r["fin"] in (1, 2) and target.fin == r["fin"]
    # one scratch solver for the tilings (the invalid one skipped), one for the finalisation layouts
    assert len(r["table"]) == 3 and len(made) == 2
    disk = json.loads(cache.read_text())
    assert not list(tmp_path.glob("*.tmp"))  # written through a temporary file, then replaced
    key = AT.signature(target)
    assert list(disk) == [key] and key.startswith(AT.kernel_hash() + ":p1:")
    assert key.endswith(":2*16x128,24x128")
    monkeypatch.setattr(AT, "_cache", {})
    made.clear()
    again = FakeSolver(target.instances, precision=1)
    made.clear()
    r2 = AT.autotune(again, cache_file=str(cache))
    assert (r2["V"], r2["ZT"], r2["fuse"]) == (2, 12, 0) and again.t == (2, 12, 0) and not made
    assert again.fin == r["fin"]
