"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test fixes one part of the oracle independently of the oracle itself
(closed forms, library routines, invariants, printed values).  Names follow the
scheme's parts: quadrature, equilibrium, collision, WENO-5, RK-3, walls, and the
whole scheme in its limits.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, special, stats

from oracle import quadrature as quad
from oracle.oracle import (VISC_POWER, VISC_SUTHERLAND, Oracle, mass_flow, nu_center, pi_stress,
                           t_center, txy_average, u_nonlinear, u_slip, u_wall, weno5)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- quadrature --
@pytest.mark.parametrize("Q", [1, 2, 4, 7, 8, 16])
def test_full_range_rule_exact(Q):
    """Gauss rule for exp(-p^2/2)/sqrt(2 pi): sum w p^n = (n-1)!! for even n <= 2Q-1."""
    x, w = quad.full_range_rule(Q)
    assert abs(math.fsum(w) - 1.0) < 1e-14
    for n in range(2 * Q):
        exact = 0.0 if n % 2 else float(special.factorial2(n - 1)) if n > 0 else 1.0
        got = math.fsum(w * x ** n)
        scale = math.fsum(w * np.abs(x) ** n)  # odd moments vanish by cancellation
        assert abs(got - exact) <= 1e-13 * scale, (Q, n, got, exact)
    # independent library rule (scipy, physicists' -> probabilists')
    xs, ws = special.roots_hermitenorm(Q)
    assert np.allclose(np.sort(x), np.sort(xs), rtol=0, atol=1e-12)


@pytest.mark.parametrize("Q", [1, 2, 4, 7, 16, 48, 64, 80, 100])
def test_half_range_rule_exact(Q):
    """Half-range rule on (0, inf): sum w p^n = 2^((n-1)/2) Gamma((n+1)/2)/sqrt(2 pi), n <= 2Q-1."""
    x, w = quad.half_range_rule(Q)
    assert np.all(x > 0) and np.all(w > 0)
    for n in range(2 * Q):
        # in logs: p^n overflows past n ~ 200 at Q = 128
        log_exact = (n - 1) / 2 * math.log(2.0) + math.lgamma((n + 1) / 2) - 0.5 * math.log(2 * math.pi)
        got = math.fsum(np.exp(np.log(w) + n * np.log(x) - log_exact))
        assert abs(got - 1.0) < 1e-13 * max(1, n / 32), (Q, n)


def test_half_range_polys_orthogonal():
    """The monic pi_l are orthogonal on (0, inf) with norms h_l (checked by scipy quad)."""
    N = 6
    c, h = quad.half_range_polys(N)
    om = lambda p: math.exp(-p * p / 2) / math.sqrt(2 * math.pi)
    for a in range(N + 1):
        for b in range(a + 1):
            val = integrate.quad(lambda p: om(p) * np.polyval(c[a][::-1], p) * np.polyval(c[b][::-1], p),
                                 0, np.inf, epsabs=1e-14, epsrel=1e-12)[0]
            assert abs(val - (h[a] if a == b else 0.0)) < 1e-10 * max(1.0, h[a])


# ---------------------------------------------------------------- equilibrium --
def _axis_sums(o, f, a, b, c_, sign=None):
    p = o.velocities()
    sel = np.ones(o.Q, bool) if sign is None else (np.sign(p[:, 2]) == sign)
    return math.fsum((f * p[:, 0] ** a * p[:, 1] ** b * p[:, 2] ** c_)[sel])


@pytest.mark.parametrize("state", [(1.0, (0.0, 0.0, 0.0), 1.0), (1.3, (0.4, -0.2, 0.3), 1.4),
                                   (0.8, (-0.7, 0.1, -0.25), 0.75)])
def test_equilibrium_moment_exactness(state):
    """Sec. III direct product: every per-axis moment up to the expansion order N_a is
    the Gaussian's own (full range: scipy.stats; half range: scipy quad on each semi-axis)."""
    n, u, T = state
    o = Oracle(6, 5, 6, 4, 8)
    f = o.equilibrium(n, u, T, (0, 0, 0), with_S=False)
    g = lambda m, uu: stats.norm(uu, math.sqrt(T)).moment(m)
    for a in range(o.Nx + 1):
        for b in range(o.Ny + 1):
            assert abs(_axis_sums(o, f, a, b, 0) - n * g(a, u[0]) * g(b, u[1])) < 1e-12 * max(1, abs(n * g(a, u[0]) * g(b, u[1])))
    for c_ in range(o.Nzq + 1):
        gz = lambda p: p ** c_ * math.exp(-(p - u[2]) ** 2 / (2 * T)) / math.sqrt(2 * math.pi * T)
        up = integrate.quad(gz, 0, np.inf, epsabs=1e-15, epsrel=1e-13)[0]
        lo = integrate.quad(gz, -np.inf, 0, epsabs=1e-15, epsrel=1e-13)[0]
        assert abs(_axis_sums(o, f, 0, 0, c_, +1) - n * up) < 1e-12
        assert abs(_axis_sums(o, f, 0, 0, c_, -1) - n * lo) < 1e-12


def _perturbed_cell(o, seed=0):
    rng = np.random.default_rng(seed)
    f = o.equilibrium(1.1, (0.3, -0.1, 0.05), 1.2, (0.02, 0.01, -0.03), with_S=True)
    return f * (1.0 + 0.05 * rng.standard_normal(o.Q))


def test_collision_invariants_and_prandtl():
    """Eqs. (boltz), (sdef): f^eq(1+S) built from the moments of f has the same n, n u and
    energy (N >= 5), and heat flux (1 - Pr) q (N >= 6: moments to order 3 + 3)."""
    Pr = 2.0 / 3.0
    o = Oracle(7, 7, 7, 6, 8, Pr=Pr)
    f = _perturbed_cell(o)
    m = o.cell_moments(f)
    fS = o.equilibrium(m["n"], (m["ux"], m["uy"], m["uz"]), m["T"], (m["qx"], m["qy"], m["qz"]))
    p = o.velocities()
    for psi in (np.ones(o.Q), p[:, 0], p[:, 1], p[:, 2], (p ** 2).sum(1)):
        assert abs(math.fsum((fS - f) * psi)) < 1e-13
    mS = o.cell_moments(fS)
    for a in ("qx", "qy", "qz"):
        assert abs(mS[a] - (1 - Pr) * m[a]) < 1e-13
    # equilibrium pressure tensor is isotropic n T
    for a in ("Pxx", "Pyy", "Pzz"):
        assert abs(mS[a] - m["n"] * m["T"]) < 1e-13


def test_collision_invariants_order4():
    """With N = 4 the Shakhov target still conserves mass and momentum (degree-4 moments)."""
    o = Oracle(8, 8, 8, 4, 8, Pr=2.0 / 3.0)
    f = _perturbed_cell(o, 1)
    m = o.cell_moments(f)
    fS = o.equilibrium(m["n"], (m["ux"], m["uy"], m["uz"]), m["T"], (m["qx"], m["qy"], m["qz"]))
    p = o.velocities()
    for psi in (np.ones(o.Q), p[:, 0], p[:, 1], p[:, 2]):
        assert abs(math.fsum((fS - f) * psi)) < 1e-13


def test_tau_laws():
    """Eq. (mw_tau): tau = Kn/n for omega = 1; mu = tau n T = Kn T^omega; Eq. (sutherland_tau)."""
    o = Oracle(4, 4, 4, 3, 8, Kn=0.3, visc_law=VISC_POWER, visc_param=1.0)
    assert abs(o.tau(2.0, 1.7) - 0.15) < 1e-15
    o = Oracle(4, 4, 4, 3, 8, Kn=0.3, visc_law=VISC_POWER, visc_param=0.5)
    assert abs(o.tau(2.0, 1.7) * 2.0 * 1.7 - 0.3 * 1.7 ** 0.5) < 1e-14
    delta, S, n, T = 1.0, 0.5239, 1.3, 1.6
    o = Oracle(4, 4, 4, 3, 8, Kn=1 / (delta * math.sqrt(2)), visc_law=VISC_SUTHERLAND, visc_param=S)
    paper = 1.0 / (n * math.sqrt(T) * delta * math.sqrt(2)) * (1 + S) / (1 + S / T)
    assert abs(o.tau(n, T) - paper) < 1e-14


# ---------------------------------------------------------------- WENO-5 --------
def test_weno_table_limits():
    """Table (weno): vanishing smoothness indicators (constant sub-stencils)."""
    d = np.array([0.1, 0.6, 0.3])
    c = lambda v: np.array([v[0] / 3 - 7 * v[1] / 6 + 11 * v[2] / 6,
                            -v[1] / 6 + 5 * v[2] / 6 + v[3] / 3,
                            v[2] / 3 + 5 * v[3] / 6 - v[4] / 6])
    cases = {  # values -> expected weights
        (2.0, 2.0, 2.0, 2.0, 2.0): d,
        (1.0, 2.0, 2.0, 2.0, 2.0): np.array([0, 2 / 3, 1 / 3]),   # sigma2 = sigma3 = 0
        (2.0, 2.0, 2.0, 5.0, 1.0): np.array([1.0, 0, 0]),          # sigma1 = 0
        (4.0, 1.0, 2.0, 2.0, 2.0): np.array([0, 0, 1.0]),          # sigma3 = 0
    }
    for v, wts in cases.items():
        assert weno5(v) == pytest.approx(float(wts @ c(v)), abs=1e-15)
    # sigma2 = 0 alone is impossible without sigma1 or sigma3 vanishing for 5 values unless
    # v1 = v2 = v3; then sigma1, sigma3 > 0 when v0, v4 differ
    v = (0.0, 1.0, 1.0, 1.0, 3.0)
    assert weno5(v) == pytest.approx(1.0, abs=1e-15)


def test_weno_smooth_limit_and_order():
    """On smooth data the weights tend to the ideal ones: the flux divergence is fifth order."""
    errs = []
    for M in (20, 40, 80):
        h = 1.0 / M
        x = (np.arange(M) + 0.5) * h
        F = np.sin(2 * np.pi * x) + 2.0
        Fp = np.concatenate([F[-3:], F, F[:3]])
        flux = np.array([weno5(Fp[s:s + 5]) for s in range(M + 1)])  # interface s - 1/2
        div = (flux[1:] - flux[:-1]) / h
        errs.append(np.abs(div - 2 * np.pi * np.cos(2 * np.pi * x)).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] > 4.5, orders


def test_rk3_order():
    """Eq. (rk3) on a uniform relaxation (periodic box, BGK, conserved n, u, T, fixed tau):
    f(t) = f_eq + (f0 - f_eq) exp(-t/tau); the error after t = 1 is third order in dt."""
    errs = []
    for dt in (0.1, 0.05, 0.025):
        o = Oracle(4, 4, 4, 3, 6, Kn=0.5, Pr=1.0, dt=dt, periodic=True, shakhov=False)
        rng = np.random.default_rng(3)
        cell = o.weights() * (1.0 + 0.1 * rng.standard_normal(o.Q))
        o.f[:] = cell
        m = o.cell_moments(cell)
        feq = o.equilibrium(m["n"], (m["ux"], m["uy"], m["uz"]), m["T"], (0, 0, 0), with_S=False)
        tau = 0.5 / m["n"]
        steps = int(round(1.0 / dt))
        o.step(steps)
        exact = feq + (cell - feq) * math.exp(-steps * dt / tau)
        errs.append(np.abs(o.f[3] - exact).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 3.0) < 0.2), orders


# ---------------------------------------------------------------- walls ----------
def test_wall_zero_mass_flux_and_incoming_maxwellian():
    """Appendix, diffuse reflection: n_w makes the net mass flux through both wall
    interfaces vanish, and the incoming ghosts are n_w times the wall equilibrium."""
    o = Oracle(4, 4, 4, 3, 16, A=0.9, Kn=0.2, uw=0.4, Pr=2 / 3)
    o.step(50)
    F, nw = o.apply_walls()
    sums = o.interface_sums()
    scale = np.abs(sums[:, 3]).max()
    assert abs(sums[0, 0]) < 1e-14 * scale and abs(sums[-1, 0]) < 1e-14 * scale
    half = o.Q // 2
    Fw_top = o.equilibrium(1.0, (0.4, 0, 0), 1.0, (0, 0, 0), with_S=False)
    Fw_bot = o.equilibrium(1.0, (-0.4, 0, 0), 1.0, (0, 0, 0), with_S=False)
    for r in (o.Nz + 3, o.Nz + 4, o.Nz + 5):
        assert np.allclose(F[r, half:], nw[1] * Fw_top[half:], rtol=1e-15, atol=0)
    for r in (0, 1, 2):
        assert np.allclose(F[r, :half], nw[0] * Fw_bot[:half], rtol=1e-15, atol=0)
    assert abs(nw[0] - nw[1]) < 1e-13  # symmetric problem


# ---------------------------------------------------------------- scheme ---------
def test_mass_conservation_stretched():
    """Conservative flux form (Eq. flux) + zero-mass-flux walls: sum n_s dx_s is constant."""
    o = Oracle(4, 4, 4, 3, 24, A=0.98, Kn=0.1, uw=0.3, Pr=2 / 3)
    m0 = o.mass()
    for _ in range(5):
        o.step(2000)
        assert abs(o.mass() / m0 - 1.0) < 1e-13


def test_centreline_symmetry():
    """Rotation by pi about y: f(s, px, py, pz) = f(Nz+1-s, -px, py, -pz), u_x odd, n, T even."""
    o = Oracle(4, 4, 4, 3, 16, A=0.9, Kn=0.1, uw=0.2, Pr=2 / 3)
    o.step(500)
    Qx, Qy, Qz, Nz = o.Qx, o.Qy, o.Qz, o.Nz
    f = o.f[3:3 + Nz].reshape(Nz, 2, Qz, Qx, Qy)
    mirror = f[::-1, ::-1, :, ::-1, :]
    assert np.abs(f - mirror).max() < 1e-13 * np.abs(f).max()
    p = o.profiles()
    assert np.abs(p["ux"] + p["ux"][::-1]).max() < 1e-13
    assert np.abs(p["T"] - p["T"][::-1]).max() < 1e-13
    assert np.abs(p["qz"] + p["qz"][::-1]).max() < 1e-13
    assert np.abs(p["Pxz"] - p["Pxz"][::-1]).max() < 1e-13


def test_steady_state_flux_invariants():
    """At steady state the interface sums of mass, x-momentum and energy fluxes are
    uniform across the channel (mass: zero), i.e. P_xz uniform and d q_z/dz + P_xz du/dz = 0."""
    o = Oracle(4, 4, 4, 3, 32, Kn=0.1, uw=0.1, Pr=1.0)
    steps, R = o.run_to_steady(1e-11, chunk=500, max_steps=20000)
    assert R < 1e-11
    sums = o.interface_sums()
    mom, en = sums[:, 1], sums[:, 3]
    # the discrete conservation laws make the change of an interface sum across the
    # channel equal to L d/dt of the conserved density, which a residual R per step
    # bounds by about R / dt (densities are O(1) here); the slowest mode is the uniform
    # temperature, so the energy sum keeps a linear tilt of that size
    bound = 5.0 * R / o.dt
    assert np.abs(sums[:, 0]).max() < bound
    assert np.ptp(mom) < bound
    assert np.ptp(en) < bound
    assert bound < 1e-4 * np.abs(mom).max()


def test_pr1_is_bgk():
    """Pr = 1 makes S vanish: the Shakhov path equals the BGK path bit for bit."""
    a = Oracle(4, 4, 4, 3, 12, Kn=0.2, uw=0.3, Pr=1.0)
    b = Oracle(4, 4, 4, 3, 12, Kn=0.2, uw=0.3, Pr=1.0, shakhov=False)
    a.step(100)
    b.step(100)
    assert np.array_equal(a.f, b.f)


@pytest.mark.parametrize("axis", ["x", "y"])
def test_parallel_axis_invariance(axis):
    """Sec. III: the axes parallel to the walls carry no advection, so with the expansion
    order fixed the moments do not depend on Q_a once N + 3 <= Q_a - 1 (the cubic S term).
    Exact for the linear (ideal-weight) reconstruction; WENO's per-node weights couple the
    Hermite modes slightly (checked to 1e-5)."""
    res = {}
    for lin in (True, False):
        for Qa in (7, 9):
            Q = (Qa, 4, 4) if axis == "x" else (4, Qa, 4)
            o = Oracle(*Q, 3, 12, Kn=0.3, uw=0.3, Pr=2 / 3, dt=0.002, weno_linear=lin)
            o.step(200)
            res[(lin, Qa)] = o.profiles()
    for k in ("n", "ux", "T", "Pxz", "qz", "qx"):
        scale = np.abs(res[(True, 7)][k]).max()
        assert np.abs(res[(True, 7)][k] - res[(True, 9)][k]).max() < 1e-12 * scale, k
        assert np.abs(res[(False, 7)][k] - res[(False, 9)][k]).max() < 1e-3 * scale, k


# ------------------------------------------------------------- reduced model --
def _y_integrals(o3):
    """phi = sum_j f_j and chi = sum_j p_y,j^2 f_j of a full-model state (weights absorbed),
    in the reduced model's storage order (j = 0: phi, 1: chi)."""
    f = o3.f.reshape(o3.Nz + 6, 2, o3.Qz, o3.Qx, o3.Qy)
    phi = f.sum(axis=-1)
    chi = (f * o3.py ** 2).sum(axis=-1)
    return np.stack([phi, chi], axis=-1).reshape(o3.Nz + 6, -1)


@pytest.mark.parametrize("A,visc", [(0.0, VISC_POWER), (0.9, VISC_SUTHERLAND)])
def test_reduced_model_is_the_y_integral_of_the_full_model(A, visc):
    """Eqs. (reduced_def), (boltz_red): with the linear reconstruction the phi / chi model
    evolves exactly as the y-integrals int f dp_y, int p_y^2 f dp_y of the full model.
    With Q_y = 7 and N_y = 4 the y-quadrature of the truncated equilibrium times (1 + S)
    and p_y^2 is exact, so the two agree to rounding -- an equilibrium, S_phi / S_chi,
    moment, wall or flux mistake in either would show."""
    kw = dict(A=A, Kn=0.2, uw=0.4, Tw=1.1, Pr=2 / 3, visc_law=visc, visc_param=0.5 if visc == 0 else 0.5239,
              dt=0.002, weno_linear=True)
    full = Oracle(5, 7, 6, 4, 14, **kw)
    red = Oracle(5, 0, 6, 4, 14, **kw)
    assert red.reduced and red.Q == 2 * 5 * 2 * 6
    full.step(60)
    red.step(60)
    ref = _y_integrals(full)[3:3 + 14]
    assert np.abs(red.f[3:3 + 14] - ref).max() < 1e-13 * np.abs(ref).max()
    pf, pr = full.profiles(), red.profiles()
    for k in ("n", "ux", "uz", "T", "qx", "qz", "Pxx", "Pyy", "Pzz", "Pxz"):
        scale = max(np.abs(pf[k]).max(), 1e-3)
        assert np.abs(pf[k] - pr[k]).max() < 1e-12 * scale, k


def test_reduced_shakhov_terms_are_y_averages():
    """Eq. (sred_def): S_phi and S_chi are the averages of the Shakhov factor S of
    Eq. (sdef) over the Maxwellian in p_y, with weights 1 and p_y^2 / T (checked by
    quadrature of S itself, u_y = q_y = 0)."""
    o = Oracle(4, 0, 4, 3, 8, Pr=0.3)
    n, u, T, q = 1.3, np.array([0.2, 0.0, -0.1]), 1.4, np.array([0.05, 0.0, -0.07])
    ratio = o.equilibrium(n, u, T, q, with_S=True) / o.equilibrium(n, u, T, q, with_S=False) - 1.0
    p = o.velocities()
    cS = (1 - 0.3) / (n * T * T)
    for k in range(o.Q):
        ex, ez, j = p[k, 0] - u[0], p[k, 2] - u[2], k % 2
        def S(py):
            xi2 = ex * ex + py * py + ez * ez
            return cS * (xi2 / (5 * T) - 1) * (ex * q[0] + ez * q[2])
        g = lambda py: math.exp(-py * py / (2 * T)) / math.sqrt(2 * math.pi * T)
        wgt = (lambda py: 1.0) if j == 0 else (lambda py: py * py / T)
        ref = integrate.quad(lambda py: g(py) * wgt(py) * S(py), -np.inf, np.inf, epsabs=1e-14)[0]
        assert abs(ratio[k] - ref) < 1e-12 * max(1.0, abs(ref)), k


def test_reduced_model_printed_values():
    """The phi / chi model is the paper's own: Ar, delta = 1, u_w = sqrt 2 on the
    HHLB(6;7) x HLB(6;7) set gives the printed nu = 0.484, Pi = 0.3720, T_0 = 1.561."""
    case = json.load(open(os.path.join(GOLDEN, "paper_tables.json")))["cases"][0]
    delta = case["delta"]
    o = Oracle(7, 0, 7, 6, 32, A=0.98, Kn=1 / (delta * math.sqrt(2)), uw=case["uw"], Pr=2 / 3,
               visc_law=VISC_SUTHERLAND, visc_param=case["S"], dt=5e-4)
    o.step(14000)
    p = o.profiles()
    assert abs(nu_center(o, p["ux"], case["uw"]) - case["nu"]) <= 1.0e-3
    assert abs(pi_stress(o, p["Pxz"], case["uw"], 0.98) / case["Pi"] - 1) < 1e-3
    assert abs(t_center(o, p["T"]) / case["T0"] - 1) < 1e-3


def test_free_molecular_closed_form():
    """tau = infinity: n = 1, u = 0, T = T_w + u_w^2/3, P_xx = T_w + u_w^2, P_yy = P_zz = T_w,
    P_xz = -u_w sqrt(2 T_w / pi) (the ballistic stress of Eq. Txy_bal), q = 0."""
    uw, Tw = 0.3, 1.0
    o = Oracle(4, 4, 4, 3, 16, A=0.5, uw=uw, Tw=Tw, collisions=False)
    o.step(2500)
    p = o.profiles()
    tol = 1e-12
    assert np.abs(p["n"] - 1).max() < tol
    assert np.abs(p["ux"]).max() < tol
    assert np.abs(p["T"] - (Tw + uw ** 2 / 3)).max() < tol
    assert np.abs(p["Pxx"] - (Tw + uw ** 2)).max() < tol
    assert np.abs(p["Pyy"] - Tw).max() < tol and np.abs(p["Pzz"] - Tw).max() < tol
    assert np.abs(p["Pxz"] + uw * math.sqrt(2 * Tw / math.pi)).max() < tol
    for q in ("qx", "qy", "qz"):
        assert np.abs(p[q]).max() < tol


def test_high_kn_near_free_molecular():
    """Kn = 100: the profiles sit within O(1/Kn) of the free-molecular closed form."""
    uw = 0.05
    o = Oracle(8, 4, 4, 4, 32, Kn=100.0, uw=uw, Pr=2 / 3, visc_param=0.5)
    o.step(2500)
    p = o.profiles()
    assert np.abs(p["Pxz"] / (-uw * math.sqrt(2 / math.pi)) - 1).max() < 2e-2
    assert np.abs(p["T"] - (1 + uw ** 2 / 3)).max() < 2e-2 * uw ** 2
    assert np.abs(p["n"] - 1).max() < 2e-2 * uw ** 2
    assert np.abs(p["ux"]).max() < 2e-2 * uw


@pytest.mark.parametrize("Q,N,Pr", [((4, 4, 4), 3, 1.0), ((7, 7, 7), 6, 2.0 / 3.0)])
def test_navier_stokes_limit(Q, N, Pr):
    """Kn = 0.01: in the bulk -P_xz / (du/dz) = mu = Kn T and -q_z / (dT/dz) = (5/2) mu / Pr
    (the Chapman-Enskog coefficients stated in Sec. II)."""
    Kn, uw, Nz = 0.01, 0.05, (32 if Q[0] == 4 else 16)
    o = Oracle(*Q, N, Nz, Kn=Kn, uw=uw, Pr=Pr)
    z = o.xc[3:3 + Nz]
    u = np.zeros((3, Nz))
    u[0] = 1.8 * uw * z
    o.init_from_moments(np.ones(Nz), u, np.ones(Nz), np.zeros((3, Nz)))
    o.step(5000 if Q[0] == 4 else 4000)
    p = o.profiles()
    du, dT = np.gradient(p["ux"], z), np.gradient(p["T"], z)
    mu = Kn * p["T"]
    b = np.arange(Nz // 4, 3 * Nz // 4)
    assert abs(np.mean(-p["Pxz"][b] / du[b] / mu[b]) - 1) < 2e-2
    b = b[np.abs(z[b]) > 0.1]
    assert abs(np.mean(-p["qz"][b] / dT[b] / (2.5 * mu[b] / Pr)) - 1) < 2e-2


# ------------------------------------------------------------ post-processing --
def test_postprocessing_exact_on_polynomials():
    """Eq. (ud0_extra) is exact for odd quintics, Eq. (T0) for even quartics and
    Eq. (uslip_extra) for parabolas (their stated orders), on the stretched grid."""
    o = Oracle(2, 2, 2, 1, 32, A=0.98)
    x = o.xc[3:3 + o.Nz]
    assert abs(x[15] + x[16]) < 1e-15 and x[16] > 0  # cells 16..31 form the upper half
    uw = 0.3
    ux = 0.7 * x - 2.1 * x ** 3 + 5.3 * x ** 5
    assert abs(nu_center(o, ux, uw) - 0.7 / (2 * uw)) < 1e-11
    T = 1.4 + 0.8 * x ** 2 - 3.0 * x ** 4
    assert abs(t_center(o, T) - 1.4) < 1e-12
    u = 0.2 + 1.1 * x - 0.9 * x ** 2
    assert abs(u_wall(o, u) - (0.2 + 1.1 * 0.5 - 0.9 * 0.25)) < 1e-12
    assert abs(u_slip(o, u, uw) - (uw - (0.2 + 0.55 - 0.225))) < 1e-12
    # x^3 is missed by exactly the interpolation remainder prod (L/2 - x_s) over the last three cells
    r = np.prod(0.5 - x[-3:])
    assert abs(u_wall(o, x ** 3) - (0.125 - r)) < 1e-15 and r > 1e-9


def test_nonlinear_velocity_profile():
    """Eq. (uy_nl): a straight profile u = c x (the Navier-Stokes one with slip) has no
    nonlinear part; for u = x^3 it is 2x - x^3 / (1/8 - r), r the interpolation
    remainder of the wall extrapolation (Eq. uslip_extra)."""
    o = Oracle(2, 2, 2, 1, 32, A=0.9)
    x = o.xc[3:3 + o.Nz]
    assert np.abs(u_nonlinear(o, 0.37 * x)).max() < 1e-14
    xs = x[16:]
    r = np.prod(0.5 - xs[-3:])
    assert np.abs(u_nonlinear(o, x ** 3) - (2 * xs - xs ** 3 / (0.125 - r))).max() < 1e-14


@pytest.mark.parametrize("A", [0.5, 0.98])
def test_rectangle_rule_second_order(A):
    """Eqs. (mflow) and (Txy) approximate the half-channel integrals with error
    O(d_eta^2): the hydrodynamic profile u = 2 u_w x / L gives rho u_w L / 4
    (Eq. mflow_hydro) and a uniform T_xy averages to itself."""
    uw = 0.25
    errs_m, errs_t = [], []
    for S in (16, 32, 64):
        o = Oracle(2, 2, 2, 1, 2 * S, A=A)
        x = o.xc[3:3 + o.Nz]
        errs_m.append(mass_flow(o, np.ones(2 * S), 2 * uw * x, A) - uw / 4)
        errs_t.append(txy_average(o, np.full(2 * S, -0.37), A) + 0.37)
    for e in (errs_m, errs_t):
        assert abs(e[0]) < 2e-2 * (uw if e is errs_m else 1)
        assert 3.6 < e[0] / e[1] < 4.4 and 3.6 < e[1] / e[2] < 4.4
    # the density enters as rho = n: doubling n doubles the flow
    o = Oracle(2, 2, 2, 1, 32, A=A)
    x = o.xc[3:3 + o.Nz]
    assert abs(mass_flow(o, 2 * np.ones(32), x, A) - 2 * mass_flow(o, np.ones(32), x, A)) < 1e-15


def _paper_case(case, steps):
    delta = case["delta"]
    o = Oracle(7, 7, 7, 6, 32, A=0.98, Kn=1 / (delta * math.sqrt(2)), uw=case["uw"], Pr=2 / 3,
               visc_law=VISC_SUTHERLAND, visc_param=case["S"], dt=5e-4)
    o.step(steps)
    p = o.profiles()
    return (nu_center(o, p["ux"], case["uw"]), pi_stress(o, p["Pxz"], case["uw"], 0.98),
            t_center(o, p["T"]))


def test_paper_printed_values():
    """Tables gradu, shear, temp (LB columns): Ar, delta = 1, u_w = sqrt 2 gives
    nu = 0.484 (+-0.001), Pi = 0.3720, T_0 = 1.561 (printed digits, < 0.1%)."""
    case = json.load(open(os.path.join(GOLDEN, "paper_tables.json")))["cases"][0]
    nu, Pi, T0 = _paper_case(case, 14000)
    assert abs(nu - case["nu"]) <= 1.0e-3
    assert abs(Pi / case["Pi"] - 1) < 1e-3
    assert abs(T0 / case["T0"] - 1) < 1e-3


def test_residual_hand_computed():
    """The steady-state residual (the paper states no criterion; the solver's definition
    R = max over W in {n, u_x, T} of ||W_new - W_old||_2 / max(||W_old||_2, s_W), with
    s_n = s_T = 1e-30 and s_u = max(|u_w| sqrt(Nz), 1e-30)) on 3-cell cases computed by
    hand.  A squared norm, an L1 norm, a missing max over the three profiles, the new
    state in the denominator, or the wall-speed scale missing, applied to n or T, or
    without the sqrt(Nz), each give another number."""
    from oracle.oracle import residual
    one = [1.0, 1.0, 1.0]
    # only u_x changes: R = 0.003 / sqrt(0.1^2 + 0.1^2) = 0.0212132034...
    Wo = [one, [0.1, 0.0, -0.1], one]
    Wn = [one, [0.1, 0.003, -0.1], [1.0, 1.0004, 1.0]]
    assert abs(residual(Wo, Wn) - 0.003 / math.sqrt(0.02)) < 1e-15
    assert abs(0.003 / math.sqrt(0.02) - 0.021213203435596) < 1e-14
    # T dominates: n changes 0.01 in one cell (0.01 / sqrt 3), T 0.05 (0.05 / sqrt 3)
    Wo = [one, [0.2, 0.0, -0.2], one]
    Wn = [[1.01, 1.0, 1.0], [0.2, 0.0, -0.2], [1.0, 1.0, 1.05]]
    assert abs(residual(Wo, Wn) - 0.05 / math.sqrt(3.0)) < 1e-15
    # u_x from rest: the norm of the old profile is floored at 1e-30
    Wo = [one, [0.0, 0.0, 0.0], one]
    Wn = [one, [1e-3, 0.0, 0.0], one]
    assert abs(residual(Wo, Wn) / 1e27 - 1.0) < 1e-12
    # nothing changes
    assert residual(Wo, Wo) == 0.0
    # the wall speed as the velocity scale: u_w = 0.5 puts s_u = 0.5 sqrt 3 = 0.8660254
    # above ||u_x|| = 0.1414..., so R = 0.003 / 0.8660254 = 0.0034641016...; T's change
    # (0.0004 / sqrt 3 = 2.3e-4) stays below it
    Wo = [one, [0.1, 0.0, -0.1], one]
    Wn = [one, [0.1, 0.003, -0.1], [1.0, 1.0004, 1.0]]
    assert abs(residual(Wo, Wn, uw=0.5) - 0.0034641016151377) < 1e-15
    assert abs(residual(Wo, Wn, uw=-0.5) - 0.0034641016151377) < 1e-15
    # a wall speed below the profile's own norm (0.01 sqrt 3 = 0.0173 < 0.1414) changes
    # nothing
    assert abs(residual(Wo, Wn, uw=0.01) - 0.003 / math.sqrt(0.02)) < 1e-15
    # u_x from rest at u_w = 0.2: 1e-3 / (0.2 sqrt 3) = 0.0028867513...
    Wo = [one, [0.0, 0.0, 0.0], one]
    Wn = [one, [1e-3, 0.0, 0.0], one]
    assert abs(residual(Wo, Wn, uw=0.2) - 0.0028867513459481) < 1e-15
    # n and T keep their own norms: a change of n by 0.01 in one cell at u_w = 0.5
    Wn = [[1.01, 1.0, 1.0], [0.0, 0.0, 0.0], one]
    assert abs(residual(Wo, Wn, uw=0.5) - 0.01 / math.sqrt(3.0)) < 1e-15


def test_residual_of_a_step_is_that_of_n_ux_T():
    """The residual oracle_step reports for a step is the one of the profiles n, u_x
    (velocity, not momentum) and T before and after that step."""
    from oracle.oracle import residual
    o = Oracle(3, 2, 3, 2, 8, Kn=0.2, uw=0.3, Pr=2.0 / 3.0)
    o.step(5)
    a = o.profiles()
    r = o.step(1, residuals=True)[0]
    b = o.profiles()
    assert abs(r / residual([a["n"], a["ux"], a["T"]], [b["n"], b["ux"], b["T"]], uw=0.3) - 1.0) < 1e-12
    mom = [b["n"], b["n"] * b["ux"], b["T"]]
    assert abs(r / residual([a["n"], a["n"] * a["ux"], a["T"]], mom, uw=0.3) - 1.0) > 1e-6
    # and the run's wall speed is the one it is measured on
    assert abs(r / residual([a["n"], a["ux"], a["T"]], [b["n"], b["ux"], b["T"]], uw=3.0) - 1.0) > 1e-6
