"""Python front end of the FP64 oracle (ctypes over couette.c, numpy set-up).

TEST INFRASTRUCTURE ONLY.  Tests, the smoke check and the CPU-baseline leg of
the benchmark use this module to compute the reference results the CUDA solver
is compared with.  The solver itself never imports it, and it imports nothing
from the solver package.

Contents:
  * `build()` compiles couette.c into oracle/_build/liboracle.so (gcc, -O2,
    OpenMP over cells, no fast-math);
  * `grid()` builds cell centres and interfaces: uniform, or the tanh-stretched
    grid of Eqs. (stretch), (etas) mirrored onto the full channel
    [-L/2, L/2], with ghost cells continuing the eta spacing;
  * `Oracle` holds one Couette problem and steps it with the scheme;
  * `nu_center`, `pi_stress`, `t_center`, `u_slip`, `mass_flow` are the
    post-processing formulas of Eqs. (vgrad)/(ud0_extra), (stress)/(Txy), (T0),
    (uslip)/(uslip_extra) and (mflow) on the upper half of the full channel.
"""
import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

from . import quadrature as quad

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "couette.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

VISC_POWER = 0
VISC_SUTHERLAND = 1
PROFILE_NAMES = ("n", "ux", "uy", "uz", "T", "qx", "qy", "qz",
                 "Pxx", "Pyy", "Pzz", "Pxy", "Pxz", "Pyz")


def build(force=False):
    """Compile the oracle shared library (idempotent)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                           "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class _Cfg(C.Structure):
    _fields_ = [(n, C.c_int) for n in ("Nz", "Qx", "Qy", "Qz", "Nx", "Ny", "Nzq",
                                       "visc_law", "collisions", "shakhov", "periodic",
                                       "weno_linear", "reduced")] + \
               [(n, C.c_double) for n in ("Kn", "uw", "Tw", "Pr", "visc_param", "dt")] + \
               [(n, C.POINTER(C.c_double)) for n in ("px", "wx", "py", "wy", "xi", "wz",
                                                     "Hx", "Hy", "Pz", "cz", "xc", "xf")]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER(_Cfg)
            D = C.POINTER(C.c_double)
            lib.oracle_step.argtypes = [P, D, C.c_long, D]
            lib.oracle_profiles.argtypes = [P, D, D]
            lib.oracle_equilibrium.argtypes = [P, D, C.c_int, D]
            lib.oracle_cell_moments.argtypes = [P, D, D]
            lib.oracle_apply_walls.argtypes = [P, D, D]
            lib.oracle_interface_sums.argtypes = [P, D, D]
            lib.oracle_weno5.argtypes = [D]
            lib.oracle_weno5.restype = C.c_double
            lib.oracle_tau.argtypes = [P, C.c_double, C.c_double]
            lib.oracle_tau.restype = C.c_double
            lib.oracle_residual.argtypes = [C.c_int, D, D, C.c_double]
            lib.oracle_residual.restype = C.c_double
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def grid(Nz, A=0.0, L=1.0):
    """Cell centres x_s (s = -2..Nz+3) and interfaces x_{s+1/2} (s = 0..Nz).

    A = 0: uniform cells of width L/Nz on [-L/2, L/2].
    0 < A < 1: Eq. (etas) on the full channel, eta_s = -atanh(A) + (s - 1/2) d_eta,
    d_eta = 2 atanh(A) / Nz, x = L tanh(eta) / (2A); the interfaces take
    eta_s +- d_eta/2 (Appendix, "Advection"); ghost cells continue eta linearly.
    """
    s = np.arange(-2, Nz + 4, dtype=np.float64)
    f = np.arange(0, Nz + 1, dtype=np.float64)
    if A == 0.0:
        return -0.5 * L + (s - 0.5) * L / Nz, -0.5 * L + f * L / Nz
    E = math.atanh(A)
    de = 2.0 * E / Nz
    return (L / (2 * A) * np.tanh(-E + (s - 0.5) * de),
            L / (2 * A) * np.tanh(-E + f * de))


class Oracle:
    """One Couette problem in the oracle.

    Parameters follow the solver's configuration: orders (Qx, Qy, Qz per sign),
    the equilibrium order N_eq (clipped per axis to Q_a - 1), Nz cells, the
    stretching A, Kn, u_w, T_w, Pr, the viscosity law (power with omega, or
    Sutherland with S) and the time step dt.

    reduced=True (or Qy=0) selects the phi / chi model of Sec. III: the transverse
    axis is integrated out and j in {0, 1} indexes phi and chi on the (p_x, p_z)
    nodes (Qy = 2 in the storage order, weights w_x w_z, p_y unused).
    """

    def __init__(self, Qx, Qy, Qz, N_eq, Nz, A=0.0, Kn=0.1, uw=0.1, Tw=1.0, Pr=1.0,
                 visc_law=VISC_POWER, visc_param=1.0, dt=None, cfl=0.5,
                 collisions=True, shakhov=True, periodic=False, weno_linear=False, reduced=False):
        self.reduced = bool(reduced or Qy == 0)
        if self.reduced:
            Qy = 2
        self.Qx, self.Qy, self.Qz, self.Nz = Qx, Qy, Qz, Nz
        self.Q = 2 * Qx * Qy * Qz
        self.Nx, self.Ny, self.Nzq = min(N_eq, Qx - 1), min(N_eq, Qy - 1), min(N_eq, Qz - 1)
        self.px, self.wx = quad.full_range_rule(Qx)
        if self.reduced:
            self.Ny = 0
            self.py, self.wy = np.zeros(2), np.ones(2)
        else:
            self.py, self.wy = quad.full_range_rule(Qy)
        self.xi, self.wz = quad.half_range_rule(Qz)
        self.Hx = np.ascontiguousarray(quad.hermite_table(self.px, self.Nx))
        self.Hy = np.ascontiguousarray(quad.hermite_table(self.py, self.Ny))
        c, h = quad.half_range_polys(self.Nzq)
        self.cz = np.ascontiguousarray(c)
        self.Pz = np.ascontiguousarray(quad.half_range_table(self.xi, c, h))
        self.xc, self.xf = grid(Nz, A)
        if dt is None:
            dt = cfl * float(np.min(np.diff(self.xf))) / float(self.xi.max())
        self.dt = dt
        self.cfg = _Cfg(Nz, Qx, Qy, Qz, self.Nx, self.Ny, self.Nzq, visc_law,
                        int(collisions), int(shakhov), int(periodic), int(weno_linear),
                        int(self.reduced),
                        Kn, uw, Tw, Pr, visc_param, dt,
                        *[_ptr(a) for a in (self.px, self.wx, self.py, self.wy, self.xi, self.wz,
                                            self.Hx, self.Hy, self.Pz, self.cz, self.xc, self.xf)])
        self.lib = _load()
        self.f = np.ascontiguousarray(np.tile(self.weights(), (Nz + 6, 1)))
        self.steps = 0

    # ---- velocity set ------------------------------------------------------
    def velocities(self):
        """p[Q, 3] in the storage order k = ((sg*Qz + m)*Qx + i)*Qy + j."""
        sg, m, i, j = np.meshgrid(np.arange(2), np.arange(self.Qz), np.arange(self.Qx),
                                  np.arange(self.Qy), indexing="ij")
        pz = np.where(sg == 0, self.xi[m], -self.xi[m])
        return np.stack([self.px[i].ravel(), self.py[j].ravel(), pz.ravel()], axis=1)

    def weights(self):
        sg, m, i, j = np.meshgrid(np.arange(2), np.arange(self.Qz), np.arange(self.Qx),
                                  np.arange(self.Qy), indexing="ij")
        return (self.wz[m] * self.wx[i] * self.wy[j]).ravel()

    # ---- scheme --------------------------------------------------------------
    def step(self, nsteps, residuals=False):
        res = np.zeros(nsteps) if residuals else None
        self.lib.oracle_step(C.byref(self.cfg), _ptr(self.f), nsteps,
                             _ptr(res) if residuals else None)
        self.steps += nsteps
        return res

    def run_to_steady(self, tol=1e-8, chunk=200, max_steps=2_000_000):
        """March until the residual R < tol; returns (steps taken, last R)."""
        taken = 0
        while taken < max_steps:
            r = self.step(chunk, residuals=True)
            taken += chunk
            below = np.nonzero(r < tol)[0]
            if below.size:
                return taken, float(r[-1])
        return taken, float(r[-1])

    def profiles(self):
        """dict of the 14 profiles over the Nz interior cells (Eq. qdef)."""
        out = np.zeros((14, self.Nz))
        self.lib.oracle_profiles(C.byref(self.cfg), _ptr(self.f), _ptr(out))
        return {k: out[a] for a, k in enumerate(PROFILE_NAMES)}

    def equilibrium(self, n, u, T, q, with_S=True):
        mom = np.array([n, u[0], u[1], u[2], T, q[0], q[1], q[2]], dtype=np.float64)
        out = np.zeros(self.Q)
        self.lib.oracle_equilibrium(C.byref(self.cfg), _ptr(mom), int(with_S), _ptr(out))
        return out

    def cell_moments(self, f_cell):
        f_cell = np.ascontiguousarray(f_cell, dtype=np.float64)
        out = np.zeros(14)
        self.lib.oracle_cell_moments(C.byref(self.cfg), _ptr(f_cell), _ptr(out))
        return dict(zip(PROFILE_NAMES, out))

    def tau(self, n, T):
        return self.lib.oracle_tau(C.byref(self.cfg), n, T)

    def apply_walls(self, F=None):
        """Impose the ghost nodes on F (default: a copy of the state); returns (F, n_w)."""
        F = np.ascontiguousarray(self.f.copy() if F is None else F)
        nw = np.zeros(2)
        self.lib.oracle_apply_walls(C.byref(self.cfg), _ptr(F), _ptr(nw))
        return F, nw

    def interface_sums(self):
        """[Nz+1, 4]: sum_k psi Flux_{s+1/2} for psi = 1, p_x, p_z, |p|^2/2."""
        out = np.zeros((self.Nz + 1, 4))
        self.lib.oracle_interface_sums(C.byref(self.cfg), _ptr(self.f), _ptr(out))
        return out

    def init_from_moments(self, n, u, T, q):
        """f = discrete Shakhov target of per-cell (n, u[3], T, q[3]) in every interior
        cell; ghosts copy the nearest interior cell (they are re-imposed every stage)."""
        for s in range(self.Nz):
            self.f[s + 3] = self.equilibrium(n[s], u[:, s], T[s], q[:, s])
        self.f[:3] = self.f[3]
        self.f[self.Nz + 3:] = self.f[self.Nz + 2]

    def cell_widths(self):
        return np.diff(self.xf)

    def mass(self):
        return float(np.sum(self.profiles()["n"] * self.cell_widths()))


def residual(W_old, W_new, uw=0.0):
    """The oracle's residual of one step from W[3][Nz] = (n, u_x, T) before and after,
    the velocity measured on the wall speed uw where u_x is smaller."""
    a = np.ascontiguousarray(W_old, dtype=np.float64)
    b = np.ascontiguousarray(W_new, dtype=np.float64)
    assert a.shape == b.shape and a.shape[0] == 3
    return _load().oracle_residual(a.shape[1], _ptr(a), _ptr(b), float(uw))


def weno5(v):
    """Reconstructed interface value of five upwind-ordered values (no p factor)."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    return _load().oracle_weno5(_ptr(v))


# ---- post-processing of Sec. VI (half channel 0 <= z <= L/2) -----------------
def _half(o):
    S = o.Nz // 2
    return S, o.xc[3 + S: 3 + 2 * S]


def nu_center(o, ux, uw):
    """nu = (L / 2u_w) u'(0), Eq. (vgrad), with u'(0) from the 3-point Eq. (ud0_extra)."""
    S, x = _half(o)
    u = ux[S:S + 3]
    x1, x2, x3 = x[0], x[1], x[2]
    d = (x2 ** 2 * x3 ** 2 * u[0] / (x1 * (x1 ** 2 - x2 ** 2) * (x1 ** 2 - x3 ** 2)) +
         x1 ** 2 * x3 ** 2 * u[1] / (x2 * (x2 ** 2 - x1 ** 2) * (x2 ** 2 - x3 ** 2)) +
         x1 ** 2 * x2 ** 2 * u[2] / (x3 * (x3 ** 2 - x1 ** 2) * (x3 ** 2 - x2 ** 2)))
    return d / (2.0 * uw)


def txy_average(o, Pxz, A):
    """Eq. (Txy): rectangle rule in eta over the half channel."""
    S, _ = _half(o)
    E = math.atanh(A)
    eta = (np.arange(1, S + 1) - 0.5) * E / S
    return E / (A * S) * float(np.sum(Pxz[S:] / np.cosh(eta) ** 2))


def pi_stress(o, Pxz, uw, A):
    """Pi = -T_xy / (u_w sqrt 2), Eq. (stress), T_xy averaged by Eq. (Txy)."""
    return -txy_average(o, Pxz, A) / (uw * math.sqrt(2.0))


def u_wall(o, ux):
    """u_y(L/2) of Eq. (uslip_extra): the parabola through the last three cells
    (S, S-1, S-2 of the half channel) evaluated at the wall x = L/2 = 0.5."""
    S, x = _half(o)
    xs, us = x[S - 3:], ux[2 * S - 3:2 * S]
    tot = 0.0
    for a in range(3):
        b, c = [e for e in range(3) if e != a]
        tot += (0.5 - xs[b]) * (0.5 - xs[c]) / ((xs[a] - xs[b]) * (xs[a] - xs[c])) * us[a]
    return tot


def u_nonlinear(o, ux):
    """Eq. (uy_nl) on the upper half: 2 x / L - u_y(x) / u_y(L/2), L = 1, with u_y(L/2)
    from Eq. (uslip_extra)."""
    S, x = _half(o)
    return 2.0 * x - ux[S:] / u_wall(o, ux)


def u_slip(o, ux, uw):
    """u_slip = u_w - u_y(L/2), Eq. (uslip)."""
    return uw - u_wall(o, ux)


def mass_flow(o, n, ux, A):
    """Half-channel mass flow of Eq. (mflow): rectangle rule in eta,
    L atanh(A) / (2 A S) sum_s rho_s u_s / cosh^2 eta_s (L = 1, rho = n)."""
    S, _ = _half(o)
    E = math.atanh(A)
    eta = (np.arange(1, S + 1) - 0.5) * E / S
    return E / (2.0 * A * S) * float(np.sum(n[S:] * ux[S:] / np.cosh(eta) ** 2))


def t_center(o, T):
    """T_0 of Eq. (T0) from the three cells next to the centre line."""
    S, x = _half(o)
    t = T[S:S + 3]
    x1, x2, x3 = x[0] ** 2, x[1] ** 2, x[2] ** 2
    return (x2 * x3 * t[0] / ((x1 - x2) * (x1 - x3)) + x3 * x1 * t[1] / ((x2 - x1) * (x2 - x3)) +
            x1 * x2 * t[2] / ((x3 - x1) * (x3 - x2)))
