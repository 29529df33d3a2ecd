"""Helpers shared by the GPU parity tests: build the same problem in the CUDA
solver and in the oracle from one parameter dict (same dt for both)."""
import numpy as np

from oracle.oracle import Oracle


def oracle_of(p, dt):
    return Oracle(p["Qx"], p["Qy"], p["Qz"], p["N_eq"], p["Nz"], A=p["A"], Kn=p["Kn"], uw=p["u_w"],
                  Tw=p["T_w"], Pr=p["Pr"], visc_law=p["visc_law"], visc_param=p["visc_param"], dt=dt)


def solver_of(ps, dt, precision):
    from paper_1702_01335_gb300 import Instance, Solver
    if isinstance(ps, dict):
        ps = [ps]
    return Solver([Instance(dt=dt, **p) for p in ps], precision=precision)


def gpu_f(solver, o, inst=0):
    """GPU state as populations with the weights applied, [Nz, Q] (oracle layout)."""
    return solver.populations(inst) * o.weights()[None, :]


def same_state(a, b):
    """Two stored states (deviations and FP32 residuals) equal bit for bit."""
    return np.array_equal(a.d, b.d) and (a.r is None) == (b.r is None) and (a.r is None or np.array_equal(a.r, b.r))


def rel_err(a, b, scale=None):
    s = np.abs(b).max() if scale is None else scale
    return float(np.abs(a - b).max() / max(s, 1e-300))


PROFILES = ("n", "ux", "uy", "uz", "T", "qx", "qy", "qz", "Pxx", "Pyy", "Pzz", "Pxy", "Pxz", "Pyz")


def profile_errors(gp, op, uw=None):
    """max |gpu - oracle| / scale per profile.  The scale is max |oracle| of the profile,
    except: u_y, u_z, P_xy, P_yz vanish by symmetry and take the scale of u_x or P_xz;
    the heat fluxes are differences of raw third moments of size n T^(3/2), so they are
    compared on that scale (a q of 1e-3 n T^(3/2) keeps ~3 fewer digits than the sums).
    With uw given, velocities are compared on the Couette scale max(max |u_x|, u_w)."""
    out = {}
    ref_scale = {"uy": "ux", "uz": "ux", "Pxy": "Pxz", "Pyz": "Pxz"}
    thermal = float(np.max(op["n"] * op["T"] ** 1.5))
    for k in PROFILES:
        if k in ("qx", "qy", "qz"):
            scale = thermal
        else:
            scale = np.abs(op[ref_scale.get(k, k)]).max()
            if uw is not None and k in ("ux", "uy", "uz"):
                scale = max(scale, uw)
        out[k] = rel_err(gp[k], op[k], max(scale, 1e-300))
    return out
