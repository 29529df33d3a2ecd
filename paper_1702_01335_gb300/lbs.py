"""Python binding of the C ABI in include/lbs.h (ctypes; argument marshalling only).

Every step of the solver runs in the CUDA kernels of liblbs.so.  There is no
CPU fallback: if the shared library is missing or cannot be loaded, `load()`
raises.  PyTorch is used only to hand the library a CUDA stream and, for
device-side checkpoints, device memory.
"""
import ctypes as C
import dataclasses
import os
import threading

import numpy as np

from . import build as _build

LBS_FP64 = 0
LBS_FP32 = 1
VISC_POWER = 0
VISC_SUTHERLAND = 1
MOMENT_NAMES = ("n", "ux", "T", "qx", "qz", "Pxx", "Pxz", "Pzz")
PROFILE_NAMES = ("n", "ux", "uy", "uz", "T", "qx", "qy", "qz",
                 "Pxx", "Pyy", "Pzz", "Pxy", "Pxz", "Pyz")
STATUS = {0: "LBS_OK", 1: "LBS_ERR_ARG", 2: "LBS_ERR_CUDA", 3: "LBS_ERR_NONFINITE",
          4: "LBS_ERR_NO_CONVERGENCE", 5: "LBS_ERR_QUADRATURE", 6: "LBS_ERR_TIMEOUT"}
LBS_ERR_ARG = 1
LBS_ERR_NONFINITE = 3
LBS_ERR_NO_CONVERGENCE = 4
LBS_ERR_TIMEOUT = 6

_lock = threading.Lock()
_lib = None


class LbsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class _Orders(C.Structure):
    _fields_ = [("Qx", C.c_int), ("Qy", C.c_int), ("Qz_half", C.c_int), ("N_eq", C.c_int)]


class _Grid(C.Structure):
    _fields_ = [("Nz", C.c_int), ("A", C.c_double), ("half", C.c_int)]


DIAG_NAMES = ("u_wall", "u_slip", "dudz0", "nu", "mflow", "mflow_hydro", "Txy", "Txy_bal", "Pi", "T0")


class _Diag(C.Structure):
    _fields_ = [(k, C.c_double) for k in DIAG_NAMES]


class _Visc(C.Structure):
    _fields_ = [("law", C.c_int), ("omega_or_S", C.c_double)]


class _Desc(C.Structure):
    _fields_ = [("orders", _Orders), ("grid", _Grid), ("Kn", C.c_double), ("u_w", C.c_double),
                ("T_w", C.c_double), ("Pr", C.c_double), ("visc", _Visc), ("dt", C.c_double),
                ("cfl", C.c_double)]


EXPORTS = ("lbs_create", "lbs_batch_create", "lbs_destroy", "lbs_step", "lbs_run_to_steady",
           "lbs_moments", "lbs_profiles", "lbs_residual", "lbs_steps_taken", "lbs_info",
           "lbs_get_state", "lbs_set_state", "lbs_init_from_profiles", "lbs_init_free_molecular", "lbs_quadrature",
           "lbs_get_stream", "lbs_profile_steps", "lbs_moments_static", "lbs_set_tiling",
           "lbs_get_tiling", "lbs_last_error", "lbs_couette_diagnostics", "lbs_diagnostics",
           "lbs_set_finalize", "lbs_couette_nonlinear_velocity", "lbs_set_wait_limit", "lbs_clear_status",
           "lbs_probe_fma_rate",
           # the warm-start network (bound in warmstart.py)
           "lbs_mlp_create", "lbs_mlp_destroy", "lbs_mlp_num_params", "lbs_mlp_set_params",
           "lbs_mlp_get_params", "lbs_mlp_forward", "lbs_mlp_loss_grad", "lbs_mlp_adam",
           "lbs_mlp_get_stream")


def load(build_if_missing=True):
    """Load liblbs.so (building it in-tree first if needed); raises if unavailable."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and _build._stale():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError("liblbs.so not built (run paper_1702_01335_gb300.build.build())")
        lib = C.CDLL(path)
        P, D, L = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_long)
        H = C.POINTER(C.c_void_p)
        lib.lbs_create.argtypes = [H, _Orders, _Grid, C.c_double, C.c_double, C.c_double, C.c_double,
                                   _Visc, C.c_int, C.c_double, P]
        lib.lbs_batch_create.argtypes = [H, C.POINTER(_Desc), C.c_int, C.c_int, P]
        lib.lbs_destroy.argtypes = [P]
        lib.lbs_step.argtypes = [P, C.c_long]
        lib.lbs_run_to_steady.argtypes = [P, C.c_double, C.c_long, C.c_int, L]
        lib.lbs_moments.argtypes = [P, C.c_int, D]
        lib.lbs_profiles.argtypes = [P, C.c_int, D]
        lib.lbs_residual.argtypes = [P, C.c_int, D]
        lib.lbs_steps_taken.argtypes = [P, C.c_int, L]
        lib.lbs_info.argtypes = [P, C.c_int, L, D]
        lib.lbs_get_state.argtypes = [P, C.c_int, P, C.c_int]
        lib.lbs_set_state.argtypes = [P, C.c_int, P, C.c_int]
        lib.lbs_init_from_profiles.argtypes = [P, C.c_int, D]
        lib.lbs_init_free_molecular.argtypes = [P, C.c_int]
        lib.lbs_quadrature.argtypes = [C.c_int, C.c_int, D, D]
        lib.lbs_couette_diagnostics.argtypes = [D, C.c_int, C.c_double, C.c_int, C.c_double, C.c_double,
                                                C.POINTER(_Diag)]
        lib.lbs_diagnostics.argtypes = [P, C.c_int, C.POINTER(_Diag)]
        lib.lbs_couette_nonlinear_velocity.argtypes = [D, C.c_int, C.c_double, C.c_int, D, D]
        lib.lbs_set_finalize.argtypes = [P, C.c_int, C.POINTER(C.c_int)]
        lib.lbs_get_stream.argtypes = [P, H]
        lib.lbs_profile_steps.argtypes = [P, C.c_long, D]
        lib.lbs_moments_static.argtypes = [P, C.c_int, P, P]
        lib.lbs_set_tiling.argtypes = [P, C.c_int, C.c_int, C.c_int]
        lib.lbs_set_wait_limit.argtypes = [P, C.c_uint]
        lib.lbs_clear_status.argtypes = [P]
        lib.lbs_probe_fma_rate.argtypes = [D, D]
        I = C.POINTER(C.c_int)
        lib.lbs_get_tiling.argtypes = [P, I, I, I, I, L]
        lib.lbs_last_error.restype = C.c_char_p
        for name in EXPORTS:
            if name != "lbs_last_error":
                getattr(lib, name).restype = C.c_int
        _lib = lib
        return lib


def _check(st):
    if st != 0:
        raise LbsError(st, _lib.lbs_last_error().decode())


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def couette_diagnostics(prof, Nz, A, half, u_w, T_w=1.0):
    """Half-channel diagnostics (host only) from profiles [14, Nz] in PROFILE_NAMES
    order: a dict over DIAG_NAMES (see lbs_diag in include/lbs.h)."""
    lib = load()
    prof = np.ascontiguousarray(prof, dtype=np.float64)
    if prof.shape != (14, Nz):
        raise ValueError("profiles must have shape (14, Nz)")
    d = _Diag()
    _check(lib.lbs_couette_diagnostics(_dptr(prof), Nz, A, half, u_w, T_w, C.byref(d)))
    return {k: getattr(d, k) for k in DIAG_NAMES}


def couette_nonlinear_velocity(prof, Nz, A, half):
    """(z_s, u_nl(z_s)) over the half channel, Eq. (uy_nl), from profiles [14, Nz]."""
    lib = load()
    prof = np.ascontiguousarray(prof, dtype=np.float64)
    if prof.shape != (14, Nz):
        raise ValueError("profiles must have shape (14, Nz)")
    S = Nz if half else Nz // 2
    z, u = np.zeros(S), np.zeros(S)
    _check(lib.lbs_couette_nonlinear_velocity(_dptr(prof), Nz, A, half, _dptr(z), _dptr(u)))
    return z, u


def probe_fma_rate():
    """(FP64, FP32) fused multiply-add rates of the current device in FLOP/s."""
    lib = load()
    a, b = C.c_double(), C.c_double()
    _check(lib.lbs_probe_fma_rate(C.byref(a), C.byref(b)))
    return a.value, b.value


def quadrature(kind, Q):
    """The solver's Gauss rule (host only): kind 0 full range, 1 half range."""
    lib = load()
    x, w = np.zeros(Q), np.zeros(Q)
    _check(lib.lbs_quadrature(kind, Q, _dptr(x), _dptr(w)))
    return x, w


@dataclasses.dataclass
class State:
    """A stored state as lbs_get_state returns it: d[Nz, Q], the deviations f / w - 1 in
    the storage dtype, and (FP32 storage) r[Nz, Q] int16, the rounding residuals in units
    of 2^-15 ulp(d); None with FP64 storage."""
    d: np.ndarray
    r: object = None

    def normalised(self):
        """f / w = 1 + d + r 2^-15 ulp(d) as float64 (exact: every term is exact in FP64)."""
        return 1.0 + self.deviation()

    def deviation(self):
        """d + r 2^-15 ulp(d) as float64."""
        d = self.d.astype(np.float64)
        if self.r is None:
            return d
        E = ((self.d.view(np.uint32) >> 23) & 0xFF).astype(np.int64)
        lo = np.where(E >= 39, self.r.astype(np.float64) * np.exp2(np.clip(E, 39, 255) - 165.0), 0.0)
        return d + lo


@dataclasses.dataclass
class Instance:
    """One Couette problem (see lbs_instance_desc in include/lbs.h).

    Qx, Qy: full-range Gauss-Hermite nodes along the flow and across it; Qy = 0 selects
    the paper's reduced phi / chi model (the transverse momentum integrated out).
    Qz: half-range nodes per sign of p_z.  N_eq: equilibrium expansion order.
    Nz cells; A: tanh stretching (0: uniform).  half = 1: the upper half channel with
    the bounce-back centre line (Nz cells of a 2 Nz grid).  Kn, u_w, T_w, Pr; the
    viscosity law (power: omega; Sutherland: S).  dt > 0 is used as given, else
    dt = cfl * min dz / max |p_z|."""
    Qx: int = 4
    Qy: int = 4
    Qz: int = 4
    N_eq: int = 3
    Nz: int = 32
    A: float = 0.0
    half: int = 0
    Kn: float = 0.1
    u_w: float = 0.1
    T_w: float = 1.0
    Pr: float = 1.0
    visc_law: int = VISC_POWER
    visc_param: float = 1.0
    dt: float = 0.0
    cfl: float = 0.5

    def desc(self):
        return _Desc(_Orders(self.Qx, self.Qy, self.Qz, self.N_eq), _Grid(self.Nz, self.A, self.half),
                     self.Kn, self.u_w, self.T_w, self.Pr, _Visc(self.visc_law, self.visc_param),
                     self.dt, self.cfl)

    @property
    def Q(self):
        """Stored values per cell (Qy = 0, the phi / chi model: two fields per node)."""
        return 2 * self.Qx * (self.Qy if self.Qy else 2) * self.Qz


def _torch_stream():
    """torch's current CUDA stream if it is a created stream (the legacy default
    stream cannot be captured into CUDA graphs; then the library makes its own)."""
    try:
        import torch
        if torch.cuda.is_available():
            h = torch.cuda.current_stream().cuda_stream
            return C.c_void_p(h) if h else None
    except Exception:
        pass
    return None


class Solver:
    """A batch of Couette instances advanced together on one GPU stream."""

    def __init__(self, instances, precision=LBS_FP64, stream=None):
        if isinstance(instances, Instance):
            instances = [instances]
        self.instances = list(instances)
        self.lib = load()
        arr = (_Desc * len(self.instances))(*[i.desc() for i in self.instances])
        self.h = C.c_void_p()
        st = _torch_stream() if stream is None else C.c_void_p(stream)
        _check(self.lib.lbs_batch_create(C.byref(self.h), arr, len(self.instances), precision, st))
        self.precision = precision
        self.dtype = np.float32 if precision == LBS_FP32 else np.float64

    def close(self):
        if getattr(self, "h", None):
            self.lib.lbs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def stream_handle(self):
        """cudaStream_t (as an int) the solver queues its work on."""
        out = C.c_void_p()
        _check(self.lib.lbs_get_stream(self.h, C.byref(out)))
        return out.value or 0

    def torch_stream(self):
        """The solver's stream as a torch.cuda.ExternalStream (for events and ordering)."""
        import torch
        return torch.cuda.ExternalStream(self.stream_handle)

    def step(self, nsteps=1):
        _check(self.lib.lbs_step(self.h, int(nsteps)))

    def set_tiling(self, V, ZT, fuse=None):
        if fuse is None:
            fuse = self.tiling()["fuse"]
        _check(self.lib.lbs_set_tiling(self.h, int(V), int(ZT), int(fuse)))

    def tiling(self):
        v, z, f, n, sm = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_long()
        _check(self.lib.lbs_get_tiling(self.h, C.byref(v), C.byref(z), C.byref(f), C.byref(n), C.byref(sm)))
        return {"V": v.value, "ZT": z.value, "fuse": f.value, "ctas": n.value, "smem": sm.value}

    def profile_steps(self, nsteps):
        """Event-timed steps: (stage-kernel ms, finalise-kernel ms, whole-step ms), summed."""
        out = np.zeros(3)
        _check(self.lib.lbs_profile_steps(self.h, int(nsteps), _dptr(out)))
        return tuple(out)

    def state_bytes(self):
        """Bytes of every instance's state in the layout of lbs_get_state (d, then the
        FP32 residuals)."""
        esize = 6 if self.precision == LBS_FP32 else 8
        return sum(i.Nz * i.Q for i in self.instances) * esize

    def set_wait_limit(self, spins):
        """Spins of the stage kernel's bounded wait for its bulk copies (failure tests)."""
        _check(self.lib.lbs_set_wait_limit(self.h, int(spins)))

    def clear_status(self):
        _check(self.lib.lbs_clear_status(self.h))

    def moments_static(self, inst, f_dev_ptr, prof_dev_ptr):
        """Profiles [14][Nz] (FP64, device) of the device state at f_dev_ptr, computed
        without any device allocation (lbs_moments_static); queued on the solver's stream."""
        _check(self.lib.lbs_moments_static(self.h, inst, C.c_void_p(f_dev_ptr), C.c_void_p(prof_dev_ptr)))

    def get_state_all_ptr(self, ptr, to_host=True):
        """Copy every instance's state, concatenated, to the buffer at address ptr."""
        _check(self.lib.lbs_get_state(self.h, -1, C.c_void_p(ptr), int(to_host)))

    def set_state_all_ptr(self, ptr, from_host=True):
        """Set every instance's state from one concatenated buffer at address ptr."""
        _check(self.lib.lbs_set_state(self.h, -1, C.c_void_p(ptr), int(from_host)))

    def moments_all_ptr(self, ptr):
        """Profiles of every instance ([8][Nz] each, concatenated) into host memory at ptr."""
        _check(self.lib.lbs_moments(self.h, -1, C.cast(C.c_void_p(ptr), C.POINTER(C.c_double))))

    def run_to_steady(self, tol=1e-8, max_steps=1_000_000, check_every=100, raise_on_fail=True):
        out = (C.c_long * len(self.instances))()
        st = self.lib.lbs_run_to_steady(self.h, tol, int(max_steps), int(check_every), out)
        if st != 0 and (raise_on_fail or st != 4):
            _check(st)
        return np.array(out[:], dtype=np.int64)

    def info(self, inst=0):
        out = (C.c_long * 4)()
        dt = C.c_double()
        _check(self.lib.lbs_info(self.h, inst, out, C.byref(dt)))
        return {"Q": out[0], "Nz": out[1], "QxQy": out[2], "esize": out[3], "dt": dt.value}

    def moments(self, inst=0):
        Nz = self.instances[inst].Nz
        a = np.zeros((8, Nz))
        _check(self.lib.lbs_moments(self.h, inst, _dptr(a)))
        return dict(zip(MOMENT_NAMES, a))

    def profiles(self, inst=0):
        Nz = self.instances[inst].Nz
        a = np.zeros((14, Nz))
        _check(self.lib.lbs_profiles(self.h, inst, _dptr(a)))
        return dict(zip(PROFILE_NAMES, a))

    def set_finalize(self, mode):
        """0 auto, 1 one thread per cell, 2 one warp per cell; returns True if the warp layout is used."""
        w = C.c_int()
        _check(self.lib.lbs_set_finalize(self.h, int(mode), C.byref(w)))
        return bool(w.value)

    def diagnostics(self, inst=0):
        """u_slip, u'(0), nu, mass flow, T_xy, Pi, T_0 of instance inst (dict over DIAG_NAMES)."""
        d = _Diag()
        _check(self.lib.lbs_diagnostics(self.h, inst, C.byref(d)))
        return {k: getattr(d, k) for k in DIAG_NAMES}

    def nonlinear_velocity(self, inst=0):
        """(z_s, u_nl) of instance inst: the departure from the straight profile, Eq. (uy_nl)."""
        I = self.instances[inst]
        p = self.profiles(inst)
        return couette_nonlinear_velocity(np.stack([p[k] for k in PROFILE_NAMES]), I.Nz, I.A, I.half)

    def residual(self, inst=0):
        r = C.c_double()
        _check(self.lib.lbs_residual(self.h, inst, C.byref(r)))
        return r.value

    def steps_taken(self, inst=0):
        r = C.c_long()
        _check(self.lib.lbs_steps_taken(self.h, inst, C.byref(r)))
        return r.value

    def get_state(self, inst=0):
        """The stored state of instance inst (a State: deviations d and, with FP32
        storage, the residuals r), copied to host arrays."""
        I = self.instances[inst]
        n = I.Nz * I.Q
        esize = np.dtype(self.dtype).itemsize
        buf = np.zeros(n * esize + (2 * n if self.precision == LBS_FP32 else 0), dtype=np.uint8)
        _check(self.lib.lbs_get_state(self.h, inst, buf.ctypes.data_as(C.c_void_p), 1))
        d = buf[:n * esize].view(self.dtype).reshape(I.Nz, I.Q).copy()
        r = buf[n * esize:].view(np.int16).reshape(I.Nz, I.Q).copy() if self.precision == LBS_FP32 else None
        return State(d, r)

    def populations(self, inst=0):
        """Normalised populations f_k / w_k, [Nz, Q], float64."""
        return self.get_state(inst).normalised()

    def get_state_device(self, inst, out_ptr):
        """Copy instance inst's state (lbs_get_state layout) to device memory at out_ptr."""
        _check(self.lib.lbs_get_state(self.h, inst, C.c_void_p(out_ptr), 0))

    def set_state(self, inst, state):
        """Set instance inst from a State (or a bare deviation array d: residuals zero)."""
        I = self.instances[inst]
        if not isinstance(state, State):
            state = State(np.asarray(state), None)
        d = np.ascontiguousarray(state.d, dtype=self.dtype).reshape(I.Nz, I.Q)
        parts = [d.view(np.uint8).ravel()]
        if self.precision == LBS_FP32:
            r = np.zeros((I.Nz, I.Q), np.int16) if state.r is None else np.ascontiguousarray(state.r, np.int16)
            parts.append(r.view(np.uint8).ravel())
        buf = np.ascontiguousarray(np.concatenate(parts))
        _check(self.lib.lbs_set_state(self.h, inst, buf.ctypes.data_as(C.c_void_p), 1))

    def set_state_device(self, inst, ptr):
        _check(self.lib.lbs_set_state(self.h, inst, C.c_void_p(ptr), 0))

    def init_from_profiles(self, inst, prof):
        """prof: [8, Nz] in the order of MOMENT_NAMES (P rows unused)."""
        prof = np.ascontiguousarray(prof, dtype=np.float64)
        _check(self.lib.lbs_init_from_profiles(self.h, inst, _dptr(prof)))

    def init_free_molecular(self, inst):
        """Seed instance inst with the free-molecular state (each velocity the equilibrium of
        the wall it left, cells at unit density): a start for strongly rarefied flows."""
        _check(self.lib.lbs_init_free_molecular(self.h, inst))
