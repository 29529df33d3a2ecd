"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same
seeded inputs, element by element (FP64 storage) and profile by profile (FP32
storage), at sizes that span several z-tiles, several velocity chunks and ragged
tails, plus the edge cases of the method."""
import math

import numpy as np
import pytest

import workloads as W
from tests._pair import gpu_f, oracle_of, profile_errors, rel_err, same_state, solver_of

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12     # relative, element-wise after tens of steps
FP32_TOL = 2e-5      # relative per profile after tens of steps (FP32 storage)


def _lbs():
    import paper_1702_01335_gb300 as P
    return P


RAGGED = dict(Qx=6, Qy=5, Qz=7, N_eq=4, Nz=37, A=0.9, Kn=0.3, u_w=0.4, T_w=1.0, Pr=2.0 / 3.0,
              visc_law=1, visc_param=0.5239)


@pytest.mark.parametrize("params,steps", [(W.C1, 40), (RAGGED, 25)])
def test_fp64_state_matches_oracle(params, steps):
    P = _lbs()
    o = oracle_of(params, dt=None)
    s = solver_of(params, o.dt, P.LBS_FP64)
    o.step(steps)
    s.step(steps)
    f_gpu = gpu_f(s, o)
    f_ora = o.f[3:3 + o.Nz]
    assert rel_err(f_gpu, f_ora) < FP64_TOL
    errs = profile_errors(s.profiles(), o.profiles())
    assert max(errs.values()) < FP64_TOL, "profile errors: " + repr(sorted(errs.items(), key=lambda kv: -kv[1]))
    assert s.steps_taken() == steps


def test_fp64_residual_sequence_matches_oracle():
    P = _lbs()
    o = oracle_of(RAGGED, dt=None)
    s = solver_of(RAGGED, o.dt, P.LBS_FP64)
    r = o.step(12, residuals=True)
    # the first step divides by ||u_x|| of the rest state (zero up to rounding), so its
    # residual is not comparable; every later one is
    s.step(1)
    for it in range(1, 12):
        s.step(1)
        assert abs(s.residual() / r[it] - 1) < 1e-9, (it, s.residual(), r[it])
    assert r[-1] > 0


# Q = 30: rows of 120 bytes are not 16-byte aligned, so the stage kernel takes its
# plain-load path instead of TMA bulk copies
UNALIGNED = dict(RAGGED, Qx=3, Qy=1, Qz=5, N_eq=2, Nz=19)


@pytest.mark.parametrize("params", [RAGGED, UNALIGNED])
def test_fp32_profiles_match_oracle(params):
    P = _lbs()
    o = oracle_of(params, dt=None)
    s = solver_of(params, o.dt, P.LBS_FP32)
    o.step(30)
    s.step(30)
    errs = profile_errors(s.profiles(), o.profiles())
    assert max(errs.values()) < FP32_TOL, "profile errors: " + repr(sorted(errs.items(), key=lambda kv: -kv[1]))


# Q / 2 = 1350 (even): the velocity-pair layout of FP32 storage applies at V = 2 and 4, with
# a ragged last chunk at each (1350 = 5 x 256 + 70 = 2 x 512 + 326 velocities)
PAIRS = dict(RAGGED, Qx=9, Qy=6, Qz=25, Nz=21)


@pytest.mark.parametrize("V,ZT,fuse", [(2, 5, 0), (4, 16, 2), (4, 7, 0), (2, 24, 1)])
def test_fp32_velocity_pair_tilings_match_oracle(V, ZT, fuse):
    """FP32 storage in every velocity-pair tiling (the packed two-lane update) against the
    FP64 oracle, and against the one-velocity-per-thread layout (V = 1) to FP32 rounding."""
    P = _lbs()
    o = oracle_of(PAIRS, dt=None)
    s = solver_of(PAIRS, o.dt, P.LBS_FP32)
    s.set_tiling(V, ZT, fuse)
    t = s.tiling()
    assert t["V"] == V and t["fuse"] == fuse
    one = solver_of(PAIRS, o.dt, P.LBS_FP32)
    one.set_tiling(1, 4, 0)
    o.step(25)
    s.step(25)
    one.step(25)
    errs = profile_errors(s.profiles(), o.profiles())
    assert max(errs.values()) < FP32_TOL, "profile errors: " + repr(sorted(errs.items(), key=lambda kv: -kv[1]))
    a, b = s.populations(), one.populations()
    assert np.abs(a - b).max() < 1e-5 * np.abs(b).max()


def test_fp32_pair_layout_needs_even_half_range():
    """Q / 2 odd: V = 2 and 4 are refused in FP32 (a pair would straddle a chunk start) and
    the untuned default takes one velocity per thread; FP64 takes them, and no V = 8."""
    P = _lbs()
    p = dict(RAGGED, Qx=3, Qy=3, Qz=5, Nz=12)  # Q / 2 = 45
    s = solver_of(p, 0.002, P.LBS_FP32)
    assert s.tiling()["V"] == 1
    for V in (2, 4):
        with pytest.raises(P.LbsError) as e:
            s.set_tiling(V, 8, 0)
        assert e.value.status == P.LBS_ERR_ARG
    d = solver_of(p, 0.002, P.LBS_FP64)
    d.set_tiling(4, 8, 0)
    with pytest.raises(P.LbsError):
        d.set_tiling(8, 8, 0)


@pytest.mark.parametrize("fuse", [None, 2])
def test_batch_of_uneven_instances_matches_single_runs(fuse):
    """A batch of instances of different Nz, Q and gas laws equals each run alone, also
    when its two halves step on two streams (fuse = 2; 15 steps: one 8-step graph and
    7 directly launched steps)."""
    P = _lbs()
    ps = W.sweep(5, seed=11, nz_set=(6, 17, 24), qx_set=(3, 4, 6), qz_set=(2, 4, 5))
    dts = [oracle_of(p, None).dt for p in ps]
    dt = min(dts)
    s = solver_of(ps, dt, P.LBS_FP64)
    if fuse is not None:
        t = s.tiling()
        s.set_tiling(t["V"], t["ZT"], fuse)
        assert s.tiling()["fuse"] == fuse
    s.step(15)
    for b, p in enumerate(ps):
        o = oracle_of(p, dt)
        o.step(15)
        assert rel_err(gpu_f(s, o, b), o.f[3:3 + o.Nz]) < FP64_TOL, b


def test_split_stepping_is_bitwise_unsplit_stepping():
    """Split stepping (the batch's halves on two streams) runs the same arithmetic per
    instance: after 11 steps (one 8-step graph and 3 direct steps) the FP32 states equal
    those of unsplit stepping bit for bit."""
    P = _lbs()
    ps = W.sweep(5, seed=13, nz_set=(12, 20, 33), qx_set=(3, 4), qz_set=(2, 3))
    dt = min(oracle_of(p, None).dt for p in ps)
    out = []
    for fuse in (0, 2):
        s = solver_of(ps, dt, P.LBS_FP32)
        t = s.tiling()
        s.set_tiling(t["V"], t["ZT"], fuse)
        s.step(11)
        out.append([s.get_state(b) for b in range(len(ps))])
    for a, b in zip(*out):
        assert same_state(a, b)


def test_edge_minimum_sizes():
    """Nz = 6 (three ghost-fed cells per wall) and the smallest velocity set (Q = 2, N = 0)."""
    P = _lbs()
    for p in (dict(W.C1, Nz=6), dict(W.C1, Qx=1, Qy=1, Qz=1, N_eq=0, Nz=8)):
        o = oracle_of(p, None)
        s = solver_of(p, o.dt, P.LBS_FP64)
        o.step(20)
        s.step(20)
        assert rel_err(gpu_f(s, o), o.f[3:3 + o.Nz]) < FP64_TOL


def test_warm_start_and_checkpoint():
    """init_from_profiles seeds n Gx Gy Gz (1 + S); get/set_state round-trips."""
    P = _lbs()
    p = RAGGED
    o = oracle_of(p, None)
    s = solver_of(p, o.dt, P.LBS_FP64)
    z = o.xc[3:3 + o.Nz]
    prof = np.zeros((8, o.Nz))
    prof[0] = 1.0 + 0.05 * np.cos(np.pi * z)
    prof[1] = 0.8 * p["u_w"] * 2 * z
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
    st = s.get_state(0)
    s.step(5)
    s.set_state(0, st)
    assert same_state(s.get_state(0), st)
    s.step(5)
    o.step(5)
    assert rel_err(gpu_f(s, o), o.f[3:3 + o.Nz]) < FP64_TOL


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_free_molecular_seed(prec):
    """lbs_init_free_molecular: every velocity carries the discrete equilibrium of the wall
    it left (the oracle's equilibrium at n = 1, u = -u_w for p_z > 0, +u_w for p_z < 0,
    T_w), each cell at unit density; FP64 to 1e-12, FP32 to its rounding."""
    P = _lbs()
    p = RAGGED
    o = oracle_of(p, None)
    s = solver_of(p, o.dt, P.LBS_FP64 if prec == "fp64" else P.LBS_FP32)
    s.init_free_molecular(0)
    z = np.zeros(3)
    fb = o.equilibrium(1.0, np.array([-p["u_w"], 0.0, 0.0]), p["T_w"], z, with_S=False)
    ft = o.equilibrium(1.0, np.array([p["u_w"], 0.0, 0.0]), p["T_w"], z, with_S=False)
    f = np.where(o.velocities()[:, 2] > 0, fb, ft)
    f = f / f.sum()
    got = gpu_f(s, o)
    tol = FP64_TOL if prec == "fp64" else 1e-6
    assert rel_err(got, np.broadcast_to(f, got.shape)) < tol
    prof = s.profiles()
    assert np.abs(prof["n"] - 1.0).max() < (1e-13 if prec == "fp64" else 1e-6)
    assert np.abs(prof["ux"]).max() < 1e-12 + (0 if prec == "fp64" else 1e-6)
    s.step(5)  # and steps from there
    assert np.all(np.isfinite(s.profiles()["T"]))


@pytest.mark.parametrize("prec,fuse,big", [("fp64", 1, True), ("fp32", 1, True), ("fp32", 0, True),
                                           ("fp32", 2, True), ("fp32", 1, False)])
def test_whole_batch_state_and_moments(prec, fuse, big):
    """Whole-batch state and moments (instance index -1) on a batch of unequal instances:
    lbs_get_state lays out every d, then every FP32 residual, in instance order, and
    lbs_moments every instance's [8][Nz] rows, bit for bit as the per-instance calls give
    them.  lbs_set_state of the whole batch restores the state bit for bit and leaves the
    profiles, and the steps that follow, exactly as a solver restored instance by
    instance: from host memory with five C3-sized instances among the small ones (60 MB
    in FP32, 80 MB in FP64: copied in two or three groups, each analysed behind the next
    group's copy), from host memory without them (one copy), and from device memory.  A
    non-finite value in one instance of the buffer is rejected."""
    import torch
    P = _lbs()
    pr = P.LBS_FP64 if prec == "fp64" else P.LBS_FP32
    ps = [dict(W.C1, Nz=40), RAGGED, dict(W.C1, Kn=1.0, Nz=37), PAIRS, dict(RAGGED, Nz=64, u_w=0.2),
          dict(W.C1, Kn=0.3, Nz=51)]
    if big:
        ps = [p for i, q in enumerate(ps) for p in ([q, dict(W.C3, Kn=10.0 * (i + 1))] if i < 5 else [q])]
    dt = min(oracle_of(p, None).dt for p in ps)
    s = solver_of(ps, dt, pr)
    t = s.tiling()
    s.set_tiling(t["V"], t["ZT"], fuse)
    s.step(7)
    nb = s.state_bytes()
    buf = np.zeros(nb, np.uint8)
    s.get_state_all_ptr(buf.ctypes.data)
    per = [s.get_state(b) for b in range(len(ps))]
    d = np.concatenate([st.d.view(np.uint8).ravel() for st in per])
    r = [st.r.view(np.uint8).ravel() for st in per] if pr == P.LBS_FP32 else []
    assert np.array_equal(buf, np.concatenate([d] + r))
    mom = np.zeros(8 * sum(p["Nz"] for p in ps))
    s.moments_all_ptr(mom.ctypes.data)
    ref = np.concatenate([np.stack(list(s.moments(b).values())).ravel() for b in range(len(ps))])
    assert np.array_equal(mom, ref)
    prof0 = [s.profiles(b) for b in range(len(ps))]

    one = solver_of(ps, dt, pr)  # restored instance by instance
    one.set_tiling(t["V"], t["ZT"], fuse)
    for b, st in enumerate(per):
        one.set_state(b, st)
    s.step(5)
    s.set_state_all_ptr(buf.ctypes.data, from_host=True)
    for b in range(len(ps)):
        assert same_state(s.get_state(b), per[b]), b
        pa, pb = s.profiles(b), one.profiles(b)
        assert all(np.array_equal(pa[k], pb[k]) for k in pa), b
        assert all(np.abs(pa[k] - prof0[b][k]).max() < 2e-6 for k in pa), b  # the moments of that state
    s.step(3)
    one.step(3)
    for b in range(len(ps)):
        assert same_state(s.get_state(b), one.get_state(b)), b

    dev = torch.from_numpy(buf).cuda()
    torch.cuda.synchronize()
    s.set_state_all_ptr(dev.data_ptr(), from_host=False)
    for b in range(len(ps)):
        assert same_state(s.get_state(b), per[b]), b

    bad = buf.copy()
    esize = 4 if pr == P.LBS_FP32 else 8
    k = (ps[0]["Nz"] * one.info(0)["Q"] + 11) * esize  # an element of instance 1
    bad[k:k + esize] = np.frombuffer(np.array([np.inf], dtype=np.float32 if esize == 4 else np.float64).tobytes(),
                                     np.uint8)
    with pytest.raises(P.LbsError) as e:
        s.set_state_all_ptr(bad.ctypes.data, from_host=True)
    assert e.value.status == 3
    s.clear_status()
    s.set_state_all_ptr(buf.ctypes.data, from_host=True)
    s.step(3)
    for b in range(len(ps)):
        assert same_state(s.get_state(b), one.get_state(b)), b
    s.close()
    one.close()


def test_nonfinite_inputs_rejected():
    P = _lbs()
    s = solver_of(W.C1, 0.004, P.LBS_FP64)
    prof = np.ones((8, 32))
    prof[2, 5] = np.nan
    with pytest.raises(P.LbsError) as e:
        s.init_from_profiles(0, prof)
    assert e.value.status == 3
    st = s.get_state(0)
    st.d[3, 7] = np.inf
    with pytest.raises(P.LbsError) as e:
        s.set_state(0, st)
    assert e.value.status == 3


def test_run_to_steady_c1():
    """Config C1 marches to R < 1e-8; the step count and profiles agree with the oracle."""
    P = _lbs()
    o = oracle_of(W.C1, None)
    s = solver_of(W.C1, o.dt, P.LBS_FP64)
    steps = s.run_to_steady(1e-8, max_steps=20000, check_every=50)[0]
    r = o.step(int(steps), residuals=True)
    first = int(np.nonzero(r < 1e-8)[0][0]) + 1
    assert first == steps
    assert rel_err(gpu_f(s, o), o.f[3:3 + o.Nz]) < 1e-10


@pytest.mark.parametrize("fuse", [0, 2])
def test_run_to_steady_batch_retires_and_restores(fuse):
    """A batch whose instances converge at different steps: run_to_steady drops the tiles of
    retired instances and, once few cells are live, finalises them a warp each.  Each
    instance takes the steps it takes alone and ends in the same state (the layouts agree
    to FP64 rounding); afterwards the full tile list and the batch's layout are back, so a
    further step of the batch equals a step of each instance alone."""
    P = _lbs()
    # 740 cells: one thread per cell at first, a warp per cell once fewer than 608 are live
    ps = [dict(W.C1, Kn=kn, Nz=nz) for kn, nz in ((0.1, 160), (0.3, 120), (1.0, 140), (0.15, 100), (3.0, 120),
                                                 (0.2, 100))]
    dt = min(oracle_of(p, None).dt for p in ps)
    s = solver_of(ps, dt, P.LBS_FP64)
    t = s.tiling()
    s.set_tiling(t["V"], t["ZT"], fuse)
    t = s.tiling()
    steps = s.run_to_steady(1e-8, max_steps=30000, check_every=50)
    assert len(set(steps)) > 2  # they retire at different checks
    assert s.tiling() == t  # every tile is back
    s.step(3)
    for b, p in enumerate(ps):
        a = solver_of(p, dt, P.LBS_FP64)
        sa = a.run_to_steady(1e-8, max_steps=30000, check_every=50)[0]
        assert sa == steps[b], (b, sa, steps[b])
        a.step(3)
        ref = a.populations()
        assert np.abs(s.populations(b) - ref).max() < 1e-11 * np.abs(ref).max(), b
        a.close()


def test_c2_full_size_sampled_parity():
    """Config C2 at full size in the benchmark's launch shape (a batch of replicas):
    after a few steps every sampled replica matches the oracle's single solve."""
    P = _lbs()
    ref = oracle_of(W.C2, None)
    ref.step(4)
    # finalisation mode 1 is the layout of the benchmark's 256-replica batch
    for prec, tol, mode in ((P.LBS_FP64, FP64_TOL, 1), (P.LBS_FP64, FP64_TOL, 2), (P.LBS_FP32, FP32_TOL, 1)):
        s = solver_of([W.C2] * 16, ref.dt, prec)
        assert s.set_finalize(mode) == (mode == 2)
        s.step(4)
        errs = [max(profile_errors(s.profiles(b), ref.profiles()).values()) for b in (0, 7, 15)]
        assert max(errs) < tol, (prec, errs)
        s.close()


def test_c4_sweep_sampled_parity():
    """Config C4 as the benchmark runs it: the 64-instance seed-1702 sweep in one batch
    (Nz 32 - 512, up to 16 x 4 x (2 x 48) velocities, both viscosity laws, each instance
    at its own CFL time step).  After 10 FP64 steps three sampled instances -- the one
    with the largest velocity set, the one with the most cells and the first -- equal
    per-instance oracle runs element by element (1e-12); every instance's profiles are
    finite and its mass conserved.  Then the same batch in FP32 storage on the
    benchmark's tiling matches the same oracle runs per profile."""
    P = _lbs()
    ps = W.sweep(64, W.SWEEP_SEED)
    q = [p["Qx"] * p["Qy"] * p["Qz"] for p in ps]
    picks = sorted({int(np.argmax(q)), int(np.argmax([p["Nz"] for p in ps])), 0})
    assert max(q) == 16 * 4 * 48 and max(p["Nz"] for p in ps) == 512
    s = solver_of(ps, 0.0, P.LBS_FP64)  # dt = 0: each instance's own CFL step
    s.step(10)
    refs = {}
    for b in picks:
        o = oracle_of(ps[b], s.info(b)["dt"])
        o.step(10)
        refs[b] = o
        assert rel_err(gpu_f(s, o, b), o.f[3:3 + o.Nz]) < FP64_TOL, (b, ps[b])
    for b in range(len(ps)):
        p = s.profiles(b)
        assert all(np.all(np.isfinite(v)) for v in p.values()), b
        assert abs(np.mean(p["n"]) - 1.0) < 1e-12, b  # uniform cells: mass = mean density
    s.close()
    s = solver_of(ps, 0.0, P.LBS_FP32)
    s.set_tiling(4, 12, 0)
    s.step(10)
    for b in picks:
        errs = profile_errors(s.profiles(b), refs[b].profiles(), uw=ps[b]["u_w"])
        assert max(errs.values()) < FP32_TOL, (b, errs)
    s.close()


def test_c3_high_kn_fp32_free_molecular_bound():
    """Config C3 (8192 velocities, Qz = 64) in FP32 storage: after a short march the shear
    stress is bounded by the ballistic value of Eq. (Txy_bal) and mass is conserved."""
    P = _lbs()
    o = oracle_of(W.C3, None)
    s = solver_of(W.C3, o.dt, P.LBS_FP32)
    s.step(20)
    o.step(20)
    errs = profile_errors(s.profiles(), o.profiles())
    assert max(errs[k] for k in ("n", "ux", "T", "Pxz", "Pxx", "Pzz")) < FP32_TOL, errs
    p = s.profiles()
    dz = np.diff(o.xf)
    assert abs(np.sum(p["n"] * dz) - 1.0) < 1e-6
    assert np.all(np.abs(p["Pxz"]) <= W.C3["u_w"] * math.sqrt(2 / math.pi) * 1.01)


@pytest.mark.parametrize("fin", [1, 2])
@pytest.mark.parametrize("V,ZT,fuse", [(1, 3, 1), (2, 7, 0), (4, 64, 1), (4, 5, 0)])
def test_tiling_does_not_change_results(V, ZT, fuse, fin):
    """Every work decomposition of the stage kernel, with the finalisation folded in
    or launched apart, one thread or one warp per cell, gives the oracle's state."""
    P = _lbs()
    o = oracle_of(RAGGED, dt=None)
    s = solver_of(RAGGED, o.dt, P.LBS_FP64)
    s.set_tiling(V, ZT, fuse)
    s.set_finalize(fin)
    t = s.tiling()
    assert t["V"] == V and t["ZT"] == ZT and t["fuse"] == fuse
    o.step(15)
    s.step(15)
    assert rel_err(gpu_f(s, o), o.f[3:3 + o.Nz]) < FP64_TOL


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_finalize_layouts_agree(prec):
    """One thread per cell and one warp per cell give the same states to rounding
    (FP64: ulps, grown by the dynamics to ~1e-13 in 30 steps; FP32 storage: the FP32
    rounding of the records), for a batch
    mixing a full and a half channel."""
    P = _lbs()
    from paper_1702_01335_gb300 import Instance, Solver
    p = P.LBS_FP64 if prec == "fp64" else P.LBS_FP32
    inst = [Instance(dt=0.002, **RAGGED), Instance(dt=0.002, half=1, **dict(RAGGED, Nz=20))]
    a, b = Solver(inst, precision=p), Solver(inst, precision=p)
    assert not a.set_finalize(1) and b.set_finalize(2)
    a.step(30)
    b.step(30)
    tol = FP64_TOL if prec == "fp64" else 1e-5
    for i in range(2):
        fa, fb = a.populations(i), b.populations(i)
        assert rel_err(fb, fa) < tol, i
        errs = profile_errors(b.profiles(i), a.profiles(i), uw=RAGGED["u_w"])
        assert max(errs.values()) < tol, errs


def test_autotuner_picks_a_valid_tiling():
    P = _lbs()
    from paper_1702_01335_gb300.autotune import autotune
    s = solver_of([W.C1] * 4, 0.004, P.LBS_FP32)
    before = s.get_state(0)
    r = autotune(s, candidates=((1, 8, 1), (2, 16, 0), (4, 99, 0)), steps=2)  # the last one is invalid
    assert (r["V"], r["ZT"], r["fuse"]) in ((1, 8, 1), (2, 16, 0))
    assert len(r["table"]) == 2
    assert s.tiling()["V"] == r["V"]
    assert same_state(s.get_state(0), before)  # tuning ran on a scratch solver
    assert s.steps_taken() == 0
