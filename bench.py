"""Benchmark: cell x velocity updates per second of the RK-3 step.

Workload (the metric's configuration, config C2): Maxwell molecules, Shakhov
Pr = 2/3, mu ~ T; Kn = 1, u_w = 0.5, T_w = 1; Nz = 128 cells stretched toward the
walls (A = 0.98); 8 x 8 full-range x 2 x 16 half-range = 2048 velocities,
equilibrium order 4; f stored in FP32 (deviations from the rest state with a
16-bit rounding residual) with FP64 moment sums.  One step is one
full RK-3 step (three stages: walls, WENO-5 advection, Shakhov relaxation,
moments, residual) of a batch of B = 256 independent replicas of C2 on each GPU
(256 MiB per state buffer, larger than the 129 MB L2, so no L2 flush is needed).

Output: one JSON line (rank 0).  `value` is the whole-job rate (all ranks) from
CUDA events on the solver's stream around exactly --steps steps after --warmup
steps, max time over ranks.  `e2e` repeats the measurement through the public
API with the state uploaded from pinned host memory and the profiles read back
every step.  `roofline` relates the stage kernels' live event time to their
algorithmic bytes (36 B per update and step in FP32) and the measured HBM copy
bandwidth.  `cpu_baseline` times the FP64 CPU oracle on a bounded sample.

--impl reference times that oracle (the only reference this method has) on the
host cores instead, with the same metric.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

BATCH = 256
# algorithmic HBM bytes per update per RK-3 step.  FP32: stage 1 reads d, writes d1 (8);
# stage 2 reads d, d1, writes d2 (12); stage 3 reads d, d2 and the 2-byte residual and
# writes d and the residual (16).  FP64: 16 + 24 + 24, no residual.
BYTES_PER_UPDATE = {"f32": 36, "f64": 64}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="lbs", choices=["lbs", "reference"])
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--precision", default=None, choices=["f32", "f64"],
                    help="default f32; f64 for the low-Mach workload, whose deviations FP32 does not resolve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-steady", action="store_true",
                    help="skip the time-to-steady-state comparison (plain vs batched vs warm-started)")
    ap.add_argument("--tiling", default=None,
                    help="V,ZT,fuse: use this stage-kernel tiling instead of the autotuner")
    ap.add_argument("--tuning-cache", default=None,
                    help="JSON cache of tile choices (default: the package's tuning_cache.json)")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3x32", "sweep", "tables", "luo"],
                    help="c2: the throughput workload (default; --precision f64 for the FP64 line); "
                         "c3x32: 32 replicas of config C3 (Kn = 100, 8192 velocities); sweep: the "
                         "64-instance seed-1702 sweep of config C4, timed per step and marched to "
                         "R < 1e-8 per instance; tables: the 20 half-channel runs of the paper's "
                         "Sec. VI tables; luo: the low-Mach runs of Sec. IV (Table luo); the last "
                         "three on one GPU")
    ap.add_argument("--model", default="full", choices=["full", "reduced"],
                    help="tables workload: the 3D velocity set (Q_y = 7) or the paper's phi / chi model")
    a = ap.parse_args()
    if a.precision is None:
        a.precision = "f64" if a.workload == "luo" else "f32"
    return a


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# FP64 floating-point operations of one cell x velocity update in one RK stage of the
# FP64 solver (an FMA counts two), counted from the stage kernel's source: the WENO-5
# correction of the interface ahead (differences 4, candidate corrections 6, smoothness
# indicators 18, weights 10 with 4 divisions, the weighted sum 8: 46), the divergence
# (5), the Shakhov factor (14), the target's deviation (6), the departure and the
# combine (8), and the 13 moment sums (26): 105 per update and stage, 315 per RK-3 step.
# Rounded to 300 (the stage-3 moments about the cell velocity add 10, stage 1's combine
# is 4 shorter): an under-count makes the reported fraction a lower bound.
FP64_FLOPS_PER_UPDATE_STEP = 300.0


class Clocks:
    """nvidia-smi samples (200 ms) during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu, self.lines, self.proc = gpu, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_c2(p=None):
    from oracle.oracle import Oracle
    p = p or W.C2
    return Oracle(p["Qx"], p["Qy"], p["Qz"], p["N_eq"], p["Nz"], A=p["A"], Kn=p["Kn"], uw=p["u_w"],
                  Tw=p["T_w"], Pr=p["Pr"], visc_law=p["visc_law"], visc_param=p["visc_param"])


def cpu_baseline(p=None, seconds=12.0):
    """The FP64 oracle as it stands on the host cores: one instance (C2 by default),
    whole RK-3 steps."""
    p = p or W.C2
    o = _oracle_c2(p)
    o.step(1)
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < seconds:
        o.step(1)
        n += 1
    dt = time.perf_counter() - t0
    upd = p["Nz"] * 2 * p["Qx"] * p["Qy"] * p["Qz"] * n
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": upd / dt, "unit": "updates/s", "cores": cores, "kind": "oracle",
            "sample": "one instance (%d cells x %d velocities), %d full RK-3 steps, FP64, "
                      "%.1f s" % (p["Nz"], 2 * p["Qx"] * p["Qy"] * p["Qz"], n, dt)}


def time_to_steady():
    """Wall time to R < 1e-7 (FP32 storage; 60000-step budget) of 256 held-out sweep
    draws: the plain single-instance solver from rest (a sample of 16, extrapolated),
    one batched launch from rest, and one batched launch from the warm-start network
    trained on 2000 steady solves."""
    try:
        from paper_1702_01335_gb300.warmstart import evaluate
        r = evaluate(W.warm_start_draws(2000, W.TRAIN_SEED), W.warm_start_draws(256, W.HELDOUT_SEED),
                     n_plain=16)
        r["workload"] = ("sweep draws: Kn log-uniform clipped to [0.05, 20], u_w in [0.05, 1], "
                         "Pr = 2/3, half mu ~ T^omega, half Sutherland; Nz 32-64, Qx 4-8, Qy 4, Qz 4-8; "
                         "FP32 storage; train seed 1703, held-out seed 1704")
        return r
    except Exception as e:  # reported, never fatal to the throughput line
        return {"error": "%s: %s" % (type(e).__name__, e)}


def whole_job(local_time, units_per_rank, dist=None, device="cpu"):
    """Whole-job rate of a run in which every rank processed units_per_rank units in
    local_time: (the slowest rank's time, all ranks' units / that time)."""
    import torch
    t = torch.tensor([float(local_time)], dtype=torch.float64, device=device)
    world = 1
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        world = dist.get_world_size()
    slowest = float(t.item())
    return slowest, units_per_rank * world / slowest


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    o = _oracle_c2()
    for _ in range(a.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        o.step(1)
    dt = time.perf_counter() - t0
    upd = W.C2["Nz"] * 2 * W.C2["Qx"] * W.C2["Qy"] * W.C2["Qz"] * a.steps
    v = upd / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    print(json.dumps({
        "impl": "reference", "metric": "cell x velocity updates/s (RK-3 steps)", "value": v,
        "unit": "updates/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "C2 Shakhov Maxwell molecules Kn=1 u_w=0.5 Nz=128 A=0.98 "
                               "Q=8x8x(2x16)=2048 N_eq=4", "sample": "one instance per step"},
        "cpu_baseline": {"value": v, "unit": "updates/s", "cores": cores, "kind": "oracle",
                         "sample": "one C2 instance per step, %d RK-3 steps" % a.steps},
        "e2e": {"value": v, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_small(a):
    """The paper-reproduction workloads, timed like the main line:
    tables  the 20 half-channel He / Ar runs of the Sec. VI tables in one batch (16 cells,
            7 x 7 x (2 x Q_n) velocities, Q_n = 7 or 30; or the phi / chi model);
    luo     the three low-Mach half-channel runs of Sec. IV (Table luo), FP64.
    Small and latency-bound: the line reports the stage and finalisation kernels' own
    times beside the step rate."""
    import torch
    from paper_1702_01335_gb300 import LBS_FP32, LBS_FP64, Instance, Solver
    torch.cuda.set_device(0)
    runs = W.paper_tables(reduced=a.model == "reduced") if a.workload == "tables" else W.luo_runs()
    inst = [Instance(**p) for _, p in runs]
    from paper_1702_01335_gb300.autotune import DEFAULT_CACHE, autotune
    s = Solver(inst, precision=LBS_FP32 if a.precision == "f32" else LBS_FP64)
    if a.tiling:
        s.set_tiling(*(int(x) for x in a.tiling.split(",")))
    else:
        autotune(s, candidates=tuple((V, ZT, F) for V in (1, 2) for ZT in (4, 6, 8, 16) for F in (0, 1, 2)),
                 steps=20, cache_file=a.tuning_cache or DEFAULT_CACHE)
    st = s.torch_stream()
    upd_step = sum(i.Nz * i.Q for i in inst)
    s.step(a.warmup)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        e0.record(st)
        s.step(a.steps)
        e1.record(st)
        torch.cuda.synchronize()
    ms = reduce(e0.elapsed_time(e1), "max")
    nprof = max(3, min(500, a.steps // 10))
    k_stage, k_fin, k_step = s.profile_steps(nprof)
    pinned = torch.empty(s.state_bytes(), dtype=torch.uint8, pin_memory=True)
    s.get_state_all_ptr(pinned.data_ptr(), to_host=True)
    nrows = sum(8 * i.Nz for i in inst)
    out_host = torch.empty(nrows, dtype=torch.float64, pin_memory=True)
    e2e_steps = max(3, min(500, a.steps // 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.set_state_all_ptr(pinned.data_ptr(), from_host=True)
        s.step(1)
        s.moments_all_ptr(out_host.data_ptr())
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    tl = s.tiling()
    line = {
        "metric": "cell x velocity updates/s (RK-3 steps)", "value": upd_step * a.steps / (ms * 1e-3),
        "unit": "updates/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": a.precision, "data": "synthetic",
        "config": {"workload": ("paper tables: 20 half channels (Ar, He; delta 0.1-40; u_w sqrt 2, "
                                "0.1 sqrt 2), Nz=16 A=0.98, N_eq=6, Sutherland, Pr=2/3; " + (
                                    "phi/chi model, Q=7x2x(2x7) or 7x2x(2x30)" if a.model == "reduced"
                                    else "3D set, Q=7x7x(2x7) or 7x7x(2x30)")) if a.workload == "tables" else
                               ("low Mach (Table luo): 3 half channels, k = 0.03, 0.1, 1 (S = 64, 32, 32; "
                                "Q = 2x2x(2x4), 2x2x(2x7), 2x2x(2x21)), phi/chi model, BGK, u_w = 1e-5, A = 0.98"),
                   "updates_per_step": upd_step,
                   "l2": "state (%d KiB) resident in L2: latency-bound" % (s.state_bytes() >> 10),
                   "tiling": {"V": tl["V"], "ZT": tl["ZT"], "fused_finalise": tl["fuse"]}},
        "kernels": {"stage_ms_per_step": k_stage / nprof, "finalize_ms_per_step": k_fin / nprof,
                    "profiled_step_ms": k_step / nprof},
        "e2e": {"value": upd_step * e2e_steps / e2e_s, "unit": "updates/s",
                "h2d_bytes_per_step": s.state_bytes(), "d2h_bytes_per_step": nrows * 8},
        "gpu_launches": {0: 6, 1: 3, 2: 12}[tl["fuse"]] * a.steps,
        "clocks": clk.summary(),
    }
    if a.workload == "luo":
        diag = [s.diagnostics(b) for b in range(len(runs))]
        line["diagnostics_after_timed_steps"] = {
            "k=%g" % lab["k"]: {"u_slip/u_w": d["u_slip"] / p["u_w"], "L u'(0)/2u_w": d["nu"],
                                "mflow/mflow_hydro": d["mflow"] / d["mflow_hydro"],
                                "Txy/Txy_bal": d["Txy"] / d["Txy_bal"]}
            for d, (lab, p) in zip(diag, runs)}
    if not a.no_cpu_baseline:
        pick = [r for r in runs if r[0].get("delta") == 1.0 or r[0].get("k") == 0.1][0]
        line["cpu_baseline"] = cpu_baseline_half(pick)
    print(json.dumps(line), flush=True)
    s.close()


def cpu_baseline_half(run, seconds=12.0):
    """The oracle on one run of a half-channel workload.  It has no half channel: it steps
    the full channel of 2 Nz cells, which costs two updates per half-channel update."""
    from oracle.oracle import Oracle
    label, p = run
    o = Oracle(p["Qx"], p["Qy"], p["Qz"], p["N_eq"], 2 * p["Nz"], A=p["A"], Kn=p["Kn"], uw=p["u_w"],
               Tw=p["T_w"], Pr=p["Pr"], visc_law=p["visc_law"], visc_param=p["visc_param"], dt=p.get("dt"))
    o.step(1)
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < seconds:
        o.step(1)
        n += 1
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": p["Nz"] * o.Q * n / dt, "unit": "updates/s", "cores": cores, "kind": "oracle",
            "sample": "%s as the full channel of %d cells (Q = %d), %d RK-3 steps in %.1f s, counted as "
                      "half-channel updates" % (json.dumps(label), 2 * p["Nz"], o.Q, n, dt)}


def run_sweep(a):
    """Config C4: the 64-instance sweep (numpy PCG64 seed 1702; Kn log-uniform in
    [0.01, 100], u_w in [0.05, 1], half mu ~ T^omega, half Sutherland; Nz 32-512, up to
    16 x 4 x (2 x 48) velocities), every instance at its own CFL time step, in one batch.
    Timed like the main line; then marched to R < 1e-8 per instance (device-side
    retirement) within a step budget, reporting each instance's steps.

    Under torchrun the 64 instances are sharded over the ranks (paper_1702_01335_gb300.shard:
    balanced by updates per step, no collective on the data path): the total work is fixed
    (strong scaling), each rank steps its share, the rate is all instances' updates over the
    slowest rank's time, and the per-instance steps and residuals are gathered on the host."""
    import torch
    from paper_1702_01335_gb300 import LBS_FP32, LBS_FP64, Instance, Solver
    from paper_1702_01335_gb300.autotune import DEFAULT_CACHE, autotune
    from paper_1702_01335_gb300.shard import gather, shard
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def reduce(x, op):
        t = torch.tensor([float(x)], dtype=torch.float64, device="cuda")
        if dist is not None:
            dist.all_reduce(t, op={"max": dist.ReduceOp.MAX, "sum": dist.ReduceOp.SUM}[op])
        return float(t.item())

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    ps_all = W.sweep(64, W.SWEEP_SEED)
    inst_all = [Instance(**p) for p in ps_all]
    idx = shard(inst_all, rank, world)
    ps = [ps_all[i] for i in idx]
    inst = [inst_all[i] for i in idx]
    upd_total = sum(i.Nz * i.Q for i in inst_all)
    prec = LBS_FP32 if a.precision == "f32" else LBS_FP64
    s = Solver(inst, precision=prec)
    if a.tiling:
        s.set_tiling(*(int(x) for x in a.tiling.split(",")))
        tuned = {"source": "--tiling"}
    else:
        tuned = autotune(s, candidates=tuple((V, ZT, F) for V in (1, 2, 4) for ZT in (8, 12, 16)
                                             for F in (0, 2)), steps=3,
                         cache_file=a.tuning_cache or DEFAULT_CACHE)
    st = s.torch_stream()
    upd_step = sum(i.Nz * i.Q for i in inst)
    s.step(a.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        e0.record(st)
        s.step(a.steps)
        e1.record(st)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    nprof = max(3, min(200, a.steps // 10))
    tl = s.tiling()
    if tl["fuse"] == 2:
        s.set_tiling(tl["V"], tl["ZT"], 0)
        s.profile_steps(1)
    k_stage, k_fin, k_step = s.profile_steps(nprof)
    if tl["fuse"] == 2:
        s.set_tiling(tl["V"], tl["ZT"], 2)
    bpu = BYTES_PER_UPDATE[a.precision]
    achieved = upd_step * bpu * nprof / (k_stage * 1e-3) / 1e9
    peak, peak_kind = peaks()
    # end to end through the C ABI with host buffers
    pinned = torch.empty(s.state_bytes(), dtype=torch.uint8, pin_memory=True)
    s.get_state_all_ptr(pinned.data_ptr(), to_host=True)
    nrows = sum(8 * i.Nz for i in inst)
    out_host = torch.empty(nrows, dtype=torch.float64, pin_memory=True)
    e2e_steps = max(3, min(100, a.steps // 30))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.set_state_all_ptr(pinned.data_ptr(), from_host=True)
        s.step(1)
        s.moments_all_ptr(out_host.data_ptr())
    torch.cuda.synchronize()
    e2e_s = reduce(time.perf_counter() - t0, "max")
    s.close()
    # to the steady state from rest, one batch per rank, device-side retirement
    budget = 60000
    s = Solver(inst, precision=prec)
    if "V" in tl:
        s.set_tiling(tl["V"], tl["ZT"], tl["fuse"])
    barrier()
    t0 = time.perf_counter()
    steps = s.run_to_steady(1e-8, max_steps=budget, check_every=500, raise_on_fail=False)
    wall = reduce(time.perf_counter() - t0, "max")
    res = [s.residual(b) for b in range(len(inst))]
    s.close()
    steps = gather([int(x) for x in steps], idx, len(inst_all), dist)
    res = gather(res, idx, len(inst_all), dist)
    conv = [r < 1e-8 for r in res]
    launches = reduce({0: 6, 1: 3, 2: 12}[tl["fuse"]] * a.steps, "sum")
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return
    line = {
        "metric": "cell x velocity updates/s (RK-3 steps)", "value": upd_total * a.steps / (ms * 1e-3),
        "unit": "updates/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": a.precision, "data": "synthetic",
        "config": {"workload": "C4 sweep: 64 instances, seed 1702, Kn 10^U(-2,2), u_w U(0.05,1), Pr 2/3, "
                               "T^omega / Sutherland (0.27, 0.52), Nz 32-512, Qx 4-16, Qy 4, Qz 4-48, "
                               "N_eq 4, uniform cells, own CFL step each",
                   "updates_per_step": upd_total,
                   "parallelism": ("instances sharded over %d ranks by updates per step (rank 0: %d "
                                   "instances)" % (world, len(inst))) if world > 1 else "one batch",
                   "l2": "inputs larger than L2 (d and two increments of %d MiB each)" % (
                       upd_step * (4 if a.precision == "f32" else 8) >> 20),
                   "tiling": {"V": tl["V"], "ZT": tl["ZT"], "fused_finalise": tl["fuse"],
                              "chosen_by": tuned.get("source", "autotune.py")}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_source": peak_kind,
                     "kernel": "stage_kernel", "algorithmic_bytes_per_update_step": bpu,
                     "stage_kernel_ms_per_step": k_stage / nprof, "finalize_ms_per_step": k_fin / nprof},
        "e2e": {"value": upd_total * e2e_steps / e2e_s, "unit": "updates/s",
                "h2d_bytes_per_step": upd_total * (6 if a.precision == "f32" else 8),
                "d2h_bytes_per_step": sum(8 * i.Nz for i in inst_all) * 8},
        "to_steady": {"tol": 1e-8, "step_budget": budget, "wall_s": wall, "converged": int(sum(conv)),
                      "steps": [int(x) for x in steps],
                      "not_converged": [{"inst": b, "Kn": ps_all[b]["Kn"], "Nz": ps_all[b]["Nz"], "R": res[b]}
                                        for b in range(len(inst_all)) if not conv[b]]},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if not a.no_cpu_baseline and world == 1:
        mid = sorted(range(len(ps)), key=lambda b: ps[b]["Nz"] * ps[b]["Qx"] * ps[b]["Qz"])[len(ps) // 2]
        line["cpu_baseline"] = cpu_baseline(ps[mid])
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.workload in ("tables", "luo"):
        return run_small(a)
    if a.workload == "sweep":
        return run_sweep(a)
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1702_01335_gb300 import LBS_FP32, LBS_FP64, Instance, Solver
    from paper_1702_01335_gb300.autotune import DEFAULT_CACHE, autotune
    prec = LBS_FP32 if a.precision == "f32" else LBS_FP64
    if a.workload == "c3x32":
        inst = [Instance(**W.C3)] * (a.batch if a.batch != BATCH else 32)
    else:
        inst = [Instance(**W.C2)] * a.batch
    s = Solver(inst, precision=prec)
    if a.tiling:
        V, ZT, F = (int(x) for x in a.tiling.split(","))
        s.set_tiling(V, ZT, F)
        tuned = {"V": V, "ZT": ZT, "fuse": F, "source": "--tiling"}
    else:
        tuned = autotune(s, candidates=tuple((V, ZT, F) for V in (1, 2, 4) for ZT in (8, 10, 12, 14, 16, 24)
                                             for F in (0, 1, 2)), steps=3,
                         cache_file=a.tuning_cache or DEFAULT_CACHE)
    st = s.torch_stream()
    upd_step = sum(i.Nz * i.Q for i in inst)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident throughput
    s.step(a.warmup)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        e0.record(st)
        s.step(a.steps)
        e1.record(st)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    s_max, value = whole_job(ms * 1e-3, upd_step * a.steps, dist, device="cuda")
    ms_max = s_max * 1e3

    # ---- roofline of the stage kernels (live CUDA events, same stream)
    nprof = max(3, min(200, a.steps // 10))
    if tuned["fuse"] == 2:
        # split stepping overlaps one half's stage kernel with the other's finalisation,
        # so the stage kernel's own launch time is taken with the batch unsplit (same
        # kernel, same V and ZT, events on the solver's stream), after the timed region
        s.set_tiling(tuned["V"], tuned["ZT"], 0)
        s.profile_steps(1)
    k_stage, k_fin, k_step = s.profile_steps(nprof)
    if tuned["fuse"] == 2:
        s.set_tiling(tuned["V"], tuned["ZT"], 2)
    bpu = BYTES_PER_UPDATE[a.precision]
    if a.precision == "f64":
        # the FP64 solver is bound by the FP64 pipe: its rate against the measured FMA rate
        from paper_1702_01335_gb300.lbs import probe_fma_rate
        f64_rate, f32_rate = probe_fma_rate()
        achieved = upd_step * FP64_FLOPS_PER_UPDATE_STEP * nprof / (k_stage * 1e-3) / 1e12
        peak, peak_kind = f64_rate / 1e12, "measured by lbs_probe_fma_rate (FP64 FMA chains, CUDA events)"
    else:
        achieved = upd_step * bpu * nprof / (k_stage * 1e-3) / 1e9
        peak, peak_kind = peaks()
        peak_kind += " (MEASURED_PEAKS.json hbm_gbs)"

    # ---- end to end through the C ABI with host buffers
    pinned = torch.empty(s.state_bytes(), dtype=torch.uint8, pin_memory=True)
    s.get_state_all_ptr(pinned.data_ptr(), to_host=True)
    nprof_rows = sum(8 * i.Nz for i in inst)
    out_host = torch.empty(nprof_rows, dtype=torch.float64, pin_memory=True)
    e2e_steps = max(3, min(100, a.steps // 30))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.set_state_all_ptr(pinned.data_ptr(), from_host=True)
        s.step(1)
        s.moments_all_ptr(out_host.data_ptr())
    barrier()
    e2e_s = time.perf_counter() - t0
    _, e2e_value = whole_job(e2e_s, upd_step * e2e_steps, dist, device="cuda")

    traffic = None
    tpath = os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")
    if os.path.exists(tpath):
        d = json.load(open(tpath))
        from paper_1702_01335_gb300.autotune import kernel_hash
        if d.get("kernel_hash") == kernel_hash() and d.get("precision") == a.precision:
            traffic = d["bytes_per_step_per_update"] * upd_step / 3.0

    if rank == 0:
        wl = ("C3 high Kn: Kn=100 u_w=0.05 T_w=1 Pr=2/3 mu~T^0.5 Nz=256 uniform Q=16x4x(2x64)=8192 N_eq=4"
              if a.workload == "c3x32" else
              "C2 Shakhov Maxwell molecules Kn=1 u_w=0.5 T_w=1 Pr=2/3 Nz=128 A=0.98 Q=8x8x(2x16)=2048 N_eq=4")
        if a.precision == "f64":
            roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None, "peak_source": peak_kind,
                    "fp32_fma_rate_tflops": f32_rate / 1e12,
                    "flops_per_update_step": FP64_FLOPS_PER_UPDATE_STEP,
                    "hbm_gbs_at_64_bytes_per_update": upd_step * bpu * nprof / (k_stage * 1e-3) / 1e9}
        else:
            roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind}
        roof.update({"kernel": "stage_kernel (3 launches per step%s)" % {
                         0: "", 1: ", finalisation folded in",
                         2: "; timed with the batch unsplit, the tuned run steps its halves on "
                            "two streams"}[tuned["fuse"]],
                     "algorithmic_bytes_per_update_step": bpu,
                     "stage_kernel_ms_per_step": k_stage / nprof,
                     "finalize_ms_per_step": k_fin / nprof,
                     "profiled_step_ms": k_step / nprof})
        line = {
            "metric": "cell x velocity updates/s (RK-3 steps)",
            "value": value, "unit": "updates/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": a.precision, "data": "synthetic",
            "config": {"workload": wl,
                       "batch_per_gpu": a.batch, "state_bytes": s.state_bytes(),
                       "l2": "inputs larger than L2 (d and two stage increments of %d MiB each)" % (
                           upd_step * (4 if a.precision == "f32" else 8) >> 20),
                       "parallelism": "replicas, independent batches per GPU",
                       "tiling": {"V": tuned["V"], "ZT": tuned["ZT"], "fused_finalise": tuned["fuse"],
                                  "finalise_layout": {1: "thread per cell", 2: "warp per cell"}.get(
                                      tuned.get("fin"), "default"),
                                  "finalise_layout_ms_per_step": tuned.get("fin_ms_per_step"),
                                  "chosen_by": tuned.get("source", "autotune.py (CUDA-event timing of "
                                                                   "candidates, cached per kernel hash)")}},
            "roofline": roof,
            "e2e": {"value": e2e_value, "unit": "updates/s",
                    "h2d_bytes_per_step": s.state_bytes(), "d2h_bytes_per_step": nprof_rows * 8,
                    "what": "lbs_set_state(all, pinned host) + lbs_step(1) + lbs_moments(all, host) "
                            "per step"},
            "gpu_launches": {0: 6, 1: 3, 2: 12}[tuned["fuse"]] * a.steps,
            "clocks": clk.summary(),
        }
        if not a.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(W.C3 if a.workload == "c3x32" else W.C2)
        if not a.no_steady and world == 1 and a.workload == "c2":
            line["time_to_steady"] = time_to_steady()
        print(json.dumps(line), flush=True)
    s.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
