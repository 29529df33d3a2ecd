"""Tile autotuner for the stage kernel.

The stage kernel's work decomposition (velocities per thread V, cells per
z-tile ZT, finalisation folded into the stage kernel or launched apart) changes
how many CTAs fit on an SM, how much halo is re-read and how the per-cell
moment reduction is amortised; it does not change the arithmetic.
`autotune(solver)` times every candidate with CUDA events on a scratch solver
built from the same instances (so the caller's state and step counters are not
touched), applies the fastest tiling to `solver`, and caches the choice per
batch signature (kernel sources, precision, GPU model, and the size, velocity model
and channel of every instance) in memory and, optionally, in a JSON file.
"""
import hashlib
import itertools
import json
import os

from .lbs import LbsError, Solver

_CSRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_cache.json")

CANDIDATES = tuple((V, ZT, F) for V in (1, 2, 4) for ZT in (4, 6, 8, 12, 16, 24, 32) for F in (0, 1, 2))
_cache = {}


_KERNEL_SOURCES = ("kernels.cuh", "kernels.cu", "lbs_internal.h", "stage_f32_full.cu", "stage_f32_red.cu",
                   "stage_f64_full.cu", "stage_f64_red.cu")


def kernel_hash():
    """Hash of the stage kernel's sources: a cached choice is ignored once they change."""
    h = hashlib.sha256()
    for f in _KERNEL_SOURCES:
        h.update(open(os.path.join(_CSRC, f), "rb").read())
    return h.hexdigest()[:16]


def device_tag():
    """The GPU a timing belongs to: its name and SM count ("cpu" without one)."""
    try:
        import torch
        if torch.cuda.is_available():
            pr = torch.cuda.get_device_properties(torch.cuda.current_device())
            return "%s/%dsm" % (pr.name.replace(" ", "_"), pr.multi_processor_count)
    except Exception:
        pass
    return "cpu"


def signature(solver):
    """Kernel hash, precision, the GPU, and the (Nz, Q) of the batch's instances with
    the velocity model (r: the reduced phi / chi model, which runs other kernels) and
    the channel (h: a half channel), run-length encoded ("256*128x2048")."""
    def tag(i):
        return "%dx%d%s%s" % (i.Nz, i.Q, "r" if i.Qy == 0 else "", "h" if i.half else "")
    runs = [(k, len(list(g))) for k, g in itertools.groupby(tag(i) for i in solver.instances)]
    return "%s:p%d:%s:" % (kernel_hash(), solver.precision, device_tag()) + ",".join(
        ("%d*%s" % (n, k)) if n > 1 else k for k, n in runs)


def _load(path):
    if path and os.path.exists(path):
        try:
            return json.load(open(path))
        except (OSError, ValueError):
            return {}
    return {}


def autotune(solver, candidates=CANDIDATES, steps=3, cache_file=None, verbose=False):
    """Pick the fastest (V, ZT, fuse) for solver's batch, then the faster finalisation
    layout for it; returns {"V", "ZT", "fuse", "fin", "ms_per_step", "table", ...}."""
    key = signature(solver)
    disk = _load(cache_file)
    hit = _cache.get(key) or disk.get(key)
    if hit:
        solver.set_tiling(hit["V"], hit["ZT"], hit["fuse"])
        if "fin" in hit:
            solver.set_finalize(hit["fin"])
        return hit
    scratch = Solver(solver.instances, precision=solver.precision)
    table = []
    try:
        for V, ZT, F in candidates:
            try:
                scratch.set_tiling(V, ZT, F)
            except LbsError:
                continue
            scratch.profile_steps(1)
            stage_ms, fin_ms, step_ms = scratch.profile_steps(steps)
            table.append({"V": V, "ZT": ZT, "fuse": F, "ms_per_step": step_ms / steps,
                          "stage_ms_per_step": stage_ms / steps, "ctas": scratch.tiling()["ctas"]})
            if verbose:
                print(table[-1], flush=True)
    finally:
        scratch.close()
    if not table:
        raise ValueError("no valid tiling among the candidates")
    best = min(table, key=lambda r: r["ms_per_step"])
    # then the finalisation layout (one thread or one warp per cell) for that tiling
    fin_times = {}
    scratch = Solver(solver.instances, precision=solver.precision)
    try:
        scratch.set_tiling(best["V"], best["ZT"], best["fuse"])
        for mode in (1, 2):
            scratch.set_finalize(mode)
            scratch.profile_steps(1)
            fin_times[mode] = scratch.profile_steps(steps)[2] / steps
    finally:
        scratch.close()
    fin = min(fin_times, key=fin_times.get)
    res = {"V": best["V"], "ZT": best["ZT"], "fuse": best["fuse"], "fin": fin,
           "ms_per_step": fin_times[fin], "fin_ms_per_step": fin_times, "table": table}
    solver.set_tiling(best["V"], best["ZT"], best["fuse"])
    solver.set_finalize(fin)
    _cache[key] = res
    if cache_file:
        # entries of other kernel versions can never hit again
        cur = kernel_hash() + ":"
        disk = {k: v for k, v in disk.items() if k.startswith(cur)}
        disk[key] = res
        # one temporary file per process: ranks tuning at once each replace the cache
        # atomically (the last one's entries win)
        tmp = "%s.%d.tmp" % (cache_file, os.getpid())
        with open(tmp, "w") as f:
            json.dump(disk, f)
        os.replace(tmp, cache_file)
    return res
