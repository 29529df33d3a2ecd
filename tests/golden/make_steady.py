"""Writes tests/golden/steady_<workload>.json: profiles of the FP64 oracle marched from
rest to the steady state of the solver's residual criterion (R < tol, the residual of
the oracle's oracle_step), for the FP32-storage precision tests.

Calls only oracle/ (and workloads.py for the parameter set).  Usage:

    python tests/golden/make_steady.py C2 --tol 1e-9 [--threads 6] [--checkpoint PATH]

Every value in the output is the oracle's.  The record holds the step count at which R
first fell below each power of ten from 1e-6 down to tol, with the profiles at each of
those steps, so that a test can march the solver the same number of steps from the same
rest state and compare trajectories (two solves stopped at R < tol each are only
R / (1 - lambda) apart along the slowest mode, far more than the storage precision).
The optional checkpoint (state and step count, numpy .npz) lets a long run resume.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle.oracle import PROFILE_NAMES, Oracle  # noqa: E402


def oracle_for(p):
    return Oracle(p["Qx"], p["Qy"], p["Qz"], p["N_eq"], p["Nz"], A=p["A"], Kn=p["Kn"], uw=p["u_w"],
                  Tw=p["T_w"], Pr=p["Pr"], visc_law=p["visc_law"], visc_param=p["visc_param"],
                  dt=p.get("dt"))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=("C1", "C2", "C3"))
    ap.add_argument("--tol", type=float, default=1e-9)
    ap.add_argument("--chunk", type=int, default=1000)
    ap.add_argument("--max-steps", type=int, default=3_000_000)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--checkpoint", default="")
    ap.add_argument("--write-only", action="store_true",
                    help="write the record of the marks reached so far (from --checkpoint) and stop")
    a = ap.parse_args()
    if a.threads:
        os.environ["OMP_NUM_THREADS"] = str(a.threads)
    p = getattr(W, a.workload)
    o = oracle_for(p)
    marks = [10.0 ** -e for e in range(7, 20) if 10.0 ** -e >= a.tol * 0.999]
    rec = {"workload": a.workload, "params": p, "dt": o.dt, "marks": []}
    if a.checkpoint and os.path.exists(a.checkpoint):
        z = np.load(a.checkpoint, allow_pickle=False)
        o.f[...] = z["f"]
        o.steps = int(z["steps"])
        rec["marks"] = json.loads(str(z["marks"]))
        print("resumed at step %d" % o.steps, flush=True)
    done = {m["tol"] for m in rec["marks"]}
    t0 = time.time()
    while o.steps < a.max_steps and not a.write_only:
        r = o.step(a.chunk, residuals=True)
        for m in marks:
            if m in done:
                continue
            hit = np.nonzero(r < m)[0]
            if hit.size:
                # the profiles at the end of this chunk, with the step count they belong to
                prof = o.profiles()
                rec["marks"].append({"tol": m, "first_step_below": int(o.steps - a.chunk + hit[0] + 1),
                                     "steps": int(o.steps), "residual": float(r[-1]),
                                     "profiles": {k: prof[k].tolist() for k in PROFILE_NAMES}})
                done.add(m)
        print("step %d R %.3e (%.0f s)" % (o.steps, r[-1], time.time() - t0), flush=True)
        if a.checkpoint and (o.steps // a.chunk) % 10 == 0:
            np.savez(a.checkpoint + ".tmp.npz", f=o.f, steps=o.steps, marks=json.dumps(rec["marks"]))
            os.replace(a.checkpoint + ".tmp.npz", a.checkpoint)
        if a.tol in done or min(done, default=1.0) <= a.tol:
            break
    rec["source"] = ("FP64 oracle (oracle/couette.c) from the rest Maxwellian; the marks are the first "
                     "steps with R below each tol, R the solver's residual (max over n, u_x, T of the L2 "
                     "change per step relative to the profile's L2 norm, the velocity's floored at "
                     "|u_w| sqrt(Nz)); written by tests/golden/make_steady.py")
    out = os.path.join(HERE, "steady_%s.json" % a.workload)
    with open(out, "w") as fh:
        json.dump(rec, fh, indent=1)
    print("wrote", out)


if __name__ == "__main__":
    main()
