"""Seeded synthetic workloads (parameter sets only; no arithmetic of the method).

Shared by the tests, the smoke check and the benchmark.  Each workload is a
plain dict of instance parameters with the field names of
`paper_1702_01335_gb300.Instance`; the oracle takes the same values.

  C1  plain BGK-limit Couette (Shakhov with Pr = 1): 4 x 4 x (2 x 4) velocities,
      N_eq = 3, Nz = 32 uniform, Kn = 0.1, u_w = 0.1
  C2  Maxwell molecules (Pr = 2/3, mu ~ T): 8 x 8 x (2 x 16) = 2048 velocities,
      N_eq = 4, Nz = 128 stretched toward the walls (A = 0.98), Kn = 1, u_w = 0.5
  C3  high Kn: 16 x 4 x (2 x 64) = 8192 velocities, N_eq = 4, Nz = 256 uniform,
      Kn = 100, u_w = 0.05, Pr = 2/3, mu ~ T^0.5
  paper_tables()  the He / Ar runs of Sec. VI (Tables gradu, shear, temp) on the half
      channel: 16 cells stretched with A = 0.98, 7 x 7 x (2 x Q_n) velocities with
      N_eq = 6, Sutherland viscosity, Pr = 2/3, delta = 1/(Kn sqrt 2) in
      {0.1, 1, 10, 20, 40}, u_w in {sqrt 2, 0.1 sqrt 2}; Q_n and dt from Table sharipov
  paper_tables_small_delta()  the same at delta = 0.01 with Q_n = 100, at dt = 1e-4
  luo_runs()  the low-Mach runs of Sec. IV (Table luo): phi / chi model, Qx = 2,
      BGK, tau = k / sqrt 2, u_w = 1e-5, half channel with S = 64 or 32, A = 0.98
  sweep(n, seed)  instances drawn like the batched Kn / wall-speed / gas-law sweep:
      Kn log-uniform in [0.01, 100], u_w uniform in [0.05, 1], T_w = 1, Pr = 2/3,
      first half mu ~ T^omega (omega uniform in [0.5, 1]), second half Sutherland
      with S alternating 0.27 / 0.52; Nz, Qx, Qz drawn from the listed sets, Qy = 4,
      N_eq = 4, uniform grid (numpy PCG64 streams)
"""
import numpy as np

C1 = dict(Qx=4, Qy=4, Qz=4, N_eq=3, Nz=32, A=0.0, Kn=0.1, u_w=0.1, T_w=1.0, Pr=1.0,
          visc_law=0, visc_param=1.0)
C2 = dict(Qx=8, Qy=8, Qz=16, N_eq=4, Nz=128, A=0.98, Kn=1.0, u_w=0.5, T_w=1.0, Pr=2.0 / 3.0,
          visc_law=0, visc_param=1.0)
C3 = dict(Qx=16, Qy=4, Qz=64, N_eq=4, Nz=256, A=0.0, Kn=100.0, u_w=0.05, T_w=1.0, Pr=2.0 / 3.0,
          visc_law=0, visc_param=0.5)

# Sec. VI: Sutherland constants of the two gases, the rarefaction parameters and the
# per-delta normal-axis order and time step of Table sharipov.  delta = 0.01 is not in
# paper_tables(): at its Q_n = 100 the largest |p_z| is 22.2, and the printed dt = 2.5e-4
# puts the CFL number of the first stretched cell at 1.65, above the RK-3 / WENO-5
# limit; paper_tables_small_delta() runs it at the stable dt = 1e-4 (CFL 0.66).
SUTHERLAND_S = {"Ar": 0.5239, "He": 0.3101}
TABLE_DELTAS = (0.1, 1.0, 10.0, 20.0, 40.0)
TABLE_RUN = {0.01: (100, 2.5e-4), 0.1: (30, 2.5e-4)}   # delta -> (Q_n, dt); else (7, 5e-4)
SMALL_DELTA_DT = 1e-4


def paper_tables(reduced=False):
    """The 20 half-channel runs of the Sec. VI tables as (label, instance parameters)
    pairs, gas-major, then delta, then u_w = sqrt 2 before 0.1 sqrt 2; the label holds
    gas, delta and u_w.  reduced=True: the paper's phi / chi model (Qy = 0) instead of
    the 3D set with Q_y = 7."""
    out = []
    for gas in ("Ar", "He"):
        for d in TABLE_DELTAS:
            Qn, dt = TABLE_RUN.get(d, (7, 5e-4))
            for uw in (2.0 ** 0.5, 0.1 * 2.0 ** 0.5):
                out.append((dict(gas=gas, delta=d, uw=uw),
                            dict(Qx=7, Qy=0 if reduced else 7, Qz=Qn, N_eq=6, Nz=16, A=0.98, half=1, Kn=1.0 / (d * 2.0 ** 0.5),
                                 u_w=uw, T_w=1.0, Pr=2.0 / 3.0, visc_law=1, visc_param=SUTHERLAND_S[gas],
                                 dt=dt)))
    return out


def paper_tables_small_delta(reduced=False):
    """The 4 delta = 0.01 runs of the Sec. VI tables (both gases, u_w = sqrt 2 and
    0.1 sqrt 2) with Table sharipov's Q_n = 100 and every other parameter as in
    paper_tables(), at dt = SMALL_DELTA_DT instead of the printed, unstable 2.5e-4."""
    out = []
    for gas in ("Ar", "He"):
        for uw in (2.0 ** 0.5, 0.1 * 2.0 ** 0.5):
            out.append((dict(gas=gas, delta=0.01, uw=uw),
                        dict(Qx=7, Qy=0 if reduced else 7, Qz=TABLE_RUN[0.01][0], N_eq=6, Nz=16, A=0.98, half=1,
                             Kn=1.0 / (0.01 * 2.0 ** 0.5), u_w=uw, T_w=1.0, Pr=2.0 / 3.0, visc_law=1,
                             visc_param=SUTHERLAND_S[gas], dt=SMALL_DELTA_DT)))
    return out


# Sec. IV (Table luo): the low-Mach runs.  k -> (N, Q_n, S)
LUO_RUNS = {0.03: (3, 4, 64), 0.1: (6, 7, 32), 1.0: (6, 21, 32), 10.0: (6, 80, 32)}


def luo_runs(u_w=1e-5):
    """The low-Mach half-channel runs of Sec. IV as (label, instance parameters): the
    phi / chi model with the HLB(1;2) rule along the flow (Qx = 2), the half-range
    order and grid of Table luo (A = 0.98), BGK (Pr = 1), tau = k / sqrt 2 (the power
    law with omega = 1 gives Kn / n, and n = 1 to O(u_w^2)), u_w = 1e-5, T_w = 1."""
    out = []
    for k, (N, Qn, S) in LUO_RUNS.items():
        out.append((dict(k=k), dict(Qx=2, Qy=0, Qz=Qn, N_eq=N, Nz=S, A=0.98, half=1, Kn=k / 2.0 ** 0.5,
                                    u_w=u_w, T_w=1.0, Pr=1.0, visc_law=0, visc_param=1.0)))
    return out


SWEEP_SEED, TRAIN_SEED, HELDOUT_SEED = 1702, 1703, 1704
NZ_SET = (32, 48, 64, 96, 128, 192, 256, 384, 512)
QX_SET = (4, 6, 8, 12, 16)
QZ_SET = (4, 8, 12, 16, 24, 32, 48)


def sweep(n=64, seed=SWEEP_SEED, nz_set=NZ_SET, qx_set=QX_SET, qz_set=QZ_SET):
    """n instances of the batched sweep, drawn from numpy PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for b in range(n):
        Kn = float(10.0 ** rng.uniform(-2.0, 2.0))
        u_w = float(rng.uniform(0.05, 1.0))
        if b < n // 2:
            law, param = 0, float(rng.uniform(0.5, 1.0))
        else:
            law, param = 1, (0.27 if (b - n // 2) % 2 == 0 else 0.52)
        out.append(dict(Qx=int(rng.choice(qx_set)), Qy=4, Qz=int(rng.choice(qz_set)), N_eq=4,
                        Nz=int(rng.choice(nz_set)), A=0.0, Kn=Kn, u_w=u_w, T_w=1.0, Pr=2.0 / 3.0,
                        visc_law=law, visc_param=param))
    return out


def warm_start_draws(n, seed):
    """Draws for training and evaluating the warm-start network: the sweep's
    distribution restricted to sizes whose steady solves a batch reaches in seconds
    (Nz in {32, 48, 64}, Qx in {4, 6, 8}, Qz in {4, 8}) and Kn clipped to [0.05, 20]."""
    ps = sweep(n, seed=seed, nz_set=(32, 48, 64), qx_set=(4, 6, 8), qz_set=(4, 8))
    for p in ps:
        p["Kn"] = float(min(max(p["Kn"], 0.05), 20.0))
    return ps


def random_state(shape, seed, amplitude=0.05):
    """Seeded multiplicative perturbation factors 1 + a N(0,1) (for parity inputs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return 1.0 + amplitude * rng.standard_normal(shape)
