/*
 * lbs.h - C ABI of the GB300 solver for the mixed-quadrature Shakhov lattice
 * Boltzmann model of Couette flow (Ambrus & Sofonea, "Half-range lattice
 * Boltzmann models for the simulation of Couette flow using the Shakhov
 * collision term", arXiv:1702.01335).
 *
 * Geometry and axes.  Two parallel plates at z = -L/2 and z = +L/2 (L = 1)
 * move along x with -u_w and +u_w and are held at T_w (Sec. III; the paper
 * calls the wall-normal axis x and the flow axis y).  The velocity set is the
 * direct product of full-range Gauss-Hermite rules with Qx nodes on x and Qy
 * nodes on y, and a half-range Gauss-Hermite rule with Qz_half nodes on each
 * semi-axis of z: Q = 2 * Qx * Qy * Qz_half velocities (Sec. III).
 *
 * Reduced model (Qy = 0).  The paper's own model (Sec. III, Eqs. reduced_def,
 * boltz_red, phieq, sred_def) integrates the transverse momentum out: two
 * distributions phi = int f dp_y and chi = int p_y^2 f dp_y on the (p_x, p_z)
 * nodes relax to phi_eq (1 + S_phi) and chi_eq (1 + S_chi), chi_eq = T phi_eq.
 * They are stored as a velocity set with Qy = 2 (j = 0: phi, j = 1: chi), so
 * Q = 4 * Qx * Qz_half and every layout below applies with Qy = 2.  The
 * transverse velocity and heat flux vanish in Couette flow and are not carried;
 * the profiles report u_y = q_y = P_xy = P_yz = 0 and P_yy = sum chi.  A batch
 * is either all reduced or all full.
 *
 * Scheme (one time step = lbs_step(h, 1)): the RK-3 TVD stages of Eq. (rk3)
 * applied to L[F] of Eq. (L_def): WENO-5 advection along z (Eqs. flux,
 * weno5_flux, weno5_omega, weno_sigma, Table weno), relaxation to the
 * truncated-Hermite Shakhov target n G_x G_y G_z (1 + S) (Eqs. boltz, sdef,
 * fyz, Fmn_def), diffuse reflection at both walls with three ghost nodes,
 * quadratic extrapolation and the wall density n_w (Appendix, "Boundary
 * conditions"), re-imposed at every RK stage.
 *
 * Conventions.
 *  - Every function returns an lbs_status; nothing aborts.  On failure
 *    lbs_last_error() returns a message (thread-local storage).
 *  - The library owns all device memory of a handle.  Output buffers passed
 *    in are owned by the caller.
 *  - Work is queued on the CUDA stream given at creation; when NULL is given
 *    the library creates (and later destroys) a non-blocking stream of its
 *    own, see lbs_get_stream.  Functions that return host data synchronise it.
 *  - Profiles are FP64, laid out [profile][cell] with cells ordered from the
 *    bottom wall (z = -L/2) to the top wall.
 *  - A handle holds a batch of independent instances (one Couette problem
 *    each, possibly of different sizes); they advance together and are
 *    addressed by index 0 .. n-1.
 */
#ifndef LBS_H
#define LBS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbs_solver* lbs_handle;

typedef enum {
    LBS_OK = 0,
    LBS_ERR_ARG = 1,              /* invalid argument or size                  */
    LBS_ERR_CUDA = 2,             /* a CUDA runtime call failed                */
    LBS_ERR_NONFINITE = 3,        /* NaN/Inf or n <= 0 / T <= 0 in a state      */
    LBS_ERR_NO_CONVERGENCE = 4,   /* residual target not met within max_steps  */
    LBS_ERR_QUADRATURE = 5,       /* quadrature construction failed            */
    LBS_ERR_TIMEOUT = 6           /* a kernel's bounded wait for its bulk
                                     copies ran out (see lbs_set_wait_limit)   */
} lbs_status;

typedef enum { LBS_VISC_POWER = 0, LBS_VISC_SUTHERLAND = 1 } lbs_visc_law;

/* Storage/arithmetic precision of the distribution.  The state is stored as the
 * deviation d_k = f_k / w_k - 1 of the normalised populations from the rest
 * Maxwellian (n = 1, u = 0, T = 1: f_k = w_k), so that the stored digits resolve the
 * departure from rest rather than the rest state itself.  FP32 stores and relaxes
 * d in FP32 and keeps the rounding residual of each stored value as a 16-bit
 * fixed-point fraction of its last place: a step's increment, far below an FP32
 * ulp near a steady state, then accumulates instead of being rounded away
 * (without it the state stalls about eps_32 / (lambda dt) short of the steady
 * state, lambda the decay rate of the slowest mode).  The RK stages hold their
 * increments over the step's start state, not stage values, for the same reason.
 * Moment sums: with FP32 storage, in FP32 within a CTA's velocity chunk and in
 * double-float (an FP32 pair, about 48 significant bits) across chunks; with FP64
 * storage, in FP64.  The cell state, the wall flux balance, the profiles and the
 * residual are FP64 in both modes. */
typedef enum { LBS_FP64 = 0, LBS_FP32_STORE_FP64_ACC = 1 } lbs_precision;

/* Velocity-set orders.  N_eq is the order of the truncated Hermite expansion
 * of the equilibrium; each axis uses min(N_eq, Q_a - 1) (Sec. III; Q_a = Qz_half
 * on the wall-normal axis).  Limits: 1 <= Qx <= 100, Qy = 0 (the reduced phi /
 * chi model above) or 1 <= Qy <= 100, 1 <= Qz_half <= 100, 0 <= N_eq <= 8,
 * Q <= 32768. */
typedef struct { int Qx, Qy, Qz_half, N_eq; } lbs_orders;

/* Grid: Nz cells (6 <= Nz <= 4096).  A = 0: uniform cells.  0 < A < 1: the
 * tanh stretching of Eqs. (stretch), (etas) mirrored onto the full channel,
 * eta_s = -atanh(A) + (s - 1/2) d_eta, d_eta = 2 atanh(A)/Nz, x = L tanh(eta)/(2A).
 *
 * half = 0: the full channel -L/2 <= z <= L/2 between two diffuse walls.
 * half = 1: only the upper half 0 <= z <= L/2 of a channel of 2 Nz cells (the
 * same cells as cells Nz .. 2Nz-1 of the full grid with 2 Nz cells, so that the
 * stretched grid follows Eq. (etas) on the half channel, eta_s = (s - 1/2)
 * atanh(A)/Nz), with the bounce-back condition of the Appendix ("Boundary
 * conditions") on the centre line z = 0: the three ghost cells below it hold the
 * populations of cells 0, 1, 2 at the velocity with p_z and p_x reversed (the
 * point symmetry of Couette flow about the centre line; p_y, which the paper's
 * reduced model integrates out, is kept).  The diffuse wall stays at z = L/2. */
typedef struct { int Nz; double A; int half; } lbs_grid;

/* Viscosity law.  POWER: mu ~ T^omega_or_S, tau = Kn T^(omega-1) / n
 * (Eq. mw_tau for omega = 1).  SUTHERLAND: Eq. (sutherland_tau) with
 * delta = 1/(Kn sqrt 2): tau = Kn sqrt(T) (1 + S) / (n (T + S)), S = omega_or_S. */
typedef struct { lbs_visc_law law; double omega_or_S; } lbs_visc;

/* One Couette instance.  dt > 0 is used as given; dt <= 0 selects
 * dt = cfl * min(dz) / max|p_z|, capped at tau(n = 2, T = T_w) / 2. */
typedef struct {
    lbs_orders orders;
    lbs_grid grid;
    double Kn, u_w, T_w, Pr;
    lbs_visc visc;
    double dt, cfl;
} lbs_instance_desc;

/* Create a single-instance solver (Sec. III model, Appendix scheme) with the
 * CFL time step.  The state starts at the rest Maxwellian n = 1, T = 1 (the
 * weights w_k).  cuda_stream is a cudaStream_t or NULL.  Errors: LBS_ERR_ARG on
 * out-of-range orders/sizes, Kn <= 0, T_w <= 0, Pr <= 0 or cfl <= 0;
 * LBS_ERR_CUDA when device memory cannot be allocated. */
lbs_status lbs_create(lbs_handle* out, lbs_orders ord, lbs_grid grid, double Kn, double u_w,
                      double T_w, double Pr, lbs_visc visc, lbs_precision prec, double cfl,
                      void* cuda_stream);

/* Create a batch of n >= 1 independent instances that advance together in
 * the same launches (shared precision and stream).  desc[n] is read only
 * during the call.  LBS_ERR_ARG, in addition to lbs_create's cases, for a batch
 * that mixes reduced (Qy = 0) and full instances. */
lbs_status lbs_batch_create(lbs_handle* out, const lbs_instance_desc* desc, int n,
                            lbs_precision prec, void* cuda_stream);

/* Release every resource of the handle (synchronises its stream). */
lbs_status lbs_destroy(lbs_handle h);

/* Queue nsteps >= 0 full RK-3 steps (Eq. rk3) of every active instance on the
 * stream; returns without waiting.  The residual of each step is kept. */
lbs_status lbs_step(lbs_handle h, long nsteps);

/* March until every instance has residual R < tol or has taken max_steps steps.
 * Each instance stops (retires) in the step where its R first drops below tol;
 * steps_out[n] (may be NULL) receives the steps each instance took.  R is
 * checked on the device every step; the host polls every check_every steps
 * (CUDA-graph launches of check_every steps).  Returns LBS_ERR_NO_CONVERGENCE
 * if some instance did not converge. */
lbs_status lbs_run_to_steady(lbs_handle h, double tol, long max_steps, int check_every,
                             long* steps_out);

/* Profiles of instance inst, host_out[8][Nz]: n, u_x, T, q_x, q_z, P_xx,
 * P_xz, P_zz (Eq. qdef, pressure tensor P_ij = sum xi_i xi_j f with xi = p - u).
 * inst = -1: every instance, concatenated in instance order ([8][Nz_b] each):
 * gathered on the device, then one copy to host_out.  Synchronises the stream. */
lbs_status lbs_moments(lbs_handle h, int inst, double* host_out);

/* All 14 profiles of instance inst, host_out[14][Nz]: n, u_x, u_y, u_z, T,
 * q_x, q_y, q_z, P_xx, P_yy, P_zz, P_xy, P_xz, P_yz. */
lbs_status lbs_profiles(lbs_handle h, int inst, double* host_out);

/* Residual of the last step of instance inst:
 * R = max over W in {n, u_x, T} of ||W_new - W_old||_2 / max(||W_old||_2, s_W)
 * over the interior cells (the paper states no criterion; this is the solver's),
 * s_n = s_T = 1e-30 and s_u = max(|u_w| sqrt(Nz), 1e-30): the velocity is measured on
 * the wall speed where the profile is smaller (it vanishes in the free-molecular limit
 * and at u_w = 0).  With FP32 storage the moment sums carry FP32 rounding: R levels
 * off near 1e-8 (a few 1e-8 for strongly rarefied flows), so FP32 targets should be
 * about 1e-7; FP64 reaches 1e-15. */
lbs_status lbs_residual(lbs_handle h, int inst, double* out);

/* Number of steps instance inst has taken. */
lbs_status lbs_steps_taken(lbs_handle h, int inst, long* out);

/* Sizes of instance inst: out[0..3] = Q, Nz, Qx*Qy, element size in bytes of
 * the stored distribution; dt_out (may be NULL) receives the time step. */
lbs_status lbs_info(lbs_handle h, int inst, long* out, double* dt_out);

/* Checkpoint: copy the distribution of instance inst to dst (host if to_host,
 * else device) exactly as stored: first d[Nz][Q], the deviations
 * d_k = f_k / w_k - 1 in the stored precision (8-byte doubles or 4-byte floats),
 * velocity order k = ((sg * Qz_half + m) * Qx + i) * Qy + j (sg = 0: p_z > 0);
 * then, with FP32 storage only, r[Nz][Q], the 16-bit residuals (int16: the value
 * is d_k + r_k * 2^-15 ulp(d_k); zero is always valid).  So an instance takes
 * Nz Q 8 bytes (FP64) or Nz Q 6 bytes (FP32).  inst = -1: every instance's d,
 * concatenated in instance order, then every instance's r, concatenated.
 * Synchronises the stream. */
lbs_status lbs_get_state(lbs_handle h, int inst, void* dst, int to_host);

/* Resume / warm start: set the distribution of instance inst from src (layout
 * and precision of lbs_get_state; host if from_host, else device) and
 * recompute its moments and wall densities.  inst = -1: every instance from
 * one buffer laid out as lbs_get_state's.  From host memory, a state of 48 MB or more
 * is copied in two to four groups of instances (at least 24 MB each), and each group's
 * moments are computed on a second stream while the next group is copied.  LBS_ERR_NONFINITE if the state has non-finite values or
 * n <= 0 or T <= 0 in a cell.  Synchronises the stream. */
lbs_status lbs_set_state(lbs_handle h, int inst, const void* src, int from_host);

/* Tests of failure detection: the number of spins a stage CTA waits for its bulk
 * copies (cp.async.bulk into shared memory, one mbarrier) before it gives up,
 * flags the instance and leaves; default 2^26 (seconds).  When a wait runs out the
 * CTA waits up to a further 2^28 spins for its copies in flight to land, so that none
 * writes shared memory after it has left, then returns without output; the next
 * call that checks the status returns LBS_ERR_TIMEOUT.  spins = 0 gives up at once
 * (the copies still land).  If the second wait also runs out (a copy that has not
 * landed after some seconds), the CTA leaves anyway, and a late copy may still write
 * the shared memory of a later CTA on that SM: after LBS_ERR_TIMEOUT, restore the
 * state (lbs_clear_status, lbs_set_state) before stepping again, and treat a repeated
 * timeout as a device fault.  Applies to every instance; synchronises the stream. */
lbs_status lbs_set_wait_limit(lbs_handle h, unsigned spins);

/* Clear the status words of every instance (after LBS_ERR_TIMEOUT or
 * LBS_ERR_NONFINITE); the state is left as it is, so a caller resumes with
 * lbs_set_state.  Synchronises the stream. */
lbs_status lbs_clear_status(lbs_handle h);

/* Warm start: seed instance inst with the discrete Shakhov target of the given
 * profiles in every cell.  prof[8][Nz] has the layout of lbs_moments (the P_ij
 * rows are not used: the seed is n G_x G_y G_z (1 + S) of n, u_x, T, q_x, q_z).
 * LBS_ERR_NONFINITE if a value is not finite or n <= 0 or T <= 0. */
lbs_status lbs_init_from_profiles(lbs_handle h, int inst, const double* prof);

/* Start for strongly rarefied instances: seed every cell of instance inst with the
 * free-molecular state of the channel, each velocity carrying the discrete equilibrium
 * of the wall it left (the incoming-ghost formula of the Appendix with n_w = 1: p_z > 0
 * the bottom wall at -u_w, p_z < 0 the top wall at +u_w), each cell rescaled to unit
 * density (the rest start's mass); FP32 residuals zero.  Not a step of the paper's
 * method: a choice of initial state.  Queued on the handle's stream; the analysis pass
 * that follows synchronises it.  LBS_ERR_ARG for an invalid handle or instance. */
lbs_status lbs_init_free_molecular(lbs_handle h, int inst);

/* Profiles of a distribution the caller holds in device memory, computed
 * without allocating device memory.  The paper has no counterpart: this is a
 * service for callers that cannot call cudaMalloc where they need moments, for
 * example code running under another framework's device-memory budget, or a
 * latency-critical loop where the device-wide synchronisation of cudaMalloc
 * and cudaFree is not acceptable.
 *   f_dev     device pointer, [Nz][Q] deviations d_k = f_k / w_k - 1 of instance
 *             inst's velocity set in the handle's precision (the d part of an
 *             lbs_get_state buffer; the FP32 residuals are not needed); read only.
 *   prof_dev  device pointer, [14][Nz] FP64 output in the layout of
 *             lbs_profiles.  A cell whose density sums to zero gets NaN
 *             profiles; the call reports no status for it.
 * The work is queued on the handle's stream; the call does not wait for it.
 * Its only scratch is a fixed 2 MiB array in the library's device image (every
 * GPU that loads the library holds it until the process exits), so the
 * instance must satisfy ceil(Q / 512) * Nz <= 20164, else LBS_ERR_ARG.  The
 * first call on a device looks the array's address up (cudaGetSymbolAddress);
 * make that first call before any stream capture.  All calls share the array:
 * calls whose GPU work overlaps (other streams, other threads on the same
 * device) race and must be serialised by the caller.  The array's address is
 * cached per device for the life of the process; like every handle, it is not
 * valid across cudaDeviceReset.  The call allocates nothing and frees nothing. */
lbs_status lbs_moments_static(lbs_handle h, int inst, const void* f_dev, double* prof_dev);

/* Run nsteps steps launching every kernel directly with CUDA events around
 * each on the handle's stream, and return summed device times in ms:
 * out_ms[0] the stage kernels (WENO advection, collision, RK combine, moments,
 * walls, and the finalisation they fold in), out_ms[1] the separate finalisation
 * launches (0 when fused), out_ms[2] the whole steps.
 * Synchronises.  For measurement only; the arithmetic is that of lbs_step. */
lbs_status lbs_profile_steps(lbs_handle h, long nsteps, double* out_ms);

/* Work decomposition of the stage kernel: each CTA of 128 threads updates 128*V
 * velocities (V in {1, 2, 4}) of about ZT consecutive cells (3 <= ZT <= 64).  No
 * effect on the arithmetic in FP64.  In FP32 the full model with V = 2 or 4 gives each
 * thread adjacent velocity pairs, moved as 64-bit words and updated by packed
 * two-lane FP32 instructions: the same operations up to the compiler's contraction
 * choices (results agree to FP32 rounding); this layout needs Q / 2 even in every
 * instance (LBS_ERR_ARG otherwise).  fuse = 1 folds the per-cell and
 * per-instance finalisation into the stage kernel (the last CTA of a z-tile /
 * of an instance does it: 3 launches per step); fuse = 0 runs it as one
 * further launch per stage; fuse = 2 does the
 * same for each half of the batch (about half the tiles each) on two streams,
 * so that one half's FP64 finalisation overlaps the other half's stage kernel
 * (the step forks from and joins back into the handle's stream; a batch of one
 * instance steps as with fuse = 0).  Used by the tile autotuner.  Without a call
 * a solver starts with V = 1, ZT = 4 below 2^22 cell x velocity updates per step
 * and V = 4, ZT = 12 above (V = 1 where the FP32 pair layout does not apply), fuse = 0.  Waits for the handle's stream and
 * recomputes the moment partials of the current state.  LBS_ERR_ARG outside the
 * ranges. */
lbs_status lbs_set_tiling(lbs_handle h, int V, int ZT, int fuse);

/* Current tiling: V, ZT, fuse, number of stage CTAs, dynamic shared memory per
 * CTA.  Any output pointer may be NULL. */
lbs_status lbs_get_tiling(lbs_handle h, int* V, int* ZT, int* fuse, int* ntiles, long* smem_bytes);

/* Finalisation layout (not in the paper: how the per-cell FP64 work of each stage
 * -- moments, profiles, equilibrium coefficients -- is spread over threads).
 * mode 1: one thread per cell; mode 2: one warp per cell (lanes share the moment
 * sums, the x / y coefficient recurrences and the two half-range tables); mode 0
 * (the default): mode 2 for batches of at most 608 cells, else mode 1.  Results
 * agree to rounding (a few ulps of FP64).  *warp_out (may be NULL) receives 1 if
 * the warp layout is in use.  Synchronises the solver's stream. */
lbs_status lbs_set_finalize(lbs_handle h, int mode, int* warp_out);

/* The CUDA stream (cudaStream_t) the handle queues its work on: the one given at
 * creation, or the stream the library created when NULL was given. */
lbs_status lbs_get_stream(lbs_handle h, void** out);

/* Host-only: the solver's Q-point Gauss rule for omega(p) = exp(-p^2/2)/sqrt(2 pi),
 * kind 0 = full range (sum w = 1), kind 1 = half range on (0, inf) (sum w = 1/2).
 * Needs no GPU.  LBS_ERR_ARG for Q outside 1..100. */
lbs_status lbs_quadrature(int kind, int Q, double* nodes, double* weights);

/* Couette-flow diagnostics over the half channel 0 <= z <= L/2 (L = 1), in the
 * build's axes: the paper's normal axis x is z here, its flow axis y is x, so
 * the paper's u_y is u_x and its T_xy is P_xz.  S cells with centres z_1..z_S
 * (0 < z_s < 1/2) enter each formula: the upper half (cells Nz/2 .. Nz-1) of a
 * full channel, or all Nz cells of a half channel. */
typedef struct {
    double u_wall;      /* u_x(L/2), quadratic extrapolation from the three cells
                           next to the wall, Eq. (uslip_extra) */
    double u_slip;      /* u_w - u_x(L/2), Eq. (uslip) */
    double dudz0;       /* u_x'(0) by the three-point formula Eq. (ud0_extra) for
                           a profile odd about the centre line */
    double nu;          /* L u_x'(0) / (2 u_w), Eq. (vgrad) */
    double mflow;       /* half-channel mass flow, rectangle rule in eta of Eq. (mflow),
                           rho = n (particle mass 1) */
    double mflow_hydro; /* rho u_w L / 4 of Eq. (mflow_hydro) with rho = 1 (the
                           channel-average density, conserved from the initial state) */
    double Txy;         /* P_xz averaged over the half channel, Eq. (Txy) */
    double Txy_bal;     /* ballistic limit -rho u_w sqrt(2 T_w / pi), Eq. (Txy_bal), rho = 1 */
    double Pi;          /* -T_xy / (u_w sqrt 2), Eq. (stress) (n_avg = 1, T_w = 1 units) */
    double T0;          /* temperature on the centre line, Eq. (T0), for an even profile */
} lbs_diag;

/* Host-only: diagnostics from profiles prof[14][Nz] in the layout of
 * lbs_profiles (read only), for the grid (Nz, A, half) of lbs_grid.  A = 0 takes
 * the limit A -> 0 of the rectangle rule (equal weights 1/S).  nu, Pi are
 * infinite or NaN when u_w = 0.  Needs no GPU.  LBS_ERR_ARG for null pointers,
 * A outside [0, 1), half not 0 or 1, a full channel with odd Nz or fewer than 6
 * cells in the half channel. */
lbs_status lbs_couette_diagnostics(const double* prof, int Nz, double A, int half, double u_w,
                                   double T_w, lbs_diag* out);

/* The diagnostics of instance inst of a solver (its profiles, grid and walls);
 * synchronises the solver's stream. */
lbs_status lbs_diagnostics(lbs_handle h, int inst, lbs_diag* out);

/* Host-only: the nonlinear part of the velocity profile, Eq. (uy_nl):
 * u_nl(z_s) = 2 z_s / L - u_x(z_s) / u_x(L/2) at the S cells of the half channel
 * (L = 1, u_x(L/2) by Eq. uslip_extra), from profiles prof[14][Nz] as for
 * lbs_couette_diagnostics.  unl_out[S] receives u_nl, z_out[S] (may be NULL)
 * the cell centres z_s.  S = Nz (half = 1) or Nz / 2.  Needs no GPU.
 * LBS_ERR_ARG as lbs_couette_diagnostics. */
lbs_status lbs_couette_nonlinear_velocity(const double* prof, int Nz, double A, int half, double* z_out,
                                          double* unl_out);

/* ---- Warm-start network (not in the paper: the learned initial state of the
 * batched sweep).  A perceptron n_in -> n_hidden -> n_hidden -> n_out with GELU
 * activations, gelu(z) = z (1 + erf(z / sqrt 2)) / 2, maps the parameters of a
 * Couette problem to its steady profiles; its output seeds a solve through
 * lbs_init_from_profiles.  Products run on tensor cores in BF16 with FP32
 * accumulation; every product operand is rounded to BF16 (nearest even);
 * biases, GELU, the loss and Adam are FP32 with FP32 master weights.
 * Parameters are packed FP32 in the order W1 [n_hidden][n_in], b1, W2
 * [n_hidden][n_hidden], b2, W3 [n_out][n_hidden], b3.  Batches are row-major
 * [B][n_in] / [B][n_out] FP32 arrays in device memory owned by the caller. */
typedef struct lbs_mlp* lbs_mlp_handle;

/* Allocate the network's parameters, Adam state and activations for batches
 * up to max_batch (all zero: call lbs_mlp_set_params).  stream as in
 * lbs_create.  LBS_ERR_ARG for sizes outside 1..4096 or max_batch outside
 * 1..2^20; LBS_ERR_CUDA if the allocation fails. */
lbs_status lbs_mlp_create(lbs_mlp_handle* out, int n_in, int n_hidden, int n_out, int max_batch, void* stream);
lbs_status lbs_mlp_destroy(lbs_mlp_handle h);
/* Number of packed parameters. */
lbs_status lbs_mlp_num_params(lbs_mlp_handle h, long* out);
/* Set the FP32 master parameters from host memory (and their BF16 copies);
 * resets the Adam state.  LBS_ERR_NONFINITE for a non-finite value. */
lbs_status lbs_mlp_set_params(lbs_mlp_handle h, const float* host_params);
/* Copy the FP32 master parameters to host memory (synchronises). */
lbs_status lbs_mlp_get_params(lbs_mlp_handle h, float* host_params);
/* y = network(x) for B rows (asynchronous on the network's stream). */
lbs_status lbs_mlp_forward(lbs_mlp_handle h, const float* x_dev, int B, float* y_dev);
/* Forward and backward pass of the loss L = mean (y - t)^2 over the batch and the
 * outputs; the gradients stay on the device for lbs_mlp_adam.  loss_out and
 * grad_host (packed like the parameters) may be NULL; either one synchronises. */
lbs_status lbs_mlp_loss_grad(lbs_mlp_handle h, const float* x_dev, const float* t_dev, int B, double* loss_out,
                             float* grad_host);
/* One Adam step (bias-corrected) with the last gradients. */
lbs_status lbs_mlp_adam(lbs_mlp_handle h, float lr, float beta1, float beta2, float eps);
/* The network's CUDA stream. */
lbs_status lbs_mlp_get_stream(lbs_mlp_handle h, void** out);

/* Measurement helper (not in the paper): the current device's fused multiply-add
 * rate in FLOP/s (2 per FMA), FP64 and FP32, from CUDA events around a kernel of
 * independent FMA chains (8 per thread, 8 blocks of 256 threads per SM, best of 3
 * launches).  The FP64 solver is bound by this FP64 rate rather than by HBM.
 * Allocates and frees a few bytes of device memory; synchronises the device. */
lbs_status lbs_probe_fma_rate(double* fp64_flops, double* fp32_flops);

/* Message of the last error of the calling thread ("" if none). */
const char* lbs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBS_H */
