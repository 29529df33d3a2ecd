/*
 * Oracle of the mixed-quadrature Shakhov finite-difference lattice Boltzmann
 * scheme for Couette flow (plain FP64 C).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct CPU
 * reference the CUDA solver is checked against.  Only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark load it.  It shares no code
 * with the solver: its own equilibrium, moments, WENO-5, walls and RK3.
 *
 * Axes: z is normal to the walls (the paper's x), x is the flow direction (the
 * paper's y), y is the transverse direction (the paper's z, kept here as a
 * third full-range Gauss-Hermite axis instead of being integrated out).
 *
 * Reduced model (cfg.reduced = 1; Sec. III, Eqs. reduced_def, boltz_red,
 * phieq, sred_def): y is integrated out.  The index j then selects the field,
 * j = 0: phi = int f dp_y, j = 1: chi = int f p_y^2 dp_y (Qy = 2, p_y unused),
 * both on the (p_x, p_z) nodes, relaxing to phi_eq (1 + S_phi) and
 * chi_eq (1 + S_chi) with chi_eq = T phi_eq.  The transverse velocity and heat
 * flux vanish in Couette flow and are not carried.
 *
 * Storage: f[(s + 2) * Q + k] for cells s = -2 .. Nz+3 (three ghost cells per
 * side); k = ((sg * Qz + m) * Qx + i) * Qy + j, with p = (px[i], py[j], pz)
 * and pz = +xi[m] for sg = 0, -xi[m] for sg = 1.  f holds the discrete
 * populations with the quadrature weights absorbed (moments are plain sums).
 *
 * Passages followed:
 *   Shakhov model, Eqs. (boltz), (feq), (sdef); moments Eq. (qdef);
 *   direct-product truncated Hermite equilibrium, Sec. III, Eqs. (fyz),
 *   (Fmn_def), (H_ortho), and the half-range expansion of the wall-normal
 *   factor described there;
 *   relaxation times Eq. (mw_tau), the mu ~ T^omega law of Sec. VI and
 *   Eq. (sutherland_tau);
 *   RK-3 TVD, Eq. (rk3); flux divergence Eq. (flux); WENO-5, Eqs.
 *   (weno5_flux), (weno5_omega), (weno_sigma) and Table (weno);
 *   diffuse reflection with ghost nodes, quadratic extrapolation and the
 *   wall density n_w, Appendix "Boundary conditions".
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int Nz, Qx, Qy, Qz;       /* cells; nodes on x, on y, per sign on z       */
    int Nx, Ny, Nzq;          /* per-axis expansion orders (<= Q_a - 1)       */
    int visc_law;             /* 0: tau = Kn T^(omega-1)/n; 1: Sutherland      */
    int collisions;           /* 0: free streaming (tau = infinity)            */
    int shakhov;              /* 0: BGK (the S term is not formed at all)      */
    int periodic;             /* 1: periodic in z instead of walls (tests)     */
    int weno_linear;          /* 1: ideal weights only (tests of the linear    */
                              /*    structure; not the paper's scheme)          */
    int reduced;              /* 1: the phi / chi model (Qy = 2: j = field)    */
    double Kn, uw, Tw, Pr, visc_param, dt;
    const double *px, *wx;    /* [Qx] full-range nodes / weights (sum 1)      */
    const double *py, *wy;    /* [Qy]                                         */
    const double *xi, *wz;    /* [Qz] half-range nodes on (0,inf), weights     */
    const double *Hx;         /* [Qx][Nx+1]  He_l(px_i) / l!                   */
    const double *Hy;         /* [Qy][Ny+1]                                   */
    const double *Pz;         /* [Qz][Nzq+1] pi_l(xi_m) / h_l                  */
    const double *cz;         /* [Nzq+1][Nzq+1] monomial coeffs of pi_l        */
    const double *xc;         /* [Nz+6] cell centres, s = -2 .. Nz+3           */
    const double *xf;         /* [Nz+1] interfaces x_{s+1/2}, s = 0 .. Nz      */
} oracle_cfg;

#define ROW(s) ((s) + 2)

static int nvel(const oracle_cfg *c) { return 2 * c->Qz * c->Qx * c->Qy; }

static void vel_of(const oracle_cfg *c, int k, double p[3], int *sg, int *m, int *i, int *j)
{
    *j = k % c->Qy;
    *i = (k / c->Qy) % c->Qx;
    *m = (k / (c->Qy * c->Qx)) % c->Qz;
    *sg = k / (c->Qy * c->Qx * c->Qz);
    p[0] = c->px[*i];
    p[1] = c->py[*j];
    p[2] = (*sg == 0) ? c->xi[*m] : -c->xi[*m];
}

/* ------------------------------------------------------------------ */
/* Equilibrium                                                          */
/* ------------------------------------------------------------------ */

/* a_l = int g(p; u, T) He_l(p) dp for a Gaussian of mean u, variance T.
 * From the generating function sum_l He_l(p) t^l / l! = exp(p t - t^2/2):
 * a_l = l! [t^l] exp(u t + (T - 1) t^2 / 2).  (Eq. Fmn_def)                */
static double full_coeff(int l, double u, double T)
{
    double s = 0.0, lf = 1.0;
    for (int q = 2; q <= l; ++q) lf *= q;
    for (int jj = 0; 2 * jj <= l; ++jj) {
        double jf = 1.0, rf = 1.0;
        for (int q = 2; q <= jj; ++q) jf *= q;
        for (int q = 2; q <= l - 2 * jj; ++q) rf *= q;
        s += lf / (jf * rf) * pow(u, l - 2 * jj) * pow(0.5 * (T - 1.0), jj);
    }
    return s;
}

/* M_k = int_0^inf p^k g(p; u, T) dp, k = 0..K.  M_0 = erfc(-u/sqrt(2T))/2,
 * and integration by parts of p^k (p - u) g = -T p^k g' gives
 * M_{k+1} = u M_k + T g(0) [k == 0] + k T M_{k-1}.                         */
static void half_moments(double u, double T, int K, double *M)
{
    double g0 = exp(-u * u / (2.0 * T)) / sqrt(2.0 * M_PI * T);
    M[0] = 0.5 * erfc(-u / sqrt(2.0 * T));
    if (K >= 1) M[1] = u * M[0] + T * g0;
    for (int k = 1; k < K; ++k) M[k + 1] = u * M[k] + k * T * M[k - 1];
}

/* Per-axis discrete factors (weights included) of the truncated expansion. */
static void axis_factors(const oracle_cfg *c, double ux, double uy, double uz, double T,
                         double *Gx, double *Gy, double *Gzp, double *Gzm)
{
    double ax[32], ay[32], bp[32], bm[32], Mp[32], Mm[32];
    for (int l = 0; l <= c->Nx; ++l) ax[l] = full_coeff(l, ux, T);
    for (int l = 0; l <= c->Ny; ++l) ay[l] = full_coeff(l, uy, T);
    for (int i = 0; i < c->Qx; ++i) {
        double s = 0.0;
        for (int l = 0; l <= c->Nx; ++l) s += ax[l] * c->Hx[i * (c->Nx + 1) + l];
        Gx[i] = c->wx[i] * s;
    }
    if (c->reduced) {  /* phi_eq carries no y factor; chi_eq = T phi_eq */
        Gy[0] = 1.0;
        Gy[1] = T;
    } else {
        for (int j = 0; j < c->Qy; ++j) {
            double s = 0.0;
            for (int l = 0; l <= c->Ny; ++l) s += ay[l] * c->Hy[j * (c->Ny + 1) + l];
            Gy[j] = c->wy[j] * s;
        }
    }
    /* half range: p > 0 uses g(p; uz), p < 0 uses g(-p; uz) = g(p; -uz)    */
    half_moments(uz, T, c->Nzq, Mp);
    half_moments(-uz, T, c->Nzq, Mm);
    for (int l = 0; l <= c->Nzq; ++l) {
        double sp = 0.0, sm = 0.0;
        for (int q = 0; q <= l; ++q) {
            sp += c->cz[l * (c->Nzq + 1) + q] * Mp[q];
            sm += c->cz[l * (c->Nzq + 1) + q] * Mm[q];
        }
        bp[l] = sp;
        bm[l] = sm;
    }
    for (int m = 0; m < c->Qz; ++m) {
        double sp = 0.0, sm = 0.0;
        for (int l = 0; l <= c->Nzq; ++l) {
            sp += bp[l] * c->Pz[m * (c->Nzq + 1) + l];
            sm += bm[l] * c->Pz[m * (c->Nzq + 1) + l];
        }
        Gzp[m] = c->wz[m] * sp;
        Gzm[m] = c->wz[m] * sm;
    }
}

/* Discrete Shakhov target f^eq (1 + S) of one cell from the macroscopic
 * state mom = {n, ux, uy, uz, T, qx, qy, qz}.  with_S = 0 gives f^eq.      */
void oracle_equilibrium(const oracle_cfg *c, const double *mom, int with_S, double *feq)
{
    int Q = nvel(c);
    double n = mom[0], u[3] = {mom[1], mom[2], mom[3]}, T = mom[4];
    double q[3] = {mom[5], mom[6], mom[7]};
    double *Gx = malloc(sizeof(double) * (c->Qx + c->Qy + 2 * c->Qz));
    double *Gy = Gx + c->Qx, *Gzp = Gy + c->Qy, *Gzm = Gzp + c->Qz;
    axis_factors(c, u[0], u[1], u[2], T, Gx, Gy, Gzp, Gzm);
    double cS = (1.0 - c->Pr) / (n * T * T);
    for (int k = 0; k < Q; ++k) {
        double p[3];
        int sg, m, i, j;
        vel_of(c, k, p, &sg, &m, &i, &j);
        double base = n * Gx[i] * Gy[j] * (sg == 0 ? Gzp[m] : Gzm[m]);
        if (with_S && c->shakhov && c->reduced) {
            /* Eq. (sred_def): the y-averages of S over the Maxwellian in p_y,
             * with weight 1 (phi) or p_y^2 / T (chi); u_y = q_y = 0          */
            double ex = p[0] - u[0], ez = p[2] - u[2];
            double xq = ex * q[0] + ez * q[2];
            double off = (j == 0) ? 0.8 : 0.4;
            double S = cS * ((ex * ex + ez * ez) / (5.0 * T) - off) * xq;
            feq[k] = base * (1.0 + S);
        } else if (with_S && c->shakhov) {
            double xi2 = 0.0, xq = 0.0;
            for (int a = 0; a < 3; ++a) {
                double x = p[a] - u[a];
                xi2 += x * x;
                xq += x * q[a];
            }
            double S = cS * (xi2 / (5.0 * T) - 1.0) * xq;
            feq[k] = base * (1.0 + S);
        } else {
            feq[k] = base;
        }
    }
    free(Gx);
}

/* ------------------------------------------------------------------ */
/* Moments, Eq. (qdef):  out = {n, ux, uy, uz, T, qx, qy, qz,            */
/*                              Pxx, Pyy, Pzz, Pxy, Pxz, Pyz}             */
/* ------------------------------------------------------------------ */
static void reduced_moments(const oracle_cfg *c, const double *f, double *out);

void oracle_cell_moments(const oracle_cfg *c, const double *f, double *out)
{
    if (c->reduced) {
        reduced_moments(c, f, out);
        return;
    }
    int Q = nvel(c);
    double n = 0.0, nu[3] = {0, 0, 0};
    for (int k = 0; k < Q; ++k) {
        double p[3];
        int sg, m, i, j;
        vel_of(c, k, p, &sg, &m, &i, &j);
        n += f[k];
        for (int a = 0; a < 3; ++a) nu[a] += p[a] * f[k];
    }
    double u[3] = {nu[0] / n, nu[1] / n, nu[2] / n};
    double P[3][3] = {{0}}, q[3] = {0, 0, 0};
    for (int k = 0; k < Q; ++k) {
        double p[3], x[3];
        int sg, m, i, j;
        vel_of(c, k, p, &sg, &m, &i, &j);
        for (int a = 0; a < 3; ++a) x[a] = p[a] - u[a];
        double x2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b) P[a][b] += x[a] * x[b] * f[k];
            q[a] += 0.5 * x2 * x[a] * f[k];
        }
    }
    out[0] = n;
    out[1] = u[0]; out[2] = u[1]; out[3] = u[2];
    out[4] = (P[0][0] + P[1][1] + P[2][2]) / (3.0 * n);
    out[5] = q[0]; out[6] = q[1]; out[7] = q[2];
    out[8] = P[0][0]; out[9] = P[1][1]; out[10] = P[2][2];
    out[11] = P[0][1]; out[12] = P[0][2]; out[13] = P[1][2];
}

/* Moments of the reduced model: the p_y integrals are carried by chi.
 * n = sum phi, n u = sum p phi (u_y = 0); P_ab = sum xi_a xi_b phi for a, b in
 * {x, z}, P_yy = sum chi, P_xy = P_yz = 0; q_a = 1/2 sum (xi_x^2 + xi_z^2) xi_a phi
 * + 1/2 sum xi_a chi, q_y = 0; T = tr P / (3n).                             */
static void reduced_moments(const oracle_cfg *c, const double *f, double *out)
{
    int Q = nvel(c);
    double n = 0.0, nux = 0.0, nuz = 0.0;
    for (int k = 0; k < Q; ++k) {
        double p[3]; int sg, m, i, j;
        vel_of(c, k, p, &sg, &m, &i, &j);
        if (j != 0) continue;
        n += f[k];
        nux += p[0] * f[k];
        nuz += p[2] * f[k];
    }
    double ux = nux / n, uz = nuz / n;
    double Pxx = 0, Pzz = 0, Pxz = 0, Pyy = 0, qx = 0, qz = 0;
    for (int k = 0; k < Q; ++k) {
        double p[3]; int sg, m, i, j;
        vel_of(c, k, p, &sg, &m, &i, &j);
        double ex = p[0] - ux, ez = p[2] - uz;
        if (j == 0) {
            Pxx += ex * ex * f[k];
            Pzz += ez * ez * f[k];
            Pxz += ex * ez * f[k];
            qx += 0.5 * (ex * ex + ez * ez) * ex * f[k];
            qz += 0.5 * (ex * ex + ez * ez) * ez * f[k];
        } else {
            Pyy += f[k];
            qx += 0.5 * ex * f[k];
            qz += 0.5 * ez * f[k];
        }
    }
    out[0] = n;
    out[1] = ux; out[2] = 0.0; out[3] = uz;
    out[4] = (Pxx + Pyy + Pzz) / (3.0 * n);
    out[5] = qx; out[6] = 0.0; out[7] = qz;
    out[8] = Pxx; out[9] = Pyy; out[10] = Pzz;
    out[11] = 0.0; out[12] = Pxz; out[13] = 0.0;
}

/* Relaxation time: Eq. (mw_tau) generalised to mu ~ T^omega (Sec. VI), or
 * Eq. (sutherland_tau) with delta = 1 / (Kn sqrt 2).                       */
double oracle_tau(const oracle_cfg *c, double n, double T)
{
    if (c->visc_law == 0) return c->Kn * pow(T, c->visc_param - 1.0) / n;
    double S = c->visc_param;
    return c->Kn * sqrt(T) * (1.0 + S) / (n * (T + S));
}

/* ------------------------------------------------------------------ */
/* WENO-5 reconstruction, Eqs. (weno5_flux)-(weno_sigma), Table (weno).   */
/* v[0..4] are F_{s-2} .. F_{s+2} taken in the upwind direction.          */
/* ------------------------------------------------------------------ */
double oracle_weno5(const double *v)
{
    const double d[3] = {0.1, 0.6, 0.3};
    double c[3], s[3], w[3];
    c[0] = v[0] / 3.0 - 7.0 * v[1] / 6.0 + 11.0 * v[2] / 6.0;
    c[1] = -v[1] / 6.0 + 5.0 * v[2] / 6.0 + v[3] / 3.0;
    c[2] = v[2] / 3.0 + 5.0 * v[3] / 6.0 - v[4] / 6.0;
    double a, b;
    a = v[0] - 2.0 * v[1] + v[2]; b = v[0] - 4.0 * v[1] + 3.0 * v[2];
    s[0] = 13.0 / 12.0 * a * a + 0.25 * b * b;
    a = v[1] - 2.0 * v[2] + v[3]; b = v[1] - v[3];
    s[1] = 13.0 / 12.0 * a * a + 0.25 * b * b;
    a = v[2] - 2.0 * v[3] + v[4]; b = 3.0 * v[2] - 4.0 * v[3] + v[4];
    s[2] = 13.0 / 12.0 * a * a + 0.25 * b * b;
    /* The weights do not change when the three sigma are scaled together,
     * so they are formed from r_q = sigma_q / max sigma.  A sigma that
     * vanishes (r_q below 1e-150, where d_q / r_q^2 would overflow) takes the
     * limits of Table (weno): the weights are then proportional to d_q over
     * the vanishing set and zero elsewhere.                                */
    double smax = s[0];
    if (s[1] > smax) smax = s[1];
    if (s[2] > smax) smax = s[2];
    int nz = 0, zero[3];
    for (int q = 0; q < 3; ++q) {
        zero[q] = (smax == 0.0) || (s[q] / smax < 1e-150);
        nz += zero[q];
    }
    double tot = 0.0;
    for (int q = 0; q < 3; ++q) {
        if (nz > 0) {
            w[q] = zero[q] ? d[q] : 0.0;
        } else {
            double r = s[q] / smax;
            w[q] = d[q] / (r * r);
        }
        tot += w[q];
    }
    return (w[0] * c[0] + w[1] * c[1] + w[2] * c[2]) / tot;
}

/* The linear fifth-order upwind reconstruction (ideal weights d_q). */
static double linear5(const double *v)
{
    double c1 = v[0] / 3.0 - 7.0 * v[1] / 6.0 + 11.0 * v[2] / 6.0;
    double c2 = -v[1] / 6.0 + 5.0 * v[2] / 6.0 + v[3] / 3.0;
    double c3 = v[2] / 3.0 + 5.0 * v[3] / 6.0 - v[4] / 6.0;
    return 0.1 * c1 + 0.6 * c2 + 0.3 * c3;
}

/* Flux through interface s+1/2 (between cells s and s+1) of velocity k.
 * For p_z < 0 the stencil is the mirror image F_{s+1-j}.                  */
static double iface_flux(const oracle_cfg *c, const double *F, int s, int k, double pz)
{
    int Q = nvel(c);
    double v[5];
    for (int jj = -2; jj <= 2; ++jj)
        v[jj + 2] = (pz > 0.0) ? F[ROW(s + jj) * Q + k] : F[ROW(s + 1 - jj) * Q + k];
    return pz * (c->weno_linear ? linear5(v) : oracle_weno5(v));
}

/* Lagrange weight of node b in the quadratic through a, b, d evaluated at x. */
static double lag(double x, double xb, double xa, double xd)
{
    return (x - xa) * (x - xd) / ((xb - xa) * (xb - xd));
}

/* ------------------------------------------------------------------ */
/* Ghost nodes: diffuse reflection at z = +-L/2 (Appendix, "Boundary      */
/* conditions"), or periodic copies when c->periodic.  nw (may be NULL)   */
/* receives {n_w bottom, n_w top}.                                        */
/* ------------------------------------------------------------------ */
void oracle_apply_walls(const oracle_cfg *c, double *F, double *nw)
{
    int Q = nvel(c), Nz = c->Nz, half = Q / 2;
    if (c->periodic) {
        for (int g = 0; g < 3; ++g) {
            memcpy(&F[ROW(-g) * Q], &F[ROW(Nz - g) * Q], sizeof(double) * Q);
            memcpy(&F[ROW(Nz + 1 + g) * Q], &F[ROW(1 + g) * Q], sizeof(double) * Q);
        }
        return;
    }
    double *Fw = malloc(sizeof(double) * Q);
    const double *x = c->xc;

    /* ---- top wall, z = +L/2, moving with +u_w; outgoing: p_z > 0 ------- */
    for (int s = Nz + 1; s <= Nz + 2; ++s) {
        double xs = x[ROW(s)], x1 = x[ROW(s - 1)], x2 = x[ROW(s - 2)], x3 = x[ROW(s - 3)];
        double l1 = lag(xs, x1, x2, x3), l2 = lag(xs, x2, x1, x3), l3 = lag(xs, x3, x1, x2);
        for (int k = 0; k < half; ++k)
            F[ROW(s) * Q + k] = l1 * F[ROW(s - 1) * Q + k] + l2 * F[ROW(s - 2) * Q + k] +
                                l3 * F[ROW(s - 3) * Q + k];
    }
    /* mass flux: every population in the full model, phi alone in the reduced one */
    double phi = 0.0, D = 0.0;
    for (int k = 0; k < half; ++k) {
        double p[3]; int sg, m, i, j;
        vel_of(c, k, p, &sg, &m, &i, &j);
        if (c->reduced && j != 0) continue;
        phi += iface_flux(c, F, Nz, k, p[2]);
    }
    double momw[8] = {1.0, c->uw, 0.0, 0.0, c->Tw, 0.0, 0.0, 0.0};
    oracle_equilibrium(c, momw, 0, Fw);
    for (int k = half; k < Q; ++k) {
        double p[3]; int sg, m, i, j;
        vel_of(c, k, p, &sg, &m, &i, &j);
        if (c->reduced && j != 0) continue;
        D += p[2] * Fw[k];
    }
    double nwt = -phi / D;
    for (int s = Nz + 1; s <= Nz + 3; ++s)
        for (int k = half; k < Q; ++k) F[ROW(s) * Q + k] = nwt * Fw[k];

    /* ---- bottom wall, z = -L/2, moving with -u_w; outgoing: p_z < 0 ---- */
    for (int s = 0; s >= -1; --s) {
        double xs = x[ROW(s)], x1 = x[ROW(s + 1)], x2 = x[ROW(s + 2)], x3 = x[ROW(s + 3)];
        double l1 = lag(xs, x1, x2, x3), l2 = lag(xs, x2, x1, x3), l3 = lag(xs, x3, x1, x2);
        for (int k = half; k < Q; ++k)
            F[ROW(s) * Q + k] = l1 * F[ROW(s + 1) * Q + k] + l2 * F[ROW(s + 2) * Q + k] +
                                l3 * F[ROW(s + 3) * Q + k];
    }
    phi = 0.0; D = 0.0;
    for (int k = half; k < Q; ++k) {
        double p[3]; int sg, m, i, j;
        vel_of(c, k, p, &sg, &m, &i, &j);
        if (c->reduced && j != 0) continue;
        phi += iface_flux(c, F, 0, k, p[2]);
    }
    momw[1] = -c->uw;
    oracle_equilibrium(c, momw, 0, Fw);
    for (int k = 0; k < half; ++k) {
        double p[3]; int sg, m, i, j;
        vel_of(c, k, p, &sg, &m, &i, &j);
        if (c->reduced && j != 0) continue;
        D += p[2] * Fw[k];
    }
    double nwb = -phi / D;
    for (int s = -2; s <= 0; ++s)
        for (int k = 0; k < half; ++k) F[ROW(s) * Q + k] = nwb * Fw[k];

    if (nw) { nw[0] = nwb; nw[1] = nwt; }
    free(Fw);
}

/* Interface fluxes (s = 0..Nz) of every velocity, walls already applied.  */
static void all_fluxes(const oracle_cfg *c, const double *F, double *flux)
{
    int Q = nvel(c), Nz = c->Nz;
#pragma omp parallel for schedule(static)
    for (int s = 0; s <= Nz; ++s) {
        for (int k = 0; k < Q; ++k) {
            double p[3]; int sg, m, i, j;
            vel_of(c, k, p, &sg, &m, &i, &j);
            flux[s * Q + k] = iface_flux(c, F, s, k, p[2]);
        }
    }
}

/* L[F] of Eq. (L_def) on the interior cells (ghosts of F already set).    */
static void rhs(const oracle_cfg *c, const double *F, double *L, double *flux)
{
    int Q = nvel(c), Nz = c->Nz;
    all_fluxes(c, F, flux);
#pragma omp parallel for schedule(static)
    for (int s = 1; s <= Nz; ++s) {
        const double *Fs = &F[ROW(s) * Q];
        double *Ls = &L[ROW(s) * Q];
        double dx = c->xf[s] - c->xf[s - 1];
        for (int k = 0; k < Q; ++k) Ls[k] = -(flux[s * Q + k] - flux[(s - 1) * Q + k]) / dx;
        if (c->collisions) {
            double mom[14];
            oracle_cell_moments(c, Fs, mom);
            double tau = oracle_tau(c, mom[0], mom[4]);
            double *fS = malloc(sizeof(double) * Q);
            oracle_equilibrium(c, mom, 1, fS);
            for (int k = 0; k < Q; ++k) Ls[k] -= (Fs[k] - fS[k]) / tau;
            free(fS);
        }
    }
}

/* Profiles n, u_x, T (interior cells) used by the residual.               */
static void res_profiles(const oracle_cfg *c, const double *F, double *W)
{
    int Q = nvel(c), Nz = c->Nz;
    for (int s = 1; s <= Nz; ++s) {
        double mom[14];
        oracle_cell_moments(c, &F[ROW(s) * Q], mom);
        W[0 * Nz + s - 1] = mom[0];
        W[1 * Nz + s - 1] = mom[1];
        W[2 * Nz + s - 1] = mom[4];
    }
}

/* R = max over W in {n, u_x, T} of ||W_new - W_old||_2 / max(||W_old||_2, s_W);
 * W[3][Nz] holds n, u_x, T of the interior cells (the paper states no criterion:
 * this is the solver's).  s_n = s_T = 1e-30; the velocity is measured on the wall
 * speed where it is smaller, s_u = max(|u_w| sqrt(Nz), 1e-30) (the norm of a profile
 * at the wall speed), since u_x itself vanishes in the free-molecular limit and at
 * u_w = 0.  Exported for its pin.                                             */
double oracle_residual(int Nz, const double *Wo, const double *Wn, double uw)
{
    double R = 0.0;
    for (int a = 0; a < 3; ++a) {
        double d = 0.0, o = 0.0;
        for (int s = 0; s < Nz; ++s) {
            double e = Wn[a * Nz + s] - Wo[a * Nz + s];
            d += e * e;
            o += Wo[a * Nz + s] * Wo[a * Nz + s];
        }
        double floor = a == 1 ? fmax(fabs(uw) * sqrt((double)Nz), 1e-30) : 1e-30;
        double r = sqrt(d) / fmax(sqrt(o), floor);
        if (r > R) R = r;
    }
    return R;
}

/* nsteps RK-3 TVD steps, Eq. (rk3), walls imposed on every stage input.
 * res (may be NULL) receives the residual of every step.                  */
void oracle_step(const oracle_cfg *c, double *F0, long nsteps, double *res)
{
    int Q = nvel(c), Nz = c->Nz;
    size_t N = (size_t)(Nz + 6) * Q;
    double *F1 = calloc(N, sizeof(double)), *F2 = calloc(N, sizeof(double));
    double *L = calloc(N, sizeof(double)), *flux = calloc((size_t)(Nz + 1) * Q, sizeof(double));
    double *Wo = malloc(sizeof(double) * 3 * Nz), *Wn = malloc(sizeof(double) * 3 * Nz);
    const double dt = c->dt;
    if (res) res_profiles(c, F0, Wo);
    for (long it = 0; it < nsteps; ++it) {
        size_t a = (size_t)ROW(1) * Q, b = (size_t)ROW(Nz + 1) * Q;
        oracle_apply_walls(c, F0, NULL);
        rhs(c, F0, L, flux);
        for (size_t e = a; e < b; ++e) F1[e] = F0[e] + dt * L[e];
        oracle_apply_walls(c, F1, NULL);
        rhs(c, F1, L, flux);
        for (size_t e = a; e < b; ++e) F2[e] = 0.75 * F0[e] + 0.25 * F1[e] + 0.25 * dt * L[e];
        oracle_apply_walls(c, F2, NULL);
        rhs(c, F2, L, flux);
        for (size_t e = a; e < b; ++e)
            F0[e] = F0[e] / 3.0 + 2.0 * F2[e] / 3.0 + 2.0 * dt * L[e] / 3.0;
        if (res) {
            res_profiles(c, F0, Wn);
            res[it] = oracle_residual(Nz, Wo, Wn, c->uw);
            double *t = Wo; Wo = Wn; Wn = t;
        }
    }
    free(F1); free(F2); free(L); free(flux); free(Wo); free(Wn);
}

/* Profiles of every interior cell: out[14][Nz] in the order of
 * oracle_cell_moments.                                                    */
void oracle_profiles(const oracle_cfg *c, const double *F, double *out)
{
    int Q = nvel(c), Nz = c->Nz;
    for (int s = 1; s <= Nz; ++s) {
        double mom[14];
        oracle_cell_moments(c, &F[ROW(s) * Q], mom);
        for (int a = 0; a < 14; ++a) out[a * Nz + s - 1] = mom[a];
    }
}

/* Interface sums sum_k psi_k Flux_{s+1/2,k}, s = 0..Nz, for
 * psi = {1, p_x, p_z, |p|^2 / 2}: out[Nz+1][4].  Walls are imposed on a
 * copy of F first (the state is not modified).                            */
void oracle_interface_sums(const oracle_cfg *c, const double *F, double *out)
{
    int Q = nvel(c), Nz = c->Nz;
    size_t N = (size_t)(Nz + 6) * Q;
    double *G = malloc(sizeof(double) * N), *flux = malloc(sizeof(double) * (Nz + 1) * Q);
    memcpy(G, F, sizeof(double) * N);
    oracle_apply_walls(c, G, NULL);
    all_fluxes(c, G, flux);
    for (int s = 0; s <= Nz; ++s) {
        double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        for (int k = 0; k < Q; ++k) {
            double p[3]; int sg, m, i, j;
            vel_of(c, k, p, &sg, &m, &i, &j);
            double fl = flux[s * Q + k];
            if (c->reduced && j == 1) {  /* chi carries the p_y^2 / 2 of the energy */
                a3 += 0.5 * fl;
                continue;
            }
            a0 += fl;
            a1 += p[0] * fl;
            a2 += p[2] * fl;
            a3 += 0.5 * (p[0] * p[0] + p[1] * p[1] + p[2] * p[2]) * fl;
        }
        out[s * 4 + 0] = a0; out[s * 4 + 1] = a1; out[s * 4 + 2] = a2; out[s * 4 + 3] = a3;
    }
    free(G); free(flux);
}
