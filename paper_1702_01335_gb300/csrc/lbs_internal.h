// Internal definitions shared by the host set-up and the CUDA kernels.
#pragma once

#if __has_include(<vector_types.h>)
#include <vector_types.h>  // float2 (also for the host-only translation units)
#else
struct float2;  // host code built without the CUDA headers holds only pointers to it
#endif

#include <cmath>
#include <vector>

#if defined(__CUDACC__)
#define LBS_HD __host__ __device__ __forceinline__
#else
#define LBS_HD inline
#endif

namespace lbs {

constexpr int kMaxQ1D = 100;    // nodes per axis (per sign on z): the largest order of the paper
constexpr int kMaxN = 8;        // equilibrium expansion order
constexpr int kNMom = 13;       // raw moments accumulated per cell
constexpr int kRecHead = 12;    // scalars at the head of a cell record
constexpr int kThreads = 128;   // threads of a stage CTA
constexpr int kMaxZT = 64;      // cells of a z-tile

enum { QUAD_FULL = 0, QUAD_HALF = 1 };

// Cell record (storage type T): n, ux, uy, uz, T, qx, qy, qz, 1/tau,
// (1 - Pr)/(n T^2), 1/(5T), R_SCALE - 1 where R_SCALE = n / (discrete weighted sums of
// the per-axis factors); then the per-node factors of the truncated equilibrium as
// deviations from the rest state's factor 1 (the populations are stored as deviations
// from the rest state too): dx[Qx] = Gx / w - 1 (before R_SCALE), dy[Qy], dz[2 Qz]
// (p_z > 0 nodes, then p_z < 0).  They are summed in FP64 in the finalisation and
// rounded once to the storage type.  Records are rec_stride values apart.
enum { R_N = 0, R_UX, R_UY, R_UZ, R_T, R_QX, R_QY, R_QZ, R_ITAU, R_CS, R_I5T, R_SCALE1 };
constexpr int R_DX = kRecHead;
// record length of an instance, rounded up to 16 bytes in either storage type
inline int rec_stride_of(int Qx, int Qy, int Qz) { return (kRecHead + Qx + Qy + 2 * Qz + 3) & ~3; }

// Everything a kernel needs to know about one instance (lives in device memory).
struct InstDev {
    int Nz, Qx, Qy, Qz, Q, QxQy;
    int Nx, Ny, Nzq;              // per-axis expansion orders
    int nchunks, bulk;            // bulk: rows are 16-byte aligned, stage them with TMA bulk copies
    int nchh;                     // chunks per half range of p_z (chunk c has p_z < 0 iff c >= nchh)
    int half;                     // 1: half channel, bounce-back ghosts below cell 0 (no bottom wall)
    int fin_warp;                 // finalisation with one warp per cell (small batches) instead of one thread
    int reduced;                  // 1: the phi / chi model (Qy = 2: j = 0 phi, j = 1 chi; p_y unused)
    int visc_law;
    double Kn, visc_param, Pr, dt, tol;
    double res_uscale;            // the residual's velocity scale max(|u_w| sqrt(Nz), 1e-30)
    double iKn, isuth;            // 1 / Kn; Sutherland: 1 / (1 + S)
    double Dtop, Dbot;            // sum over incoming velocities of w p_z Gw (n_w = 1)
    int rec_stride;               // values per cell record
    double mrest[kNMom];          // raw moments of the rest state f = w (the stored weights and
                                  // nodes): the partials hold sums over the deviations only
    double frest_bot, frest_top;  // outgoing wall flux of the rest state (sum w p_z over the
                                  // velocities leaving through each wall)
    unsigned wait_limit;          // spins of the bounded wait for the bulk copies
    double ext_top[2][3];         // ghost Nz+1 <- (Nz, Nz-1, Nz-2); Nz+2 <- (Nz+1, Nz, Nz-1)
    double ext_bot[2][3];         // ghost 0 <- (1, 2, 3); ghost -1 <- (0, 1, 2)
    // tables
    const double *Hx, *Hy, *Pz;   // FP64, [Q_a][N_a + 1] basis values He_l/l!, pi_l/h_l
    const float2 *Hx2, *Hy2, *Pz2;  // the same as FP32 (hi, lo) pairs, hi + lo = the FP64 value
                                    // to 2^-48 (FP32 storage: the records' node sums)
    double sumw_x, sumw_y, sumw_z;  // sums of the stored weights (z: over both half ranges)
    const double *alpha, *beta;   // half-range recurrence, [kMaxN + 2]
    // storage-typed tables (float or double)
    const void *px, *py, *xi, *wx, *wy, *wz;
    const void *gwx_top, *gwx_bot, *gwy, *gwz;  // wall equilibria per axis (Q_x, Q_x, Q_y, 2Q_z),
                                                 // deviations from 1 of the normalised factors
    const void *inv_dz;                          // [Nz]
    // state and work.  The state is d = f / w - 1 (deviation of the normalised populations
    // from the rest Maxwellian), [Nz][Q].  F0 and F1 take turns: *cur = 0 means F0 holds d
    // and F1 the stage-1 increment d1 = F1 - F_l; *cur = 1 the reverse.  F2 holds the
    // stage-2 increment d2 = F2 - F_l.  Stage 3 writes the new d over the stage-1
    // increment (no longer needed) and flips *cur, so no stage writes what another CTA
    // of the same launch still reads.  FP32 storage keeps the rounding residual of d in
    // L0 (16-bit fixed point in units of 2^-15 ulp(d), see lo_encode).
    void *F0, *F1, *F2;
    unsigned short *L0;           // [Nz][Q], FP32 storage only
    int *cur;                     // [1]
    void *rec;                    // [Nz][rec_stride]
    void *partial;                // [nchunks][kNMom][Nz] in the accumulation type (FP32 sums of FP32 storage)
    double *flux_part;            // [nchunks][2]: bottom, top outgoing flux
    double *nw;                   // [2]: bottom, top wall density
    double *prof;                 // [14][Nz]
    double *Wold, *Wnew;          // [3][Nz]: n, u_x, T
    double *res;                  // [1]
    long long *steps;             // [1]
    int *active;                  // [1]
    int *zcount;                  // [nzt] chunks of a z-tile finished this stage (ticket counters)
    int *icount;                  // [1] z-tiles of the instance finalised this stage
    int nzt;                      // z-tiles of the current tiling
    int *status;                  // [1]: bit 0 non-finite / non-positive n, T; bit 1 a bounded
                                  // wait for the bulk copies ran out
};

enum { STATUS_NONFINITE = 1, STATUS_TIMEOUT = 2 };
constexpr unsigned kWaitLimit = 1u << 26;   // default spins of the bounded wait (~seconds)
constexpr unsigned kDrainLimit = 1u << 28;  // spins granted to copies still in flight after a timeout

struct Tile { int inst, z0, zn, chunk, zt; };

// ---- equilibrium coefficients (shared by host set-up and device finalise) ----

// a_l = int g(p; u, T) He_l(p) dp: a_0 = 1, a_1 = u, a_{l+1} = u a_l + l (T - 1) a_{l-1}
// (from int g p He_l = u a_l + T l a_{l-1} and He_{l+1} = p He_l - l He_{l-1}).
// Loops below run to a bound NB on the order (the largest order kMaxN by default;
// device code instantiates smaller bounds for batches of low order) and test the
// actual order inside, so that, unrolled, every array index is a constant and device
// code keeps the arrays in registers instead of local memory.
#if defined(__CUDACC__)
#define LBS_UNROLL _Pragma("unroll")
#else
#define LBS_UNROLL
#endif

template <int NB = kMaxN>
LBS_HD void full_coeffs(double u, double T, int N, double* a)
{
    a[0] = 1.0;
    a[1] = u;  // read only when N >= 1
    LBS_UNROLL
    for (int l = 1; l < NB; ++l)
        if (l < N) a[l + 1] = u * a[l] + l * (T - 1.0) * a[l - 1];
}

// b_l = int_0^inf g(p; u, T) pi_l(p) dp for the monic half-range polynomials,
// by the modified-moment recurrence J_{l+1,k} = J_{l,k+1} - alpha_l J_{l,k} -
// beta_l J_{l-1,k} started from the half-line Gaussian moments
// J_{0,k} = M_k: M_0 = erfc(-u/sqrt(2T))/2, M_1 = u M_0 + T g(0),
// M_{k+1} = u M_k + k T M_{k-1}.
LBS_HD void half_coeffs(double u, double T, int N, const double* alpha, const double* beta,
                        double* b)
{
    double J[kMaxN + 1][kMaxN + 1];  // J[l][k] is needed for k <= N - l only
    const int K = N;
    const double g0 = exp(-u * u / (2.0 * T)) * (1.0 / sqrt(2.0 * M_PI * T));
    J[0][0] = 0.5 * erfc(-u / sqrt(2.0 * T));
    if (K >= 1) J[0][1] = u * J[0][0] + T * g0;
    for (int k = 1; k < K; ++k) J[0][k + 1] = u * J[0][k] + k * T * J[0][k - 1];
    for (int l = 0; l < N; ++l)
        for (int k = 0; k + l + 1 <= K; ++k)
            J[l + 1][k] = J[l][k + 1] - alpha[l] * J[l][k] - (l > 0 ? beta[l] * J[l - 1][k] : 0.0);
    for (int l = 0; l <= N; ++l) b[l] = J[l][0];
}

// erfc(x) for x >= 0.  For x < 1/2 from the Maclaurin series of erf,
//   erf(x) = (2 / sqrt(pi)) sum_n (-1)^n x^(2n+1) / (n! (2n+1))
// (Abramowitz & Stegun 7.1.5), 14 terms in Horner form in x^2: the last omitted
// term is below 3e-18 of erf(1/2), and erfc = 1 - erf lies in [0.47, 1] there, so
// the result is accurate to rounding.  That is a chain of 14 FMAs instead of the
// library's much longer evaluation.  It sits on the critical path of every cell
// record; in Couette flow the wall-normal drift u_z, hence x, is small.  Larger x
// use erfc itself.
struct ErfSeries {
    double c[14];
    constexpr ErfSeries() : c()
    {
        double fact = 1.0;
        for (int n = 0; n < 14; ++n) {
            if (n > 0) fact *= n;
            c[n] = (n % 2 ? -1.0 : 1.0) * 1.1283791670955125739 / (fact * (2 * n + 1));  // 2 / sqrt(pi)
        }
    }
};
LBS_HD double erfc_nonneg(double x)
{
    if (x >= 0.5) return erfc(x);
    constexpr ErfSeries S;
    const double t = x * x;
    double p = S.c[13];
#pragma unroll
    for (int n = 12; n >= 0; --n) p = fma(p, t, S.c[n]);
    return 1.0 - x * p;
}

// Both half-range coefficient sets at once: bp for u, bm for -u (the p_z < 0 half
// range, written in xi = -p_z >= 0).  The two share g(0) and, through
// erfc(x) + erfc(-x) = 2, one erfc: the one of |x| is evaluated (no cancellation)
// and the other is 2 minus it (a value in [1, 2], exact to an ulp).
template <int NB = kMaxN>
LBS_HD void half_coeffs_pm(double u, double T, double iT, int N, const double* alpha, const double* beta,
                           double* bp, double* bm)
{
    // iT = 1 / T, which the caller has at hand.  Rows J_{l,k} (k <= N - l) of the two
    // recurrences; only rows l - 1 and l are kept.
    const int K = N;
    const double r2T = sqrt(0.5 * iT);
    const double g0 = exp(-0.5 * u * u * iT) * (r2T * (1.0 / sqrt(M_PI)));
    const double e = erfc_nonneg(fabs(u) * r2T);  // erfc of the non-negative argument
    double Pp[kMaxN + 1], Pc[kMaxN + 1], Mp[kMaxN + 1], Mc[kMaxN + 1];
    Pc[0] = u >= 0.0 ? 1.0 - 0.5 * e : 0.5 * e;  // erfc(-u / sqrt(2T)) / 2
    Mc[0] = u >= 0.0 ? 0.5 * e : 1.0 - 0.5 * e;  // erfc(u / sqrt(2T)) / 2
    Pc[1] = u * Pc[0] + T * g0;                  // used only when K >= 1
    Mc[1] = -u * Mc[0] + T * g0;
    LBS_UNROLL
    for (int k = 1; k < NB; ++k)
        if (k < K) {
            Pc[k + 1] = u * Pc[k] + k * T * Pc[k - 1];
            Mc[k + 1] = -u * Mc[k] + k * T * Mc[k - 1];
        }
    bp[0] = Pc[0];
    bm[0] = Mc[0];
    LBS_UNROLL
    for (int l = 0; l < NB; ++l) {
        if (l < N) {
            const double al = alpha[l], be = l > 0 ? beta[l] : 0.0;
            double Pn[kMaxN + 1], Mn[kMaxN + 1];
            LBS_UNROLL
            for (int k = 0; k + l + 1 <= NB; ++k)
                if (k + l + 1 <= K) {
                    Pn[k] = Pc[k + 1] - al * Pc[k] - (l > 0 ? be * Pp[k] : 0.0);
                    Mn[k] = Mc[k + 1] - al * Mc[k] - (l > 0 ? be * Mp[k] : 0.0);
                }
            LBS_UNROLL
            for (int k = 0; k + l + 1 <= NB; ++k) {
                Pp[k] = Pc[k];
                Pc[k] = Pn[k];
                Mp[k] = Mc[k];
                Mc[k] = Mn[k];
            }
            bp[l + 1] = Pc[0];
            bm[l + 1] = Mc[0];
        }
    }
}

// Macroscopic state of a cell from its 13 raw moments (FP64): n, u, the central
// second moments P_ab = sum p_a p_b f - n u_a u_b, T = tr P / (3n) and the heat flux
// q_a = 1/2 sum |xi|^2 xi_a f with xi = p - u (Eq. qdef), expanded in raw moments.
struct CellState {
    double n, in, u[3], T, q[3], P[6];  // P: xx, yy, zz, xy, xz, yz
};
LBS_HD void cell_state(const double* mom, CellState& c)
{
    const double n = mom[0], in = 1.0 / n;
    c.n = n;
    c.in = in;
    c.u[0] = mom[1] * in; c.u[1] = mom[2] * in; c.u[2] = mom[3] * in;
    const double* u = c.u;
    c.P[0] = mom[4] - n * u[0] * u[0]; c.P[1] = mom[5] - n * u[1] * u[1];
    c.P[2] = mom[6] - n * u[2] * u[2]; c.P[3] = mom[7] - n * u[0] * u[1];
    c.P[4] = mom[8] - n * u[0] * u[2]; c.P[5] = mom[9] - n * u[1] * u[2];
    c.T = (c.P[0] + c.P[1] + c.P[2]) * (1.0 / 3.0) * in;
    const double M2[3][3] = {{mom[4], mom[7], mom[8]}, {mom[7], mom[5], mom[9]}, {mom[8], mom[9], mom[6]}};
    const double tr = mom[4] + mom[5] + mom[6];
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double um = u[0] * mom[1] + u[1] * mom[2] + u[2] * mom[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double uM2 = u[0] * M2[0][a] + u[1] * M2[1][a] + u[2] * M2[2][a];
        c.q[a] = 0.5 * (mom[10 + a] - u[a] * tr - 2.0 * uM2 + 2.0 * u[a] * um + uu * mom[1 + a] - uu * u[a] * n);
    }
}

// The 13 raw moments m (order of cell_state: 1, p_a, p_a p_b (xx yy zz xy xz yz),
// |p|^2 p_a) of a distribution re-expressed about the velocity u: the moments of
// psi(p - u).  |p - u|^2 (p_a - u_a) = |p|^2 p_a - u_a |p|^2 - 2 (p.u) p_a + 2 u_a (p.u)
// + |u|^2 p_a - |u|^2 u_a.
LBS_HD void shift_moments(const double* m, const double* u, double* out)
{
    const double m0 = m[0], m1[3] = {m[1], m[2], m[3]};
    const double M2[3][3] = {{m[4], m[7], m[8]}, {m[7], m[5], m[9]}, {m[8], m[9], m[6]}};
    out[0] = m0;
    for (int a = 0; a < 3; ++a) out[1 + a] = m1[a] - u[a] * m0;
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    for (int e = 0; e < 6; ++e) {
        const int a = ia[e], b = ib[e];
        out[4 + e] = M2[a][b] - u[a] * m1[b] - u[b] * m1[a] + u[a] * u[b] * m0;
    }
    const double tr = m[4] + m[5] + m[6], uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double um = u[0] * m1[0] + u[1] * m1[1] + u[2] * m1[2];
    for (int a = 0; a < 3; ++a) {
        const double uM2 = u[0] * M2[0][a] + u[1] * M2[1][a] + u[2] * M2[2][a];
        out[10 + a] = m[10 + a] - u[a] * tr - 2.0 * uM2 + 2.0 * u[a] * um + uu * m1[a] - uu * u[a] * m0;
    }
}

// 1 / tau from 1 / n, 1 / T, 1 / Kn and (Sutherland) 1 / (1 + S), without a
// division: power law n T^(1 - omega) / Kn, Sutherland n (T + S) / (Kn sqrt(T) (1 + S))
LBS_HD double inv_relax_time(int law, double iKn, double param, double isuth, double n, double T, double iT)
{
    if (law == 0) {
        if (param == 1.0) return n * iKn;
        if (param == 0.5) return n * iKn * sqrt(T);
        return n * iKn * pow(T, 1.0 - param);
    }
    return n * (T + param) * iKn * isuth * sqrt(iT);
}

// relaxation time: power law tau = Kn T^(omega-1)/n, Sutherland tau = Kn sqrt(T)(1+S)/(n(T+S))
LBS_HD double relax_time(int law, double Kn, double param, double n, double T)
{
    if (law == 0) {
        // the hard-sphere and Maxwell-molecule exponents without a general pow
        if (param == 1.0) return Kn / n;
        if (param == 0.5) return Kn / (n * sqrt(T));
        return Kn * pow(T, param - 1.0) / n;
    }
    return Kn * sqrt(T) * (1.0 + param) / (n * (T + param));
}

// ---- access to a handle for entry points defined outside api.cu ----
struct HandleView {
    const InstDev* d_inst;   // device array of descriptors
    InstDev inst;            // host copy of the selected instance's descriptor
    int fp32, device;
    void* stream;            // cudaStream_t
};
// fills *out for instance inst of handle h (an lbs_handle); returns 0 or an lbs_status
int handle_view(void* h, int inst, HandleView* out);
// records msg as the calling thread's last error and returns status
int record_error(int status, const char* msg);

// ---- host helpers (quadrature.cpp) ----
void recurrence(int kind, int n, std::vector<double>& alpha, std::vector<double>& beta);
int gauss_rule(int kind, int Q, double* nodes, double* weights);
void hermite_basis(const double* p, int Q, int N, double* out);
void half_basis(const double* xi, int Q, int N, const std::vector<double>& a,
                const std::vector<double>& b, double* out);

}  // namespace lbs
