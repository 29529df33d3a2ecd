// CUDA kernels of one RK-3 stage of the mixed-quadrature Shakhov scheme.
//
// Per stage (Eq. rk3 around Eq. L_def):
//   stage_kernel     one CTA per tile = (instance, z-range, velocity chunk).
//                    Each thread owns V velocities and marches up its z-range
//                    with a register window of F_in; it forms the WENO-5
//                    interface fluxes (Eqs. weno5_flux - weno_sigma, Table
//                    weno), the divergence of Eq. (flux), the relaxation to
//                    the cell's Shakhov target and the Shu-Osher combine, and
//                    stores F_out.  Ghost values are synthesised in registers:
//                    outgoing ones by the quadratic extrapolation of the
//                    Appendix, incoming ones as n_w times the wall
//                    equilibrium.  In the same pass it accumulates the raw
//                    moments of F_out per cell and, in tiles that end at a
//                    wall, the outgoing WENO flux of F_out through the wall
//                    interface, so the next stage needs no extra read of F.
//   finalize_cells   one CTA per cell: sums the per-chunk moment partials in
//                    FP64, forms n, u, P, T, q (Eq. qdef) and tau, and writes
//                    the cell record (the per-axis factors of the truncated
//                    Hermite equilibrium, Sec. III) used by the next stage.
//   finalize_inst    one CTA per instance: wall densities n_w (zero net mass
//                    flux, Appendix) and, after the third stage, the residual.
//
// Storage: F[s][k] for interior cells s = 0..Nz-1 (no ghost rows), velocity
// k = ((sg*Qz + m)*Qx + i)*Qy + j fastest, holding f_k / w_k.
#include <cuda_runtime.h>

#include "lbs_internal.h"

namespace lbs {

template <typename T> struct Acc { typedef double type; };
template <> struct Acc<float> { typedef float type; };

// WENO-5 reconstruction of five upwind-ordered values (no advection factor).
// The weights are scale free, so they are formed from r_q = sigma_q / max
// sigma; an r_q below kTiny counts as vanishing and the weights of Table
// (weno) apply (proportional to the ideal weights over the vanishing set).
template <typename T>
__device__ __forceinline__ T weno5(T v0, T v1, T v2, T v3, T v4)
{
    const T kTiny = sizeof(T) == 8 ? T(1e-150) : T(1e-18);
    const T c1 = v0 * T(1.0 / 3.0) - v1 * T(7.0 / 6.0) + v2 * T(11.0 / 6.0);
    const T c2 = -v1 * T(1.0 / 6.0) + v2 * T(5.0 / 6.0) + v3 * T(1.0 / 3.0);
    const T c3 = v2 * T(1.0 / 3.0) + v3 * T(5.0 / 6.0) - v4 * T(1.0 / 6.0);
    T a = v0 - T(2) * v1 + v2, b = v0 - T(4) * v1 + T(3) * v2;
    const T s1 = T(13.0 / 12.0) * a * a + T(0.25) * b * b;
    a = v1 - T(2) * v2 + v3;
    b = v1 - v3;
    const T s2 = T(13.0 / 12.0) * a * a + T(0.25) * b * b;
    a = v2 - T(2) * v3 + v4;
    b = T(3) * v2 - T(4) * v3 + v4;
    const T s3 = T(13.0 / 12.0) * a * a + T(0.25) * b * b;
    const T smax = fmax(s1, fmax(s2, s3));
    T w1, w2, w3;
    if (smax == T(0)) {
        w1 = T(0.1); w2 = T(0.6); w3 = T(0.3);
    } else {
        const T inv = T(1) / smax;
        const T r1 = s1 * inv, r2 = s2 * inv, r3 = s3 * inv;
        const bool z1 = r1 < kTiny, z2 = r2 < kTiny, z3 = r3 < kTiny;
        if (z1 | z2 | z3) {
            w1 = z1 ? T(0.1) : T(0); w2 = z2 ? T(0.6) : T(0); w3 = z3 ? T(0.3) : T(0);
        } else {
            w1 = T(0.1) / (r1 * r1); w2 = T(0.6) / (r2 * r2); w3 = T(0.3) / (r3 * r3);
        }
    }
    return (w1 * c1 + w2 * c2 + w3 * c3) / (w1 + w2 + w3);
}

template <typename T>
__device__ __forceinline__ T ld(const void* p, int i) { return static_cast<const T*>(p)[i]; }

// Block-wide FP64 sum (all threads get the result); deterministic order.
__device__ double block_sum(double v, double* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s += red[i];
    __syncthreads();
    return s;
}

// ----------------------------------------------------------------------------
// stage_kernel<T, V, STAGE>: STAGE 1..3 are the RK stages; STAGE 0 only
// analyses F_in (moments and wall fluxes) without writing F.
// ----------------------------------------------------------------------------
template <typename T, int V, int STAGE>
__global__ void __launch_bounds__(kThreads)
stage_kernel(const InstDev* __restrict__ insts, const Tile* __restrict__ tiles)
{
    typedef typename Acc<T>::type A;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Tile tile = tiles[blockIdx.x];
    const InstDev& I = insts[tile.inst];
    if (*I.active == 0) return;

    const int Nz = I.Nz, Q = I.Q, Qx = I.Qx, Qy = I.Qy, Qz = I.Qz, QxQy = I.QxQy;
    const int z0 = tile.z0, zn = tile.zn;            // cells z0 .. z0+zn-1 (0-based)
    const int KC = kThreads * V;
    const int k0 = tile.chunk * KC;
    const int kend = min(Q, k0 + KC);
    const int zm_lo = k0 / QxQy, zm_hi = (kend - 1) / QxQy, nzm = zm_hi - zm_lo + 1;
    const int RS = kRecHead + Qx + Qy + nzm;         // smem record stride
    const int nwarp = kThreads / 32, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // shared memory: per-warp moment partials [zn][nwarp][kNMom] (double), then
    // the cell records [zn][RS] (T)
    double* red = reinterpret_cast<double*>(smem_raw);
    T* recs = reinterpret_cast<T*>(red + (size_t)zn * nwarp * kNMom);
    __shared__ double wall_red[8];

    const T* Fin = static_cast<const T*>(STAGE == 0 ? I.F0 : STAGE == 1 ? I.F0 : STAGE == 2 ? I.F1 : I.F2);
    T* Fout = static_cast<T*>(STAGE == 1 ? I.F1 : STAGE == 2 ? I.F2 : I.F0);
    const T* F0 = static_cast<const T*>(I.F0);

    if (STAGE > 0) {
        const T* R = static_cast<const T*>(I.rec);
        for (int e = threadIdx.x; e < zn * RS; e += kThreads) {
            const int c = e / RS, r = e - c * RS;
            const int gr = r < kRecHead + Qx + Qy ? r : r + zm_lo;  // skip unused Gz rows
            recs[e] = R[(size_t)(z0 + c) * I.rec_stride + gr];
        }
        __syncthreads();
    }

    // per-velocity constants
    int kk[V], ii[V], jj[V], zz[V];
    T px[V], py[V], pz[V], wk[V];
    bool up[V], ok[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int k = k0 + threadIdx.x + v * kThreads;
        ok[v] = k < kend;
        const int kc = ok[v] ? k : kend - 1;
        kk[v] = kc;
        jj[v] = kc % Qy;
        ii[v] = (kc / Qy) % Qx;
        zz[v] = kc / QxQy;
        const int sg = zz[v] >= Qz, m = zz[v] - sg * Qz;
        px[v] = ld<T>(I.px, ii[v]);
        py[v] = ld<T>(I.py, jj[v]);
        const T x = ld<T>(I.xi, m);
        pz[v] = sg ? -x : x;
        up[v] = !sg;
        wk[v] = ld<T>(I.wx, ii[v]) * ld<T>(I.wy, jj[v]) * ld<T>(I.wz, m);
    }

    // ghost values next to the walls (only needed if the window reaches them)
    T gb[V][3], gt[V][3];
    const bool near_bot = z0 < 3, near_top = z0 + zn + 3 > Nz;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const size_t k = kk[v];
        if (near_bot) {
            if (up[v]) {  // incoming at the bottom wall
                const T g = T(I.nw[0]) * ld<T>(I.gwx_bot, ii[v]) * ld<T>(I.gwy, jj[v]) * ld<T>(I.gwz, zz[v]);
                gb[v][0] = gb[v][1] = gb[v][2] = g;
            } else {      // outgoing: quadratic extrapolation of the Appendix
                const T f1 = Fin[k], f2 = Fin[(size_t)Q + k], f3 = Fin[2 * (size_t)Q + k];
                const T g0 = T(I.ext_bot[0][0]) * f1 + T(I.ext_bot[0][1]) * f2 + T(I.ext_bot[0][2]) * f3;
                const T g1 = T(I.ext_bot[1][0]) * g0 + T(I.ext_bot[1][1]) * f1 + T(I.ext_bot[1][2]) * f2;
                gb[v][0] = g0; gb[v][1] = g1; gb[v][2] = g1;  // cell -2 is never read for p_z < 0
            }
        }
        if (near_top) {
            if (!up[v]) {
                const T g = T(I.nw[1]) * ld<T>(I.gwx_top, ii[v]) * ld<T>(I.gwy, jj[v]) * ld<T>(I.gwz, zz[v]);
                gt[v][0] = gt[v][1] = gt[v][2] = g;
            } else {
                const T f1 = Fin[(size_t)(Nz - 1) * Q + k], f2 = Fin[(size_t)(Nz - 2) * Q + k],
                        f3 = Fin[(size_t)(Nz - 3) * Q + k];
                const T g0 = T(I.ext_top[0][0]) * f1 + T(I.ext_top[0][1]) * f2 + T(I.ext_top[0][2]) * f3;
                const T g1 = T(I.ext_top[1][0]) * g0 + T(I.ext_top[1][1]) * f1 + T(I.ext_top[1][2]) * f2;
                gt[v][0] = g0; gt[v][1] = g1; gt[v][2] = g1;  // cell Nz+3 is never read for p_z > 0
            }
        }
    }

    auto fetch = [&](int v, int s) -> T {  // F at cell s (0-based; ghosts outside 0..Nz-1)
        if (s < 0) return gb[v][-1 - s];
        if (s >= Nz) return gt[v][s - Nz];
        return Fin[(size_t)s * Q + kk[v]];
    };

    // window F(s-3 .. s+2) and the flux through s - 1/2
    T w[V][6], flm[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
#pragma unroll
        for (int d = 0; d < 6; ++d) w[v][d] = fetch(v, z0 - 3 + d);
        flm[v] = pz[v] * (up[v] ? weno5<T>(w[v][0], w[v][1], w[v][2], w[v][3], w[v][4])
                                : weno5<T>(w[v][5], w[v][4], w[v][3], w[v][2], w[v][1]));
    }

    T first[V][3], last[V][3];  // outputs of the first / last three cells (wall fluxes)
    const T dt = T(I.dt);
    for (int c = 0; c < zn; ++c) {
        const int s = z0 + c;
        T n_ = 0, ux = 0, uy = 0, uz = 0, i5T = 0, qx = 0, qy = 0, qz = 0, itau = 0, cS = 0, idz = 0;
        const T* rc = recs + (size_t)c * RS;
        if (STAGE > 0) {
            ux = rc[R_UX]; uy = rc[R_UY]; uz = rc[R_UZ];
            qx = rc[R_QX]; qy = rc[R_QY]; qz = rc[R_QZ];
            itau = rc[R_ITAU]; cS = rc[R_CS]; i5T = rc[R_I5T];
            idz = ld<T>(I.inv_dz, s);
            (void)n_;
        }
        A acc[kNMom];
#pragma unroll
        for (int a = 0; a < kNMom; ++a) acc[a] = A(0);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const T wn = fetch(v, s + 3);
            T out = w[v][3];
            if (STAGE > 0) {
                const T flp = pz[v] * (up[v] ? weno5<T>(w[v][1], w[v][2], w[v][3], w[v][4], w[v][5])
                                             : weno5<T>(wn, w[v][5], w[v][4], w[v][3], w[v][2]));
                const T f = w[v][3];
                // Shakhov target n Gx Gy Gz (1 + S), S = cS (xi^2/(5T) - 1) xi.q
                const T ex = px[v] - ux, ey = py[v] - uy, ez = pz[v] - uz;
                const T xi2 = ex * ex + ey * ey + ez * ez;
                const T xq = ex * qx + ey * qy + ez * qz;
                const T S = cS * (xi2 * i5T - T(1)) * xq;
                const T geq = rc[kRecHead + ii[v]] * rc[kRecHead + Qx + jj[v]] *
                              rc[kRecHead + Qx + Qy + zz[v] - zm_lo];
                const T Lv = -(flp - flm[v]) * idz - (f - geq * (T(1) + S)) * itau;
                const T f1 = f + dt * Lv;
                if (STAGE == 1) out = f1;
                else if (STAGE == 2) out = T(0.75) * F0[(size_t)s * Q + kk[v]] + T(0.25) * f1;
                else out = T(1.0 / 3.0) * F0[(size_t)s * Q + kk[v]] + T(2.0 / 3.0) * f1;
                if (ok[v]) Fout[(size_t)s * Q + kk[v]] = out;
                flm[v] = flp;
            }
            if (c < 3) first[v][c] = out;
            last[v][0] = last[v][1]; last[v][1] = last[v][2]; last[v][2] = out;
#pragma unroll
            for (int d = 0; d < 5; ++d) w[v][d] = w[v][d + 1];
            w[v][5] = wn;
            // raw moments of the output: sum w f psi(p)
            if (ok[v]) {
                const A g = A(wk[v]) * A(out);
                const A X = A(px[v]), Y = A(py[v]), Z = A(pz[v]);
                const A p2 = X * X + Y * Y + Z * Z;
                acc[0] += g;
                acc[1] += g * X; acc[2] += g * Y; acc[3] += g * Z;
                acc[4] += g * X * X; acc[5] += g * Y * Y; acc[6] += g * Z * Z;
                acc[7] += g * X * Y; acc[8] += g * X * Z; acc[9] += g * Y * Z;
                acc[10] += g * p2 * X; acc[11] += g * p2 * Y; acc[12] += g * p2 * Z;
            }
        }
#pragma unroll
        for (int a = 0; a < kNMom; ++a) {
            A x = acc[a];
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) red[((size_t)c * nwarp + warp) * kNMom + a] = double(x);
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < zn * kNMom; e += kThreads) {
        const int c = e / kNMom, a = e - c * kNMom;
        double s = 0.0;
        for (int q = 0; q < nwarp; ++q) s += red[((size_t)c * nwarp + q) * kNMom + a];
        I.partial[((size_t)tile.chunk * Nz + z0 + c) * kNMom + a] = s;
    }

    // outgoing WENO flux of F_out through the wall interfaces (for n_w)
    if (z0 == 0) {  // bottom: p_z < 0 leaves through s = -1/2
        double fl = 0.0;
#pragma unroll
        for (int v = 0; v < V; ++v)
            if (ok[v] && !up[v]) {
                const T f1 = first[v][0], f2 = first[v][1], f3 = first[v][2];
                const T g0 = T(I.ext_bot[0][0]) * f1 + T(I.ext_bot[0][1]) * f2 + T(I.ext_bot[0][2]) * f3;
                const T g1 = T(I.ext_bot[1][0]) * g0 + T(I.ext_bot[1][1]) * f1 + T(I.ext_bot[1][2]) * f2;
                fl += double(wk[v]) * double(pz[v] * weno5<T>(f3, f2, f1, g0, g1));
            }
        fl = block_sum(fl, wall_red);
        if (threadIdx.x == 0) I.flux_part[tile.chunk * 2 + 0] = fl;
    }
    if (z0 + zn == Nz) {  // top: p_z > 0 leaves through s = Nz - 1/2
        double fl = 0.0;
#pragma unroll
        for (int v = 0; v < V; ++v)
            if (ok[v] && up[v]) {
                const T f1 = last[v][2], f2 = last[v][1], f3 = last[v][0];
                const T g0 = T(I.ext_top[0][0]) * f1 + T(I.ext_top[0][1]) * f2 + T(I.ext_top[0][2]) * f3;
                const T g1 = T(I.ext_top[1][0]) * g0 + T(I.ext_top[1][1]) * f1 + T(I.ext_top[1][2]) * f2;
                fl += double(wk[v]) * double(pz[v] * weno5<T>(f3, f2, f1, g0, g1));
            }
        fl = block_sum(fl, wall_red);
        if (threadIdx.x == 0) I.flux_part[tile.chunk * 2 + 1] = fl;
    }
}

// ----------------------------------------------------------------------------
// Cell record: scalars and the per-axis factors of the truncated Hermite
// equilibrium (Sec. III, Eqs. fyz, Fmn_def) of a macroscopic state.  Called by
// the whole CTA; thread 0 has set sc[] (n, u, T, q, 1/tau, ...) beforehand.
// ----------------------------------------------------------------------------
template <typename T>
__device__ void write_record(const InstDev& I, int cell, const double* sc, double (*coef)[kMaxN + 1])
{
    T* rec = static_cast<T*>(I.rec) + (size_t)cell * I.rec_stride;
    const int t = threadIdx.x;
    if (t < kRecHead) rec[t] = T(sc[t]);
    const int Qx = I.Qx, Qy = I.Qy, Qz = I.Qz;
    for (int e = t; e < Qx + Qy + 2 * Qz; e += blockDim.x) {
        double g = 0.0;
        if (e < Qx) {
            for (int l = 0; l <= I.Nx; ++l) g += coef[0][l] * I.Hx[e * (I.Nx + 1) + l];
            g *= sc[R_N];
        } else if (e < Qx + Qy) {
            const int j = e - Qx;
            for (int l = 0; l <= I.Ny; ++l) g += coef[1][l] * I.Hy[j * (I.Ny + 1) + l];
        } else {
            const int zm = e - Qx - Qy, sg = zm >= Qz, m = zm - sg * Qz;
            for (int l = 0; l <= I.Nzq; ++l) g += coef[2 + sg][l] * I.Pz[m * (I.Nzq + 1) + l];
        }
        rec[kRecHead + e] = T(g);
    }
}

// thread 0: scalars and expansion coefficients of (n, u, T, q); returns false
// for a non-finite or non-positive state (then a neutral state is used)
__device__ bool macro_to_coeffs(const InstDev& I, double n, const double* u, double T_, const double* q,
                                double* sc, double (*coef)[kMaxN + 1])
{
    bool bad = !(n > 0.0) || !(T_ > 0.0) || !isfinite(n) || !isfinite(T_);
    for (int a = 0; a < 3; ++a) bad |= !isfinite(u[a]) || !isfinite(q[a]);
    const double nn = bad ? 1.0 : n, Tc = bad ? 1.0 : T_;
    const double u0 = bad ? 0.0 : u[0], u1 = bad ? 0.0 : u[1], u2 = bad ? 0.0 : u[2];
    full_coeffs(u0, Tc, I.Nx, coef[0]);
    full_coeffs(u1, Tc, I.Ny, coef[1]);
    half_coeffs(u2, Tc, I.Nzq, I.alpha, I.beta, coef[2]);
    half_coeffs(-u2, Tc, I.Nzq, I.alpha, I.beta, coef[3]);
    const double tau = relax_time(I.visc_law, I.Kn, I.visc_param, nn, Tc);
    sc[R_N] = nn; sc[R_UX] = u0; sc[R_UY] = u1; sc[R_UZ] = u2; sc[R_T] = Tc;
    sc[R_QX] = bad ? 0.0 : q[0]; sc[R_QY] = bad ? 0.0 : q[1]; sc[R_QZ] = bad ? 0.0 : q[2];
    sc[R_ITAU] = 1.0 / tau;
    sc[R_CS] = (1.0 - I.Pr) / (nn * Tc * Tc);
    sc[R_I5T] = 1.0 / (5.0 * Tc);
    sc[11] = 0.0;
    return !bad;
}

// ----------------------------------------------------------------------------
// finalize_cells<T>: moments -> macroscopic state -> cell record
// ----------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) finalize_cells(const InstDev* __restrict__ insts)
{
    const InstDev& I = insts[blockIdx.y];
    const int cell = blockIdx.x, Nz = I.Nz;
    if (cell >= Nz || *I.active == 0) return;
    __shared__ double mom[kNMom];
    __shared__ double coef[4][kMaxN + 1];
    __shared__ double sc[kRecHead];
    const int t = threadIdx.x;
    if (t < kNMom) {
        double s = 0.0;
        for (int c = 0; c < I.nchunks; ++c) s += I.partial[((size_t)c * Nz + cell) * kNMom + t];
        mom[t] = s;
    }
    __syncthreads();
    if (t == 0) {
        const double n = mom[0];
        const double u[3] = {mom[1] / n, mom[2] / n, mom[3] / n};
        // central second moments P_ab = sum p_a p_b f - n u_a u_b
        const double Pxx = mom[4] - n * u[0] * u[0], Pyy = mom[5] - n * u[1] * u[1];
        const double Pzz = mom[6] - n * u[2] * u[2], Pxy = mom[7] - n * u[0] * u[1];
        const double Pxz = mom[8] - n * u[0] * u[2], Pyz = mom[9] - n * u[1] * u[2];
        const double T_ = (Pxx + Pyy + Pzz) / (3.0 * n);
        // q_a = 1/2 sum |xi|^2 xi_a f with xi = p - u, expanded in raw moments
        const double M2[3][3] = {{mom[4], mom[7], mom[8]}, {mom[7], mom[5], mom[9]}, {mom[8], mom[9], mom[6]}};
        const double tr = mom[4] + mom[5] + mom[6];
        const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const double um = u[0] * mom[1] + u[1] * mom[2] + u[2] * mom[3];
        double q[3];
        for (int a = 0; a < 3; ++a) {
            const double uM2 = u[0] * M2[0][a] + u[1] * M2[1][a] + u[2] * M2[2][a];
            q[a] = 0.5 * (mom[10 + a] - u[a] * tr - 2.0 * uM2 + 2.0 * u[a] * um + uu * mom[1 + a] -
                          uu * u[a] * n);
        }
        const double vals[14] = {n, u[0], u[1], u[2], T_, q[0], q[1], q[2], Pxx, Pyy, Pzz, Pxy, Pxz, Pyz};
        bool bad = false;
        for (int a = 0; a < 14; ++a) {
            I.prof[(size_t)a * Nz + cell] = vals[a];
            bad |= !isfinite(vals[a]);
        }
        I.Wnew[cell] = n;
        I.Wnew[Nz + cell] = u[0];
        I.Wnew[2 * Nz + cell] = T_;
        bad |= !macro_to_coeffs(I, n, u, T_, q, sc, coef);
        if (bad) atomicOr(I.status, 1);
    }
    __syncthreads();
    write_record<T>(I, cell, sc, coef);
}

// records from given macroscopic profiles macro[8][Nz] = n, ux, uy, uz, T, qx, qy, qz
template <typename T>
__global__ void __launch_bounds__(128) records_from_macro(const InstDev* __restrict__ insts, int inst,
                                                         const double* __restrict__ macro)
{
    const InstDev& I = insts[inst];
    const int cell = blockIdx.x, Nz = I.Nz;
    __shared__ double coef[4][kMaxN + 1];
    __shared__ double sc[kRecHead];
    if (threadIdx.x == 0) {
        const double u[3] = {macro[Nz + cell], macro[2 * Nz + cell], macro[3 * Nz + cell]};
        const double q[3] = {macro[5 * Nz + cell], macro[6 * Nz + cell], macro[7 * Nz + cell]};
        if (!macro_to_coeffs(I, macro[cell], u, macro[4 * Nz + cell], q, sc, coef)) atomicOr(I.status, 1);
    }
    __syncthreads();
    write_record<T>(I, cell, sc, coef);
}

// ----------------------------------------------------------------------------
// finalize_inst: wall densities; after stage 3 the residual and retirement
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256) finalize_inst(const InstDev* __restrict__ insts, int stage)
{
    const InstDev& I = insts[blockIdx.x];
    if (*I.active == 0) return;
    __shared__ double red[8];
    const int t = threadIdx.x, Nz = I.Nz;
    double fb = 0.0, ft = 0.0;
    for (int c = t; c < I.nchunks; c += blockDim.x) {
        fb += I.flux_part[2 * c];
        ft += I.flux_part[2 * c + 1];
    }
    fb = block_sum(fb, red);
    ft = block_sum(ft, red);
    if (t == 0) {
        I.nw[0] = -fb / I.Dbot;
        I.nw[1] = -ft / I.Dtop;
        if (!isfinite(I.nw[0]) || !isfinite(I.nw[1])) atomicOr(I.status, 1);
    }
    if (stage == 3) {
        double R = 0.0;
        for (int a = 0; a < 3; ++a) {
            double d = 0.0, o = 0.0;
            for (int s = t; s < Nz; s += blockDim.x) {
                const double e = I.Wnew[a * Nz + s] - I.Wold[a * Nz + s];
                d += e * e;
                o += I.Wold[a * Nz + s] * I.Wold[a * Nz + s];
            }
            d = block_sum(d, red);
            o = block_sum(o, red);
            R = fmax(R, sqrt(d) / fmax(sqrt(o), 1e-30));
        }
        __syncthreads();
        for (int e = t; e < 3 * Nz; e += blockDim.x) I.Wold[e] = I.Wnew[e];
        if (t == 0) {
            *I.res = R;
            *I.steps += 1;
            if (!(R == R)) atomicOr(I.status, 1);
            if (I.tol > 0.0 && R < I.tol) *I.active = 0;
        }
    } else if (stage == 0) {
        for (int e = t; e < 3 * Nz; e += blockDim.x) I.Wold[e] = I.Wnew[e];
    }
}

// ---- seed a cell from macroscopic values: n Gx Gy Gz (1 + S) --------------
template <typename T>
__global__ void __launch_bounds__(128) seed_cells(const InstDev* __restrict__ insts, int inst, int fbuf)
{
    const InstDev& I = insts[inst];
    const int cell = blockIdx.x;
    const T* rc = static_cast<const T*>(I.rec) + (size_t)cell * I.rec_stride;
    T* F = static_cast<T*>(fbuf == 0 ? I.F0 : fbuf == 1 ? I.F1 : I.F2) + (size_t)cell * I.Q;
    for (int k = threadIdx.x; k < I.Q; k += blockDim.x) {
        const int j = k % I.Qy, i = (k / I.Qy) % I.Qx, zm = k / I.QxQy;
        const int sg = zm >= I.Qz, m = zm - sg * I.Qz;
        const T x = ld<T>(I.xi, m);
        const T ex = ld<T>(I.px, i) - rc[R_UX], ey = ld<T>(I.py, j) - rc[R_UY], ez = (sg ? -x : x) - rc[R_UZ];
        const T S = rc[R_CS] * ((ex * ex + ey * ey + ez * ez) * rc[R_I5T] - T(1)) *
                    (ex * rc[R_QX] + ey * rc[R_QY] + ez * rc[R_QZ]);
        F[k] = rc[kRecHead + i] * rc[kRecHead + I.Qx + j] * rc[kRecHead + I.Qx + I.Qy + zm] * (T(1) + S);
    }
}

// ---- host launchers ---------------------------------------------------------
template <typename T, int V, int STAGE>
static cudaError_t launch_stage_t(const InstDev* d_inst, const Tile* d_tiles, int ntiles, size_t smem,
                                  cudaStream_t st)
{
    auto kfn = stage_kernel<T, V, STAGE>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kfn<<<ntiles, kThreads, smem, st>>>(d_inst, d_tiles);
    return cudaGetLastError();
}

template <typename T, int V>
static cudaError_t launch_stage_v(int stage, const InstDev* d, const Tile* t, int n, size_t smem,
                                  cudaStream_t st)
{
    switch (stage) {
        case 0: return launch_stage_t<T, V, 0>(d, t, n, smem, st);
        case 1: return launch_stage_t<T, V, 1>(d, t, n, smem, st);
        case 2: return launch_stage_t<T, V, 2>(d, t, n, smem, st);
        default: return launch_stage_t<T, V, 3>(d, t, n, smem, st);
    }
}

cudaError_t launch_stage(int fp32, int V, int stage, const InstDev* d_inst, const Tile* d_tiles,
                         int ntiles, size_t smem, cudaStream_t st)
{
    if (fp32) {
        if (V == 1) return launch_stage_v<float, 1>(stage, d_inst, d_tiles, ntiles, smem, st);
        if (V == 2) return launch_stage_v<float, 2>(stage, d_inst, d_tiles, ntiles, smem, st);
        return launch_stage_v<float, 4>(stage, d_inst, d_tiles, ntiles, smem, st);
    }
    if (V == 1) return launch_stage_v<double, 1>(stage, d_inst, d_tiles, ntiles, smem, st);
    if (V == 2) return launch_stage_v<double, 2>(stage, d_inst, d_tiles, ntiles, smem, st);
    return launch_stage_v<double, 4>(stage, d_inst, d_tiles, ntiles, smem, st);
}

cudaError_t launch_finalize(int fp32, int stage, const InstDev* d_inst, int ninst, int maxNz,
                            cudaStream_t st)
{
    dim3 g(maxNz, ninst);
    if (fp32) finalize_cells<float><<<g, 128, 0, st>>>(d_inst);
    else finalize_cells<double><<<g, 128, 0, st>>>(d_inst);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    finalize_inst<<<ninst, 256, 0, st>>>(d_inst, stage);
    return cudaGetLastError();
}

cudaError_t launch_seed(int fp32, const InstDev* d_inst, int inst, int Nz, const double* d_macro,
                        cudaStream_t st)
{
    if (fp32) records_from_macro<float><<<Nz, 128, 0, st>>>(d_inst, inst, d_macro);
    else records_from_macro<double><<<Nz, 128, 0, st>>>(d_inst, inst, d_macro);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (fp32) seed_cells<float><<<Nz, 128, 0, st>>>(d_inst, inst, 0);
    else seed_cells<double><<<Nz, 128, 0, st>>>(d_inst, inst, 0);
    return cudaGetLastError();
}

}  // namespace lbs
