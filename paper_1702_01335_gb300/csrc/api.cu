// C ABI of the solver (include/lbs.h): host set-up of each Couette instance
// (velocity set, Hermite bases, grid, wall equilibria, time step), one device
// memory pool per handle, and the launch sequence of a time step.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbs.h"
#include "lbs_internal.h"

namespace lbs {
cudaError_t launch_stage(int fp32, int red, int V, int stage, const InstDev* d_inst, const Tile* d_tiles,
                         int ntiles, size_t smem, int fuse, int ninst, int maxNz, int fin_warp, int nb,
                         cudaStream_t st);
cudaError_t launch_stage_only(int fp32, int red, int V, int stage, const InstDev* d_inst, const Tile* d_tiles,
                              int ntiles, size_t smem, int fuse, cudaStream_t st);
cudaError_t launch_finalize(int fp32, int stage, const InstDev* d_inst, int ninst, int maxNz, int fin_warp,
                            int nb, cudaStream_t st);
cudaError_t launch_seed(int fp32, const InstDev* d_inst, int inst, int Nz, const double* d_macro,
                        cudaStream_t st);
cudaError_t launch_seed_free_molecular(int fp32, const InstDev* d_inst, int inst, int Nz, cudaStream_t st);
cudaError_t launch_gather_moments(const InstDev* d_inst, int ninst, const double* prof_all, double* out,
                                  cudaStream_t st);
size_t stage_smem_bytes(int fp32, int V, int zn, int G, int stage, int rstride);
}  // namespace lbs

using namespace lbs;

static thread_local std::string g_err;

static lbs_status fail(lbs_status s, const std::string& m)
{
    g_err = m;
    return s;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(LBS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

namespace {

struct InstHost {
    lbs_instance_desc d;
    int Nz, Q, Qx, Qy, Qz, Nx, Ny, Nzq, nchunks, nchh, nzm_max, nzt;
    bool reduced;  // the phi / chi model (lbs_orders.Qy = 0)
    double dt;
    std::vector<double> xc, xf;  // cell centres (s = -3..Nz+2, 0-based), interfaces
};

constexpr size_t kSmemBudget = 200 * 1024;  // dynamic shared memory of a stage CTA

struct Pool {  // bump allocator over one device allocation
    size_t bytes = 0;
    size_t take(size_t n)
    {
        size_t o = (bytes + 255) & ~size_t(255);
        bytes = o + n;
        return o;
    }
};

}  // namespace

struct lbs_solver {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int fp32 = 0, esize = 8, V = 1, ZT = 16, fuse = 1, ninst = 0, maxNz = 0, nb = 0;
    int fin_mode = 0, fin_warp = 0;  // finalisation: 0 auto, 1 thread per cell, 2 warp per cell
    int reduced = 0;                 // the batch runs the phi / chi model (all instances alike)
    std::vector<InstHost> ih;
    std::vector<InstDev> idev;
    InstDev* d_inst = nullptr;
    Tile* d_tiles = nullptr;
    int ntiles = 0;
    size_t max_tiles = 0;
    size_t smem = 0;
    unsigned char* pool = nullptr;
    double* d_macro = nullptr;  // [8][maxNz] staging for warm starts
    // every instance's profiles ([14][Nz] each) and status word, back to back in
    // instance order: whole-batch reads are one copy each
    double* prof_all = nullptr;
    size_t prof_all_n = 0;
    double* mom_all = nullptr;  // [8][Nz] per instance: lbs_moments' rows, gathered for one copy
    int* status_all = nullptr;
    int* cur_all = nullptr;  // per instance: which of F0 / F1 holds the state
    cudaGraphExec_t gexec = nullptr;
    int gsteps = 0;
    // split stepping (fuse = 2): instances [0, nA) on stream, [nA, ninst) on stream2
    int nA = 0, ntilesA = 0;
    // first tile of each instance in the full tile list (ninst + 1 entries), and whether
    // the list on the device is the full one (run_to_steady launches a compacted list)
    std::vector<int> tile_first;
    bool tiles_full = true;
    cudaStream_t stream2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int device = 0;
};

int lbs::handle_view(void* hv, int inst, HandleView* out)
{
    lbs_solver* h = static_cast<lbs_solver*>(hv);
    if (!h || !out || inst < 0 || inst >= h->ninst) return fail(LBS_ERR_ARG, "invalid handle or instance index");
    out->d_inst = h->d_inst;
    out->inst = h->idev[inst];
    out->fp32 = h->fp32;
    out->device = h->device;
    out->stream = static_cast<void*>(h->stream);
    return LBS_OK;
}

int lbs::record_error(int status, const char* msg) { return fail(static_cast<lbs_status>(status), msg); }

// ---------------------------------------------------------------- set-up ----
static lbs_status validate(const lbs_instance_desc& d)
{
    const lbs_orders& o = d.orders;
    if (o.Qx < 1 || o.Qx > kMaxQ1D || o.Qy < 0 || o.Qy > kMaxQ1D || o.Qz_half < 1 ||
        o.Qz_half > kMaxQ1D)
        return fail(LBS_ERR_ARG, "velocity orders must lie in 1..100 (Qy = 0: the reduced model)");
    if (o.N_eq < 0 || o.N_eq > kMaxN) return fail(LBS_ERR_ARG, "N_eq must lie in 0..8");
    if ((long)2 * o.Qx * std::max(o.Qy, 2) * o.Qz_half > 32768)
        return fail(LBS_ERR_ARG, "Q = 2 Qx Qy Qz_half exceeds 32768");
    if (d.grid.Nz < 6 || d.grid.Nz > 4096) return fail(LBS_ERR_ARG, "Nz must lie in 6..4096");
    if (!(d.grid.A >= 0.0 && d.grid.A < 1.0)) return fail(LBS_ERR_ARG, "grid stretching A must lie in [0, 1)");
    if (d.grid.half != 0 && d.grid.half != 1) return fail(LBS_ERR_ARG, "grid.half must be 0 or 1");
    if (!(d.Kn > 0.0) || !(d.T_w > 0.0) || !(d.Pr > 0.0) || !std::isfinite(d.u_w))
        return fail(LBS_ERR_ARG, "Kn, T_w and Pr must be positive and u_w finite");
    if (d.visc.law != LBS_VISC_POWER && d.visc.law != LBS_VISC_SUTHERLAND)
        return fail(LBS_ERR_ARG, "unknown viscosity law");
    if (d.visc.law == LBS_VISC_SUTHERLAND && !(d.visc.omega_or_S > 0.0))
        return fail(LBS_ERR_ARG, "Sutherland constant must be positive");
    if (!(d.dt > 0.0) && !(d.cfl > 0.0)) return fail(LBS_ERR_ARG, "either dt or cfl must be positive");
    return LBS_OK;
}

// cell centre / interface positions; Eqs. (stretch), (etas) on the full channel
static double xpos(int Nz, double A, double s)  // s in cell units from the bottom wall
{
    if (A == 0.0) return -0.5 + s / Nz;
    const double E = std::atanh(A);
    return std::tanh(-E + s * 2.0 * E / Nz) / (2.0 * A);
}

static void lagrange3(double x, double a, double b, double c, double* w)
{
    w[0] = (x - b) * (x - c) / ((a - b) * (a - c));
    w[1] = (x - a) * (x - c) / ((b - a) * (b - c));
    w[2] = (x - a) * (x - b) / ((c - a) * (c - b));
}

template <typename T>
static void put(std::vector<unsigned char>& host, size_t off, const std::vector<double>& v)
{
    T* p = reinterpret_cast<T*>(host.data() + off);
    for (size_t i = 0; i < v.size(); ++i) p[i] = T(v[i]);
}

// FP32 (hi, lo) pairs of FP64 values: hi the nearest float, lo the nearest float to
// the remainder
static void put_pairs(std::vector<unsigned char>& host, size_t off, const std::vector<double>& v)
{
    float* p = reinterpret_cast<float*>(host.data() + off);
    for (size_t i = 0; i < v.size(); ++i) {
        const float hi = float(v[i]);
        p[2 * i] = hi;
        p[2 * i + 1] = float(v[i] - double(hi));
    }
}

template <typename T>
static std::vector<double> rounded(const std::vector<double>& v)
{
    std::vector<double> r(v.size());
    for (size_t i = 0; i < v.size(); ++i) r[i] = double(T(v[i]));
    return r;
}

static void build_tiles(lbs_solver* h, std::vector<Tile>& tiles)
{
    tiles.clear();
    const int KC = kThreads * h->V;
    size_t smem = 0;
    for (int b = 0; b < h->ninst; ++b) {
        InstHost& I = h->ih[b];
        // chunks never straddle p_z = 0: nchh chunks per half range of Q / 2 velocities,
        // so that each CTA marches its velocities in their common upwind direction
        const int Qh = I.Q / 2;
        I.nchh = (Qh + KC - 1) / KC;
        I.nchunks = 2 * I.nchh;
        int nzm_max = 0;
        for (int c = 0; c < I.nchunks; ++c) {
            const int sg = c / I.nchh, k0 = sg * Qh + (c - sg * I.nchh) * KC;
            const int k1 = std::min((sg + 1) * Qh, k0 + KC) - 1;
            nzm_max = std::max(nzm_max, k1 / (I.Qx * I.Qy) - k0 / (I.Qx * I.Qy) + 1);
        }
        I.nzm_max = nzm_max;
        const int G = I.Qx + I.Qy + nzm_max;
        const int rs = rec_stride_of(I.Qx, I.Qy, I.Qz);
        // z-tiles of about ZT cells, at least 3 cells each, within the shared-memory budget
        int zt = std::max(3, std::min(h->ZT, kMaxZT));
        while (zt > 3 && stage_smem_bytes(h->fp32, h->V, zt, G, 3, rs) > kSmemBudget) --zt;
        int nzt = std::min((I.Nz + zt - 1) / zt, I.Nz / 3);
        nzt = std::max(nzt, 1);
        const int base = I.Nz / nzt, rem = I.Nz % nzt;
        const int zmax = base + (rem ? 1 : 0);
        I.nzt = nzt;
        smem = std::max(smem, stage_smem_bytes(h->fp32, h->V, zmax, G, 3, rs));
        for (int c = 0; c < I.nchunks; ++c) {
            int z0 = 0;
            for (int t = 0; t < nzt; ++t) {
                const int zn = base + (t < rem ? 1 : 0);
                tiles.push_back(Tile{b, z0, zn, c, t});
                z0 += zn;
            }
        }
    }
    h->smem = smem;
    h->tile_first.assign(h->ninst + 1, 0);
    for (const Tile& x : tiles) ++h->tile_first[x.inst + 1];
    for (int b = 0; b < h->ninst; ++b) h->tile_first[b + 1] += h->tile_first[b];
    // split point of the batch for fuse = 2: about half the tiles on each side
    h->nA = 0;
    h->ntilesA = 0;
    if (h->ninst >= 2) {
        size_t t = 0;
        int b = 0;
        while (b < h->ninst - 1) {
            size_t tb = 0;
            for (const Tile& x : tiles)
                if (x.inst == b) ++tb;
            if (2 * (t + tb) > tiles.size() && b > 0) break;
            t += tb;
            ++b;
        }
        h->nA = b;
        h->ntilesA = (int)t;
    }
}


// Finalisation with one warp per cell pays while the batch has at most one cell per
// warp scheduler (152 SMs x 4): each cell's FP64 chain then runs on a scheduler of
// its own, with its loads, coefficient sets and half-range tables spread over the
// lanes.  Beyond that one thread per cell keeps every lane busy (measured: 320
// cells 30 us per launch with warps vs 48 us with threads; 2048 cells 57 vs 34 us).
constexpr long kFinWarpMaxCells = 608;
static void choose_finalize(lbs_solver* h)
{
    long cells = 0;
    for (int b = 0; b < h->ninst; ++b) cells += h->ih[b].Nz;
    h->fin_warp = h->fin_mode == 2 || (h->fin_mode == 0 && cells <= kFinWarpMaxCells);
    for (int b = 0; b < h->ninst; ++b) h->idev[b].fin_warp = h->fin_warp;
}

template <typename T>
static lbs_status setup(lbs_solver* h, const lbs_instance_desc* desc)
{
    // ---- per-instance host tables
    std::vector<std::vector<double>> tabs_d;  // per instance, concatenated later
    Pool pool;
    struct Off {
        size_t Hx, Hy, Pz, Hx2, Hy2, Pz2, alpha, beta, px, py, xi, wx, wy, wz, gxt, gxb, gwy, gwz, idz;
        size_t F0, F1, F2, L0, cur, rec, partial, flux, nw, prof, Wold, Wnew, res, steps, active, status, zcount,
            icount;
    };
    std::vector<Off> off(h->ninst);
    struct Tables {
        std::vector<double> Hx, Hy, Pz, alpha, beta, px, wx, py, wy, xi, wz, gxt, gxb, gwy, gwz, idz;
    };
    std::vector<Tables> tb(h->ninst);
    h->idev.assign(h->ninst, InstDev());
    std::vector<Tile> tiles;
    // first pass: sizes that do not depend on the tiling
    for (int b = 0; b < h->ninst; ++b) {
        const lbs_instance_desc& d = desc[b];
        InstHost& I = h->ih[b];
        I.d = d;
        I.Nz = d.grid.Nz;
        I.Qx = d.orders.Qx;
        I.reduced = d.orders.Qy == 0;
        I.Qy = I.reduced ? 2 : d.orders.Qy;  // reduced: j = 0 phi, j = 1 chi
        I.Qz = d.orders.Qz_half;
        I.Q = 2 * I.Qx * I.Qy * I.Qz;
        I.Nx = std::min(d.orders.N_eq, I.Qx - 1);
        I.Ny = I.reduced ? 1 : std::min(d.orders.N_eq, I.Qy - 1);
        I.Nzq = std::min(d.orders.N_eq, I.Qz - 1);
        h->maxNz = std::max(h->maxNz, I.Nz);
        h->nb = std::max(h->nb, std::max(I.Nx, std::max(I.Ny, I.Nzq)));  // the batch's largest order
    }
    build_tiles(h, tiles);
    for (int b = 0; b < h->ninst; ++b) {
        InstHost& I = h->ih[b];
        Tables& t = tb[b];
        const lbs_instance_desc& d = I.d;
        // quadratures
        t.px.resize(I.Qx); t.wx.resize(I.Qx); t.py.resize(I.Qy); t.wy.resize(I.Qy);
        t.xi.resize(I.Qz); t.wz.resize(I.Qz);
        if (gauss_rule(QUAD_FULL, I.Qx, t.px.data(), t.wx.data()) ||
            (!I.reduced && gauss_rule(QUAD_FULL, I.Qy, t.py.data(), t.wy.data())) ||
            gauss_rule(QUAD_HALF, I.Qz, t.xi.data(), t.wz.data()))
            return fail(LBS_ERR_QUADRATURE, "Gauss rule construction failed");
        if (I.reduced) {  // phi and chi on the same (p_x, p_z) node: no y node, weight 1
            t.py.assign(2, 0.0);
            t.wy.assign(2, 1.0);
        }
        for (double v : t.wz)
            if (!(v > 0.0) || !std::isfinite(v)) return fail(LBS_ERR_QUADRATURE, "non-positive half-range weight");
        recurrence(QUAD_HALF, kMaxN + 2, t.alpha, t.beta);
        t.Hx.resize(I.Qx * (I.Nx + 1)); t.Hy.resize(I.Qy * (I.Ny + 1)); t.Pz.resize(I.Qz * (I.Nzq + 1));
        hermite_basis(t.px.data(), I.Qx, I.Nx, t.Hx.data());
        if (I.reduced)  // Gy_j = a_j: the record's y coefficients are the factors (1, T)
            t.Hy = {1.0, 0.0, 0.0, 1.0};
        else
            hermite_basis(t.py.data(), I.Qy, I.Ny, t.Hy.data());
        half_basis(t.xi.data(), I.Qz, I.Nzq, t.alpha, t.beta, t.Pz.data());
        // wall equilibria per axis (n = 1, T = T_w, u = +-u_w along x, q = 0), stored as the
        // deviations of the normalised factors from 1: sum_l (c_l - r_l) basis_l with the
        // rest coefficients r (1, 0, 0, ...) on x and y, (1, 1) on the reduced y (factors
        // 1 and T), (1/2, 0, ...) on z, as the cell records hold them
        double a[kMaxN + 1], bb[kMaxN + 1];
        t.gxt.assign(I.Qx, 0.0); t.gxb.assign(I.Qx, 0.0); t.gwy.assign(I.Qy, 0.0); t.gwz.assign(2 * I.Qz, 0.0);
        full_coeffs(d.u_w, d.T_w, I.Nx, a);
        for (int i = 0; i < I.Qx; ++i)
            for (int l = 1; l <= I.Nx; ++l) t.gxt[i] += a[l] * t.Hx[i * (I.Nx + 1) + l];
        full_coeffs(-d.u_w, d.T_w, I.Nx, a);
        for (int i = 0; i < I.Qx; ++i)
            for (int l = 1; l <= I.Nx; ++l) t.gxb[i] += a[l] * t.Hx[i * (I.Nx + 1) + l];
        if (I.reduced) {  // phi_w and chi_w = T_w phi_w
            t.gwy[0] = 0.0;
            t.gwy[1] = d.T_w - 1.0;
        } else {
            full_coeffs(0.0, d.T_w, I.Ny, a);
            for (int j = 0; j < I.Qy; ++j)
                for (int l = 1; l <= I.Ny; ++l) t.gwy[j] += a[l] * t.Hy[j * (I.Ny + 1) + l];
        }
        half_coeffs(0.0, d.T_w, I.Nzq, t.alpha.data(), t.beta.data(), bb);
        bb[0] -= 0.5;  // exactly 0: erfc(0) = 1
        for (int m = 0; m < I.Qz; ++m)
            for (int l = 0; l <= I.Nzq; ++l) {
                t.gwz[m] += bb[l] * t.Pz[m * (I.Nzq + 1) + l];
                t.gwz[I.Qz + m] += bb[l] * t.Pz[m * (I.Nzq + 1) + l];
            }
        // grid: the full channel of Nz cells, or (half) cells Nz .. 2Nz-1 of the full
        // channel of 2Nz cells, whose centre line is the interface below cell 0
        const int Nz = I.Nz, half = d.grid.half, Nfull = half ? 2 * Nz : Nz, s0 = half ? Nz : 0;
        I.xc.resize(Nz + 6);
        for (int s = -3; s <= Nz + 2; ++s) I.xc[s + 3] = xpos(Nfull, d.grid.A, s0 + s + 0.5);
        I.xf.resize(Nz + 1);
        for (int s = 0; s <= Nz; ++s) I.xf[s] = xpos(Nfull, d.grid.A, s0 + s);
        if (half) I.xf[0] = 0.0;  // tanh(0) exactly, whatever the rounding of -E + Nz (2E / 2Nz)
        t.idz.resize(Nz);
        double dzmin = 1e300;
        for (int s = 0; s < Nz; ++s) {
            t.idz[s] = 1.0 / (I.xf[s + 1] - I.xf[s]);
            dzmin = std::min(dzmin, I.xf[s + 1] - I.xf[s]);
        }
        // time step
        if (d.dt > 0.0) {
            I.dt = d.dt;
        } else {
            const double pmax = *std::max_element(t.xi.begin(), t.xi.end());
            const double cap = 0.5 * relax_time(d.visc.law, d.Kn, d.visc.omega_or_S, 2.0, d.T_w);
            I.dt = std::min(d.cfl * dzmin / pmax, cap);
        }
        // device descriptor (pointers filled after allocation)
        InstDev& D = h->idev[b];
        D.Nz = Nz; D.Qx = I.Qx; D.Qy = I.Qy; D.Qz = I.Qz; D.Q = I.Q; D.QxQy = I.Qx * I.Qy;
        D.Nx = I.Nx; D.Ny = I.Ny; D.Nzq = I.Nzq;
        D.nchunks = I.nchunks;
        D.nchh = I.nchh;
        D.half = half;
        D.reduced = I.reduced;
        // every row segment (row s, chunk start k0 in either half) starts on 16 bytes
        D.bulk = ((size_t)(I.Q / 2) * sizeof(T)) % 16 == 0;
        D.visc_law = d.visc.law; D.Kn = d.Kn; D.visc_param = d.visc.omega_or_S; D.Pr = d.Pr;
        D.iKn = 1.0 / d.Kn;
        D.isuth = d.visc.law == 1 ? 1.0 / (1.0 + d.visc.omega_or_S) : 0.0;
        D.dt = I.dt; D.tol = 0.0;
        D.res_uscale = std::max(std::fabs(d.u_w) * std::sqrt((double)Nz), 1e-30);
        const std::vector<double>& xc = I.xc;  // xc[s + 3]
        lagrange3(xc[Nz + 3], xc[Nz + 2], xc[Nz + 1], xc[Nz], D.ext_top[0]);
        lagrange3(xc[Nz + 4], xc[Nz + 3], xc[Nz + 2], xc[Nz + 1], D.ext_top[1]);
        lagrange3(xc[2], xc[3], xc[4], xc[5], D.ext_bot[0]);
        lagrange3(xc[1], xc[2], xc[3], xc[4], D.ext_bot[1]);
        // D = sum over incoming velocities of w p_z Gw, from the stored (rounded) tables
        // (Gw = 1 + the stored deviation on each axis)
        const std::vector<double> wx = rounded<T>(t.wx), wy = rounded<T>(t.wy), wz = rounded<T>(t.wz);
        const std::vector<double> xi = rounded<T>(t.xi), gxt = rounded<T>(t.gxt), gxb = rounded<T>(t.gxb);
        const std::vector<double> gwy = rounded<T>(t.gwy), gwz = rounded<T>(t.gwz);
        const std::vector<double> px = rounded<T>(t.px), py = rounded<T>(t.py);
        double sxt = 0, sxb = 0, sy = 0, szp = 0, szm = 0;
        for (int i = 0; i < I.Qx; ++i) { sxt += wx[i] * (1.0 + gxt[i]); sxb += wx[i] * (1.0 + gxb[i]); }
        for (int j = 0; j < I.Qy; ++j) sy += wy[j] * (1.0 + gwy[j]);
        if (I.reduced) sy = 1.0 + gwy[0];  // mass is carried by phi alone
        for (int m = 0; m < I.Qz; ++m) {
            szp += wz[m] * xi[m] * (1.0 + gwz[m]);
            szm += wz[m] * (-xi[m]) * (1.0 + gwz[I.Qz + m]);
        }
        D.Dtop = sxt * sy * szm;
        D.Dbot = sxb * sy * szp;
        // the rest state f = w: its raw moments (the kernels sum the deviations from it)
        // and its outgoing flux through each wall, over the stored nodes and weights
        for (int a2 = 0; a2 < kNMom; ++a2) D.mrest[a2] = 0.0;
        D.frest_top = D.frest_bot = 0.0;
        for (int sg = 0; sg < 2; ++sg)
            for (int m = 0; m < I.Qz; ++m)
                for (int i = 0; i < I.Qx; ++i)
                    for (int j = 0; j < I.Qy; ++j) {
                        const double w = wx[i] * wy[j] * wz[m];
                        const double X = px[i], Y = I.reduced ? 0.0 : py[j], Z = sg ? -xi[m] : xi[m];
                        if (I.reduced && j == 1) {  // chi: the p_y^2 moments only
                            D.mrest[5] += w;
                            D.mrest[10] += w * X;
                            D.mrest[12] += w * Z;
                            continue;
                        }
                        const double p2 = X * X + Y * Y + Z * Z, m1[kNMom] = {
                            1.0, X, Y, Z, X * X, Y * Y, Z * Z, X * Y, X * Z, Y * Z, p2 * X, p2 * Y, p2 * Z};
                        for (int a2 = 0; a2 < kNMom; ++a2) D.mrest[a2] += w * m1[a2];
                        if (sg) D.frest_bot += w * Z;
                        else D.frest_top += w * Z;
                    }
        if (half) D.frest_bot = 0.0;  // no wall below a half channel
        D.wait_limit = kWaitLimit;
        // memory layout
        Off& o = off[b];
        const size_t es = sizeof(T);
        o.Hx = pool.take(t.Hx.size() * 8); o.Hy = pool.take(t.Hy.size() * 8); o.Pz = pool.take(t.Pz.size() * 8);
        o.Hx2 = pool.take(t.Hx.size() * 8); o.Hy2 = pool.take(t.Hy.size() * 8); o.Pz2 = pool.take(t.Pz.size() * 8);
        o.alpha = pool.take(t.alpha.size() * 8); o.beta = pool.take(t.beta.size() * 8);
        o.px = pool.take(I.Qx * es); o.py = pool.take(I.Qy * es); o.xi = pool.take(I.Qz * es);
        o.wx = pool.take(I.Qx * es); o.wy = pool.take(I.Qy * es); o.wz = pool.take(I.Qz * es);
        o.gxt = pool.take(I.Qx * es); o.gxb = pool.take(I.Qx * es); o.gwy = pool.take(I.Qy * es);
        o.gwz = pool.take(2 * I.Qz * es); o.idz = pool.take(Nz * es);
        const size_t nf = (size_t)Nz * I.Q;
        o.F2 = pool.take(nf * es);  // F0, F1, L0: below
        o.rec = pool.take((size_t)Nz * rec_stride_of(I.Qx, I.Qy, I.Qz) * es);
        const size_t maxch = 2 * ((I.Q / 2 + kThreads - 1) / kThreads);  // chunks at V = 1, the finest tiling
        o.partial = pool.take(maxch * Nz * kNMom * 8);
        o.flux = pool.take(maxch * 2 * 8);
        o.nw = pool.take(2 * 8);  // prof: below
        o.Wold = pool.take(3 * (size_t)Nz * 8); o.Wnew = pool.take(3 * (size_t)Nz * 8);
        o.res = pool.take(8); o.steps = pool.take(8); o.active = pool.take(4);  // status: below
        o.zcount = pool.take(4 * (size_t)std::max(1, Nz / 3)); o.icount = pool.take(4);
    }
    // The two state buffers F0 and F1 of every instance back to back (one region each),
    // and likewise the FP32 rounding residuals L0, each state rounded up to 256 bytes so
    // that every one starts aligned.  Where the rounding adds nothing (states of a
    // multiple of 256 bytes, such as C2's 1 MiB), a whole-batch lbs_get_state /
    // lbs_set_state is one copy per region.  Profiles, status words and the state
    // selectors are packed.
    size_t prof_base = 0, status_base = 0, cur_base = 0;
    {
        size_t f0_total = 0, l0_total = 0, prof_total = 0;
        for (int b = 0; b < h->ninst; ++b) {
            const size_t nf = (size_t)h->ih[b].Nz * h->ih[b].Q;
            f0_total += (nf * sizeof(T) + 255) & ~size_t(255);
            if (h->fp32) l0_total += (nf * 2 + 255) & ~size_t(255);
            prof_total += 14 * (size_t)h->ih[b].Nz;
        }
        const size_t f0_base = pool.take(f0_total), f1_base = pool.take(f0_total);
        const size_t l0_base = h->fp32 ? pool.take(l0_total) : 0;
        prof_base = pool.take(prof_total * 8);
        status_base = pool.take(4 * (size_t)h->ninst);
        cur_base = pool.take(4 * (size_t)h->ninst);
        h->prof_all_n = prof_total;
        size_t fo = 0, lo = 0, po = 0;
        for (int b = 0; b < h->ninst; ++b) {
            const size_t nf = (size_t)h->ih[b].Nz * h->ih[b].Q;
            off[b].F0 = f0_base + fo;
            off[b].F1 = f1_base + fo;
            fo += (nf * sizeof(T) + 255) & ~size_t(255);
            off[b].L0 = l0_base + lo;
            if (h->fp32) lo += (nf * 2 + 255) & ~size_t(255);
            off[b].prof = prof_base + 8 * po;
            po += 14 * (size_t)h->ih[b].Nz;
            off[b].status = status_base + 4 * (size_t)b;
            off[b].cur = cur_base + 4 * (size_t)b;
        }
    }
    const size_t inst_off = pool.take(sizeof(InstDev) * h->ninst);
    size_t max_tiles = 0;  // tiles of the finest tiling (V = 1, 3-cell z-tiles)
    for (int b = 0; b < h->ninst; ++b)
        max_tiles += (size_t)(2 * ((h->ih[b].Q / 2 + kThreads - 1) / kThreads)) * std::max(1, h->ih[b].Nz / 3);
    h->max_tiles = max_tiles;
    const size_t tile_off = pool.take(sizeof(Tile) * max_tiles);
    const size_t macro_off = pool.take(8 * (size_t)h->maxNz * 8);
    const size_t mom_off = pool.take(8 * (h->prof_all_n / 14) * 8);
    void* mem = nullptr;
    CK(cudaMalloc(&mem, pool.bytes));
    h->pool = static_cast<unsigned char*>(mem);
    unsigned char* P = h->pool;
    // host image of the constant tables, descriptors and tiles; state set below
    std::vector<unsigned char> img(pool.bytes, 0);
    for (int b = 0; b < h->ninst; ++b) {
        const Off& o = off[b];
        const Tables& t = tb[b];
        const InstHost& I = h->ih[b];
        put<double>(img, o.Hx, t.Hx); put<double>(img, o.Hy, t.Hy); put<double>(img, o.Pz, t.Pz);
        put_pairs(img, o.Hx2, t.Hx); put_pairs(img, o.Hy2, t.Hy); put_pairs(img, o.Pz2, t.Pz);
        put<double>(img, o.alpha, t.alpha); put<double>(img, o.beta, t.beta);
        put<T>(img, o.px, t.px); put<T>(img, o.py, t.py); put<T>(img, o.xi, t.xi);
        put<T>(img, o.wx, t.wx); put<T>(img, o.wy, t.wy); put<T>(img, o.wz, t.wz);
        put<T>(img, o.gxt, t.gxt); put<T>(img, o.gxb, t.gxb); put<T>(img, o.gwy, t.gwy);
        put<T>(img, o.gwz, t.gwz); put<T>(img, o.idz, t.idz);
        (void)I;  // the state starts at the rest Maxwellian n = 1, T = 1 (f_k = w_k): d = 0,
                  // the zeros of the image, with residual 0 and F0 holding the state
        *reinterpret_cast<int*>(img.data() + o.active) = 1;
        InstDev& D = h->idev[b];
        D.Hx = reinterpret_cast<const double*>(P + o.Hx);
        D.Hy = reinterpret_cast<const double*>(P + o.Hy);
        D.Pz = reinterpret_cast<const double*>(P + o.Pz);
        D.Hx2 = reinterpret_cast<const float2*>(P + o.Hx2);
        D.Hy2 = reinterpret_cast<const float2*>(P + o.Hy2);
        D.Pz2 = reinterpret_cast<const float2*>(P + o.Pz2);
        D.sumw_x = D.sumw_y = D.sumw_z = 0.0;  // of the weights as stored
        for (int i = 0; i < I.Qx; ++i) D.sumw_x += double(T(t.wx[i]));
        for (int j = 0; j < I.Qy; ++j) D.sumw_y += double(T(t.wy[j]));
        for (int m = 0; m < I.Qz; ++m) D.sumw_z += 2.0 * double(T(t.wz[m]));
        D.alpha = reinterpret_cast<const double*>(P + o.alpha);
        D.beta = reinterpret_cast<const double*>(P + o.beta);
        D.px = P + o.px; D.py = P + o.py; D.xi = P + o.xi; D.wx = P + o.wx; D.wy = P + o.wy; D.wz = P + o.wz;
        D.gwx_top = P + o.gxt; D.gwx_bot = P + o.gxb; D.gwy = P + o.gwy; D.gwz = P + o.gwz;
        D.inv_dz = P + o.idz;
        D.F0 = P + o.F0; D.F1 = P + o.F1; D.F2 = P + o.F2; D.rec = P + o.rec;
        D.L0 = h->fp32 ? reinterpret_cast<unsigned short*>(P + o.L0) : nullptr;
        D.cur = reinterpret_cast<int*>(P + o.cur);
        D.partial = P + o.partial;
        D.flux_part = reinterpret_cast<double*>(P + o.flux);
        D.nw = reinterpret_cast<double*>(P + o.nw);
        D.prof = reinterpret_cast<double*>(P + o.prof);
        D.Wold = reinterpret_cast<double*>(P + o.Wold);
        D.Wnew = reinterpret_cast<double*>(P + o.Wnew);
        D.res = reinterpret_cast<double*>(P + o.res);
        D.steps = reinterpret_cast<long long*>(P + o.steps);
        D.active = reinterpret_cast<int*>(P + o.active);
        D.status = reinterpret_cast<int*>(P + o.status);
        D.zcount = reinterpret_cast<int*>(P + o.zcount);
        D.icount = reinterpret_cast<int*>(P + o.icount);
        D.nzt = I.nzt;
        D.rec_stride = rec_stride_of(I.Qx, I.Qy, I.Qz);
    }
    choose_finalize(h);
    std::memcpy(img.data() + inst_off, h->idev.data(), sizeof(InstDev) * h->ninst);
    std::memcpy(img.data() + tile_off, tiles.data(), sizeof(Tile) * tiles.size());
    h->d_inst = reinterpret_cast<InstDev*>(P + inst_off);
    h->d_tiles = reinterpret_cast<Tile*>(P + tile_off);
    h->d_macro = reinterpret_cast<double*>(P + macro_off);
    h->prof_all = reinterpret_cast<double*>(P + prof_base);
    h->mom_all = reinterpret_cast<double*>(P + mom_off);
    h->status_all = reinterpret_cast<int*>(P + status_base);
    h->cur_all = reinterpret_cast<int*>(P + cur_base);
    h->ntiles = (int)tiles.size();
    CK(cudaMemcpyAsync(P, img.data(), pool.bytes, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBS_OK;
}

// NVTX ranges on the host thread (no cost without an attached profiler): one per C
// call that queues GPU work and one per RK stage as it is enqueued (inside a CUDA-graph
// capture they mark the capture, the graph launches carry their own range)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
static const char* const kStageRange[4] = {"lbs analysis", "lbs RK stage 1", "lbs RK stage 2", "lbs RK stage 3"};

// moments, records, wall densities and W_old of the current F0 (every active instance)
static lbs_status analyse(lbs_solver* h)
{
    NvtxRange r(kStageRange[0]);
    CK(launch_stage(h->fp32, h->reduced, h->V, 0, h->d_inst, h->d_tiles, h->ntiles, h->smem, h->fuse & 1, h->ninst, h->maxNz,
                    h->fin_warp, h->nb, h->stream));
    return LBS_OK;
}

// fuse = 2: the batch's two halves advance on two streams, each with its own
// (unfused) finalisation, so that one half's FP64 finalisation overlaps the other
// half's stage kernel; the step forks from and joins back into the handle's stream
static bool split(const lbs_solver* h) { return h->fuse == 2 && h->nA > 0 && h->stream2; }

// the second stream and its fork / join events, made on first use (split stepping, the
// pipelined lbs_set_state)
static lbs_status ensure_stream2(lbs_solver* h)
{
    if (h->stream2) return LBS_OK;
    CK(cudaStreamCreateWithFlags(&h->stream2, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    return LBS_OK;
}

static lbs_status enqueue_step(lbs_solver* h)
{
    if (!split(h)) {
        for (int s = 1; s <= 3; ++s) {
            NvtxRange r(kStageRange[s]);
            CK(launch_stage(h->fp32, h->reduced, h->V, s, h->d_inst, h->d_tiles, h->ntiles, h->smem, h->fuse & 1, h->ninst,
                            h->maxNz, h->fin_warp, h->nb, h->stream));
        }
        return LBS_OK;
    }
    CK(cudaEventRecord(h->ev_fork, h->stream));
    CK(cudaStreamWaitEvent(h->stream2, h->ev_fork, 0));
    // the stage kernel finds a tile's instance by its absolute index (full descriptor
    // array, a range of tiles); the finalisation kernels take a range of instances
    for (int s = 1; s <= 3; ++s) {
        NvtxRange r(kStageRange[s]);
        CK(launch_stage_only(h->fp32, h->reduced, h->V, s, h->d_inst, h->d_tiles, h->ntilesA, h->smem, 0, h->stream));
        CK(launch_finalize(h->fp32, s, h->d_inst, h->nA, h->maxNz, h->fin_warp, h->nb, h->stream));
        CK(launch_stage_only(h->fp32, h->reduced, h->V, s, h->d_inst, h->d_tiles + h->ntilesA, h->ntiles - h->ntilesA, h->smem,
                             0, h->stream2));
        CK(launch_finalize(h->fp32, s, h->d_inst + h->nA, h->ninst - h->nA, h->maxNz, h->fin_warp, h->nb, h->stream2));
    }
    CK(cudaEventRecord(h->ev_join, h->stream2));
    CK(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    return LBS_OK;
}

static void drop_graph(lbs_solver* h)
{
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    h->gsteps = 0;
}

static lbs_status get_graph(lbs_solver* h, int nsteps)
{
    if (h->gexec && h->gsteps == nsteps) return LBS_OK;
    drop_graph(h);
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    lbs_status st = LBS_OK;
    for (int i = 0; i < nsteps && st == LBS_OK; ++i) st = enqueue_step(h);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (st != LBS_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(LBS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(LBS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    h->gsteps = nsteps;
    return LBS_OK;
}

static lbs_status check_status(lbs_solver* h)
{
    std::vector<int> st(h->ninst);
    CK(cudaMemcpyAsync(st.data(), h->status_all, 4 * (size_t)h->ninst, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int b = 0; b < h->ninst; ++b)
        if (st[b] & STATUS_TIMEOUT)
            return fail(LBS_ERR_TIMEOUT, "instance " + std::to_string(b) +
                                             ": a stage CTA's bounded wait for its bulk copies ran out; that stage's "
                                             "output is incomplete");
    for (int b = 0; b < h->ninst; ++b)
        if (st[b]) return fail(LBS_ERR_NONFINITE, "instance " + std::to_string(b) + " reached a non-finite or non-positive state");
    return LBS_OK;
}

// ---------------------------------------------------------------- C ABI -----
extern "C" {

const char* lbs_last_error(void) { return g_err.c_str(); }

lbs_status lbs_quadrature(int kind, int Q, double* nodes, double* weights)
{
    if ((kind != 0 && kind != 1) || Q < 1 || Q > kMaxQ1D || !nodes || !weights)
        return fail(LBS_ERR_ARG, "kind must be 0 or 1 and Q in 1..100");
    if (gauss_rule(kind == 0 ? QUAD_FULL : QUAD_HALF, Q, nodes, weights))
        return fail(LBS_ERR_QUADRATURE, "Gauss rule construction failed");
    return LBS_OK;
}

// Three-point Lagrange value at x of the samples (x_a, y_a), used for u_x(L/2) of
// Eq. (uslip_extra).
static double lagrange_at(double x, const double* xs, const double* ys)
{
    double w[3];
    lagrange3(x, xs[0], xs[1], xs[2], w);
    return w[0] * ys[0] + w[1] * ys[1] + w[2] * ys[2];
}

// Checks the grid arguments of the diagnostics; S = the cells of the half channel 0 <= z <= L/2
// (all Nz of a half channel, the upper Nz/2 of a full one).
static lbs_status half_cells(int Nz, double A, int half, int* S)
{
    if (!(A >= 0.0 && A < 1.0) || (half != 0 && half != 1)) return fail(LBS_ERR_ARG, "need 0 <= A < 1, half 0 or 1");
    if (!half && (Nz % 2 != 0 || Nz < 12)) return fail(LBS_ERR_ARG, "a full channel needs an even Nz >= 12");
    if (half && Nz < 6) return fail(LBS_ERR_ARG, "a half channel needs Nz >= 6");
    *S = half ? Nz : Nz / 2;
    return LBS_OK;
}

// Eq. (etas) on the half channel: eta_s = (s - 1/2) atanh(A) / S, x_s = L tanh(eta_s) / (2A)
// (uniform cells for A = 0), and the rectangle-rule weights of Eqs. (mflow), (Txy) divided
// by L / 2 (they sum to 1 up to the rule's error).
static void half_positions(int S, double A, std::vector<double>& x, std::vector<double>& wrect)
{
    const double E = A > 0.0 ? std::atanh(A) : 0.0;
    x.resize(S);
    wrect.resize(S);
    for (int s = 0; s < S; ++s) {
        if (A > 0.0) {
            const double eta = (s + 0.5) * E / S, c = std::cosh(eta);
            x[s] = std::tanh(eta) / (2.0 * A);
            wrect[s] = E / (A * S) / (c * c);  // L dx/deta at eta_s times d_eta, / (L / 2)
        } else {
            x[s] = (s + 0.5) / (2.0 * S);
            wrect[s] = 1.0 / S;
        }
    }
}

lbs_status lbs_couette_nonlinear_velocity(const double* prof, int Nz, double A, int half, double* z_out,
                                          double* unl_out)
{
    if (!prof || !unl_out) return fail(LBS_ERR_ARG, "null profiles or output");
    int S = 0;
    lbs_status st = half_cells(Nz, A, half, &S);
    if (st != LBS_OK) return st;
    const double* u = prof + 1 * (size_t)Nz + (Nz - S);
    std::vector<double> x, wrect;
    half_positions(S, A, x, wrect);
    const double xw[3] = {x[S - 1], x[S - 2], x[S - 3]}, uw3[3] = {u[S - 1], u[S - 2], u[S - 3]};
    const double uwall = lagrange_at(0.5, xw, uw3);  // u_x(L/2), Eq. (uslip_extra)
    for (int s = 0; s < S; ++s) {
        unl_out[s] = 2.0 * x[s] - u[s] / uwall;  // Eq. (uy_nl) with L = 1
        if (z_out) z_out[s] = x[s];
    }
    return LBS_OK;
}

lbs_status lbs_couette_diagnostics(const double* prof, int Nz, double A, int half, double u_w, double T_w,
                                   lbs_diag* out)
{
    if (!prof || !out) return fail(LBS_ERR_ARG, "null profiles or output");
    int S = 0;
    lbs_status st = half_cells(Nz, A, half, &S);
    if (st != LBS_OK) return st;
    const int s0 = Nz - S;  // cells s0 .. Nz-1 form the upper half
    const double* n = prof + 0 * (size_t)Nz + s0;
    const double* u = prof + 1 * (size_t)Nz + s0;
    const double* T = prof + 4 * (size_t)Nz + s0;
    const double* Pxz = prof + 12 * (size_t)Nz + s0;
    std::vector<double> x, wrect;
    half_positions(S, A, x, wrect);
    lbs_diag d;
    const double xw[3] = {x[S - 1], x[S - 2], x[S - 3]}, uw3[3] = {u[S - 1], u[S - 2], u[S - 3]};
    d.u_wall = lagrange_at(0.5, xw, uw3);
    d.u_slip = u_w - d.u_wall;
    // odd profile u = c1 x + c3 x^3 + c5 x^5 through the first three cells: u'(0) = c1
    const double a1 = x[0] * x[0], a2 = x[1] * x[1], a3 = x[2] * x[2];
    d.dudz0 = a2 * a3 * u[0] / (x[0] * (a1 - a2) * (a1 - a3)) + a1 * a3 * u[1] / (x[1] * (a2 - a1) * (a2 - a3)) +
              a1 * a2 * u[2] / (x[2] * (a3 - a1) * (a3 - a2));
    // even profile T = c0 + c2 x^2 + c4 x^4: T(0) = c0
    d.T0 = a2 * a3 * T[0] / ((a1 - a2) * (a1 - a3)) + a3 * a1 * T[1] / ((a2 - a1) * (a2 - a3)) +
           a1 * a2 * T[2] / ((a3 - a1) * (a3 - a2));
    d.nu = d.dudz0 / (2.0 * u_w);
    double m = 0.0, t = 0.0;
    for (int s = 0; s < S; ++s) {
        m += wrect[s] * n[s] * u[s];
        t += wrect[s] * Pxz[s];
    }
    d.mflow = 0.5 * m;  // the rectangle weights average over L/2: the integral is L/2 times that
    d.mflow_hydro = 0.25 * u_w;
    d.Txy = t;
    d.Txy_bal = -u_w * std::sqrt(2.0 * T_w / 3.14159265358979323846);
    d.Pi = -t / (u_w * std::sqrt(2.0));
    *out = d;
    return LBS_OK;
}

lbs_status lbs_batch_create(lbs_handle* out, const lbs_instance_desc* desc, int n, lbs_precision prec,
                            void* cuda_stream)
{
    if (!out || !desc || n < 1) return fail(LBS_ERR_ARG, "need an output handle and n >= 1 descriptors");
    if (prec != LBS_FP64 && prec != LBS_FP32_STORE_FP64_ACC) return fail(LBS_ERR_ARG, "unknown precision");
    *out = nullptr;
    for (int b = 0; b < n; ++b) {
        lbs_status s = validate(desc[b]);
        if (s != LBS_OK) return fail(s, "instance " + std::to_string(b) + ": " + g_err);
        if ((desc[b].orders.Qy == 0) != (desc[0].orders.Qy == 0))
            return fail(LBS_ERR_ARG, "a batch cannot mix the reduced (Qy = 0) and the full velocity models");
    }
    lbs_solver* h = new lbs_solver();
    h->reduced = desc[0].orders.Qy == 0;
    if (cudaGetDevice(&h->device) != cudaSuccess) h->device = 0;
    h->fp32 = prec == LBS_FP32_STORE_FP64_ACC;
    h->esize = h->fp32 ? 4 : 8;
    h->ninst = n;
    h->ih.resize(n);
    long work = 0;
    for (int b = 0; b < n; ++b)
        work += (long)desc[b].grid.Nz * 2 * desc[b].orders.Qx * std::max(desc[b].orders.Qy, 2) *
                desc[b].orders.Qz_half;
    // untuned default: small batches are latency-bound (short z-tiles, one velocity per
    // thread, more CTAs); large ones take the throughput tiling.  Finalisation apart.
    h->V = work >= (1L << 22) ? 4 : 1;
    h->ZT = work >= (1L << 22) ? 12 : 4;
    // the FP32 full model with V = 2, 4 takes velocities in pairs (64-bit words), which
    // needs Q / 2 even in every instance; else one velocity per thread
    for (int b = 0; b < n; ++b)
        if (h->fp32 && !h->reduced &&
            (desc[b].orders.Qx * std::max(desc[b].orders.Qy, 2) * desc[b].orders.Qz_half) % 2)
            h->V = 1;
    h->fuse = 0;
    if (cuda_stream) {
        h->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete h;
            return fail(LBS_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
        }
        h->own_stream = true;
    }
    lbs_status s = h->fp32 ? setup<float>(h, desc) : setup<double>(h, desc);
    if (s == LBS_OK) s = analyse(h);
    if (s == LBS_OK) s = check_status(h);
    if (s != LBS_OK) {
        std::string m = g_err;
        lbs_destroy(h);
        return fail(s, m);
    }
    *out = h;
    return LBS_OK;
}

lbs_status lbs_create(lbs_handle* out, lbs_orders ord, lbs_grid grid, double Kn, double u_w, double T_w,
                      double Pr, lbs_visc visc, lbs_precision prec, double cfl, void* cuda_stream)
{
    lbs_instance_desc d;
    d.orders = ord;
    d.grid = grid;
    d.Kn = Kn; d.u_w = u_w; d.T_w = T_w; d.Pr = Pr;
    d.visc = visc;
    d.dt = 0.0;
    d.cfl = cfl;
    if (!(cfl > 0.0)) return fail(LBS_ERR_ARG, "cfl must be positive");
    return lbs_batch_create(out, &d, 1, prec, cuda_stream);
}

lbs_status lbs_destroy(lbs_handle h)
{
    if (!h) return LBS_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graph(h);
    if (h->pool) cudaFree(h->pool);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    if (h->stream2) cudaStreamDestroy(h->stream2);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    delete h;
    return LBS_OK;
}

lbs_status lbs_step(lbs_handle h, long nsteps)
{
    if (!h || nsteps < 0) return fail(LBS_ERR_ARG, "invalid handle or negative step count");
    NvtxRange r("lbs_step");
    const int G = 8;  // steps per CUDA-graph launch
    const long full = nsteps / G, rest = nsteps % G;
    if (full > 0) {
        lbs_status s = get_graph(h, G);
        if (s != LBS_OK) return s;
        NvtxRange rg("lbs 8-step graph launches");
        for (long i = 0; i < full; ++i) CK(cudaGraphLaunch(h->gexec, h->stream));
    }
    for (long i = 0; i < rest; ++i) {
        lbs_status s = enqueue_step(h);
        if (s != LBS_OK) return s;
    }
    return LBS_OK;
}

// The stage kernel's tile list over the instances still marching (act[b] != 0), or
// over all instances (act == nullptr).  run_to_steady drops the tiles of retired
// instances, whose CTAs would only read the descriptor and leave; only whole
// instances are dropped, so the per-instance counts of the fused finalisation hold.
// The split point of fuse = 2 stays at instance nA; a half left without tiles launches
// nothing.  Invalidates the captured graph.
static lbs_status upload_tiles(lbs_solver* h, const std::vector<int>* act)
{
    std::vector<Tile> all, tiles;
    build_tiles(h, all);
    int tA = 0;
    for (const Tile& t : all)
        if (!act || (*act)[t.inst]) {
            tiles.push_back(t);
            tA += t.inst < h->nA;
        }
    if (tiles.empty()) return LBS_OK;  // nothing left to launch: keep the current list
    if (act) h->ntilesA = tA;
    CK(cudaMemcpyAsync(h->d_tiles, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice, h->stream));
    h->ntiles = (int)tiles.size();
    h->tiles_full = tiles.size() == all.size();
    drop_graph(h);
    return LBS_OK;
}

lbs_status lbs_run_to_steady(lbs_handle h, double tol, long max_steps, int check_every, long* steps_out)
{
    if (!h || !(tol > 0.0) || max_steps < 1 || check_every < 1)
        return fail(LBS_ERR_ARG, "need tol > 0, max_steps >= 1, check_every >= 1");
    NvtxRange r("lbs_run_to_steady");
    // arm the device-side retirement test
    for (int b = 0; b < h->ninst; ++b) h->idev[b].tol = tol;
    CK(cudaMemcpyAsync(h->d_inst, h->idev.data(), sizeof(InstDev) * h->ninst, cudaMemcpyHostToDevice, h->stream));
    std::vector<long long> st0(h->ninst), st(h->ninst);
    std::vector<int> act(h->ninst);
    for (int b = 0; b < h->ninst; ++b)
        CK(cudaMemcpyAsync(&st0[b], h->idev[b].steps, 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    lbs_status s = get_graph(h, check_every);
    long done = 0;
    bool all = false;
    while (s == LBS_OK && done < max_steps && !all) {
        CK(cudaGraphLaunch(h->gexec, h->stream));
        done += check_every;
        all = true;
        for (int b = 0; b < h->ninst; ++b)
            CK(cudaMemcpyAsync(&act[b], h->idev[b].active, 4, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        for (int b = 0; b < h->ninst; ++b) all &= act[b] == 0;
        // once a quarter of the launched tiles belong to retired instances, launch only
        // the live ones; once few cells are left, finalise them with a warp per cell
        // (the automatic layout), whose FP64 chains are shorter
        long live = 0, cells = 0;
        for (int b = 0; b < h->ninst; ++b) {
            live += act[b] ? (long)h->ih[b].nchunks * h->ih[b].nzt : 0;
            cells += act[b] ? h->ih[b].Nz : 0;
        }
        bool regraph = false;
        if (!all && 4 * live <= 3L * h->ntiles) {
            s = upload_tiles(h, &act);
            regraph = true;
        }
        if (!all && s == LBS_OK && h->fin_mode == 0 && !h->fin_warp && cells <= kFinWarpMaxCells) {
            h->fin_warp = 1;
            for (int b = 0; b < h->ninst; ++b) h->idev[b].fin_warp = 1;
            CK(cudaMemcpyAsync(h->d_inst, h->idev.data(), sizeof(InstDev) * h->ninst, cudaMemcpyHostToDevice,
                               h->stream));
            drop_graph(h);
            regraph = true;
        }
        if (regraph && s == LBS_OK) s = get_graph(h, check_every);
    }
    // disarm and reactivate every instance, with every tile and the batch's own
    // finalisation layout
    choose_finalize(h);
    for (int b = 0; b < h->ninst; ++b) h->idev[b].tol = 0.0;
    CK(cudaMemcpyAsync(h->d_inst, h->idev.data(), sizeof(InstDev) * h->ninst, cudaMemcpyHostToDevice, h->stream));
    const int one = 1;
    for (int b = 0; b < h->ninst; ++b) {
        CK(cudaMemcpyAsync(&st[b], h->idev[b].steps, 8, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(h->idev[b].active, &one, 4, cudaMemcpyHostToDevice, h->stream));
    }
    const lbs_status su = upload_tiles(h, nullptr);
    if (s == LBS_OK) s = su;
    CK(cudaStreamSynchronize(h->stream));
    if (s != LBS_OK) return s;
    if (steps_out)
        for (int b = 0; b < h->ninst; ++b) steps_out[b] = (long)(st[b] - st0[b]);
    s = check_status(h);
    if (s != LBS_OK) return s;
    if (!all) return fail(LBS_ERR_NO_CONVERGENCE, "residual target not reached within max_steps");
    return LBS_OK;
}

lbs_status lbs_profile_steps(lbs_handle h, long nsteps, double* out_ms)
{
    if (!h || nsteps < 1 || !out_ms) return fail(LBS_ERR_ARG, "need a handle, nsteps >= 1 and an output");
    std::vector<cudaEvent_t> ev(7);  // per step: before/after each stage kernel, after its finalisation
    for (auto& e : ev) CK(cudaEventCreate(&e));
    double tstage = 0.0, tfin = 0.0, tstep = 0.0;
    lbs_status st = LBS_OK;
    if (split(h)) {  // stage kernels overlap the other half's finalisation: whole steps only
        for (long it = 0; it < nsteps && st == LBS_OK; ++it) {
            CK(cudaEventRecord(ev[0], h->stream));
            st = enqueue_step(h);
            CK(cudaEventRecord(ev[6], h->stream));
            CK(cudaEventSynchronize(ev[6]));
            float w = 0.f;
            CK(cudaEventElapsedTime(&w, ev[0], ev[6]));
            tstep += w;
        }
        for (auto& e : ev) cudaEventDestroy(e);
        if (st != LBS_OK) return st;
        out_ms[0] = tstep;
        out_ms[1] = 0.0;
        out_ms[2] = tstep;
        return check_status(h);
    }
    for (long it = 0; it < nsteps && st == LBS_OK; ++it) {
        CK(cudaEventRecord(ev[0], h->stream));
        for (int s = 1; s <= 3; ++s) {
            CK(launch_stage_only(h->fp32, h->reduced, h->V, s, h->d_inst, h->d_tiles, h->ntiles, h->smem, h->fuse & 1, h->stream));
            CK(cudaEventRecord(ev[2 * s - 1], h->stream));
            if (!(h->fuse & 1)) CK(launch_finalize(h->fp32, s, h->d_inst, h->ninst, h->maxNz, h->fin_warp, h->nb, h->stream));
            CK(cudaEventRecord(ev[2 * s], h->stream));
        }
        CK(cudaEventSynchronize(ev[6]));
        for (int s = 1; s <= 3; ++s) {
            float a = 0.f, b = 0.f;
            CK(cudaEventElapsedTime(&a, ev[2 * s - 2], ev[2 * s - 1]));
            CK(cudaEventElapsedTime(&b, ev[2 * s - 1], ev[2 * s]));
            tstage += a;
            tfin += b;
        }
        float w = 0.f;
        CK(cudaEventElapsedTime(&w, ev[0], ev[6]));
        tstep += w;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    out_ms[0] = tstage;
    out_ms[1] = tfin;
    out_ms[2] = tstep;
    return check_status(h);
}

lbs_status lbs_set_tiling(lbs_handle h, int V, int ZT, int fuse)
{
    if (!h || (V != 1 && V != 2 && V != 4) || ZT < 3 || ZT > kMaxZT || fuse < 0 || fuse > 2)
        return fail(LBS_ERR_ARG, "tiling needs V in {1, 2, 4}, 3 <= ZT <= 64 and fuse in {0, 1, 2}");
    if (h->fp32 && !h->reduced && V != 1)
        for (int b = 0; b < h->ninst; ++b)
            if ((h->ih[b].Q / 2) % 2)
                return fail(LBS_ERR_ARG, "V = 2, 4 in FP32 (velocity pairs) needs Q / 2 even in every instance");
    CK(cudaStreamSynchronize(h->stream));
    drop_graph(h);
    if (fuse == 2) {
        const lbs_status s2 = ensure_stream2(h);
        if (s2 != LBS_OK) return s2;
    }
    h->V = V;
    h->ZT = ZT;
    h->fuse = fuse;
    std::vector<Tile> tiles;
    build_tiles(h, tiles);
    if (tiles.size() > h->max_tiles) return fail(LBS_ERR_ARG, "tile list exceeds its buffer");
    for (int b = 0; b < h->ninst; ++b) {
        h->idev[b].nchunks = h->ih[b].nchunks;
        h->idev[b].nchh = h->ih[b].nchh;
        h->idev[b].nzt = h->ih[b].nzt;
    }
    CK(cudaMemcpyAsync(h->d_tiles, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->d_inst, h->idev.data(), sizeof(InstDev) * h->ninst, cudaMemcpyHostToDevice, h->stream));
    h->ntiles = (int)tiles.size();
    h->tiles_full = true;
    lbs_status s = analyse(h);  // partial sums of the new chunking
    if (s != LBS_OK) return s;
    return check_status(h);
}

lbs_status lbs_get_tiling(lbs_handle h, int* V, int* ZT, int* fuse, int* ntiles, long* smem_bytes)
{
    if (!h) return fail(LBS_ERR_ARG, "invalid handle");
    if (V) *V = h->V;
    if (ZT) *ZT = h->ZT;
    if (fuse) *fuse = h->fuse;
    if (ntiles) *ntiles = h->ntiles;
    if (smem_bytes) *smem_bytes = (long)h->smem;
    return LBS_OK;
}

lbs_status lbs_set_finalize(lbs_handle h, int mode, int* warp_out)
{
    if (!h || mode < 0 || mode > 2) return fail(LBS_ERR_ARG, "finalisation mode must be 0, 1 or 2");
    CK(cudaStreamSynchronize(h->stream));
    drop_graph(h);
    h->fin_mode = mode;
    choose_finalize(h);
    CK(cudaMemcpyAsync(h->d_inst, h->idev.data(), sizeof(InstDev) * h->ninst, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (warp_out) *warp_out = h->fin_warp;
    return check_status(h);
}

lbs_status lbs_get_stream(lbs_handle h, void** out)
{
    if (!h || !out) return fail(LBS_ERR_ARG, "invalid handle or null output");
    *out = static_cast<void*>(h->stream);
    return LBS_OK;
}

static lbs_status inst_ok(lbs_handle h, int inst)
{
    if (!h || inst < 0 || inst >= h->ninst) return fail(LBS_ERR_ARG, "invalid handle or instance index");
    return LBS_OK;
}

static lbs_status copy_profiles(lbs_handle h, int inst, double* host_out)
{
    const int Nz = h->ih[inst].Nz;
    CK(cudaMemcpyAsync(host_out, h->idev[inst].prof, 14 * (size_t)Nz * 8, cudaMemcpyDeviceToHost, h->stream));
    return LBS_OK;
}

lbs_status lbs_profiles(lbs_handle h, int inst, double* host_out)
{
    lbs_status s = inst_ok(h, inst);
    if (s != LBS_OK) return s;
    if (!host_out) return fail(LBS_ERR_ARG, "null output");
    s = copy_profiles(h, inst, host_out);
    if (s != LBS_OK) return s;
    CK(cudaStreamSynchronize(h->stream));
    return check_status(h);
}

lbs_status lbs_diagnostics(lbs_handle h, int inst, lbs_diag* out)
{
    lbs_status s = inst_ok(h, inst);
    if (s != LBS_OK) return s;
    if (!out) return fail(LBS_ERR_ARG, "null output");
    const InstHost& I = h->ih[inst];
    std::vector<double> prof(14 * (size_t)I.Nz);
    s = lbs_profiles(h, inst, prof.data());
    if (s != LBS_OK) return s;
    return lbs_couette_diagnostics(prof.data(), I.Nz, I.d.grid.A, I.d.grid.half, I.d.u_w, I.d.T_w, out);
}

lbs_status lbs_moments(lbs_handle h, int inst, double* host_out)
{
    if (h && inst == -1 && host_out) {
        // every instance: the reported rows gathered on the device, then one copy
        CK(launch_gather_moments(h->d_inst, h->ninst, h->prof_all, h->mom_all, h->stream));
        CK(cudaMemcpyAsync(host_out, h->mom_all, 8 * 8 * (h->prof_all_n / 14), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        return LBS_OK;
    }
    lbs_status s = inst_ok(h, inst);
    if (s != LBS_OK) return s;
    if (!host_out) return fail(LBS_ERR_ARG, "null output");
    const int Nz = h->ih[inst].Nz;
    std::vector<double> all(14 * (size_t)Nz);
    s = copy_profiles(h, inst, all.data());
    if (s != LBS_OK) return s;
    CK(cudaStreamSynchronize(h->stream));
    const int rows[8] = {0, 1, 4, 5, 7, 8, 12, 10};  // n, u_x, T, q_x, q_z, P_xx, P_xz, P_zz
    for (int r = 0; r < 8; ++r) std::memcpy(host_out + (size_t)r * Nz, all.data() + (size_t)rows[r] * Nz, 8 * Nz);
    return LBS_OK;
}

lbs_status lbs_residual(lbs_handle h, int inst, double* out)
{
    lbs_status s = inst_ok(h, inst);
    if (s != LBS_OK) return s;
    if (!out) return fail(LBS_ERR_ARG, "null output");
    CK(cudaMemcpyAsync(out, h->idev[inst].res, 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return check_status(h);
}

lbs_status lbs_steps_taken(lbs_handle h, int inst, long* out)
{
    lbs_status s = inst_ok(h, inst);
    if (s != LBS_OK) return s;
    if (!out) return fail(LBS_ERR_ARG, "null output");
    long long v = 0;
    CK(cudaMemcpyAsync(&v, h->idev[inst].steps, 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *out = (long)v;
    return LBS_OK;
}

lbs_status lbs_info(lbs_handle h, int inst, long* out, double* dt_out)
{
    lbs_status s = inst_ok(h, inst);
    if (s != LBS_OK) return s;
    if (!out) return fail(LBS_ERR_ARG, "null output");
    const InstHost& I = h->ih[inst];
    out[0] = I.Q;
    out[1] = I.Nz;
    out[2] = (long)I.Qx * I.Qy;
    out[3] = h->esize;
    if (dt_out) *dt_out = I.dt;
    return LBS_OK;
}

// The state of instances b0 .. b1-1 as the C ABI exposes it (see lbs_get_state): the
// deviations d of every instance, concatenated, then (FP32) their rounding residuals,
// concatenated.  ext + off0 is where instance b0's d lies in the external buffer, ext +
// off1 where its residuals lie (a range of a larger whole-batch buffer).  Consecutive
// instances whose device buffers are adjacent go in one copy.  sel[b] picks F1 instead of
// F0 for instance b (get: where the state is; set: always F0).
static lbs_status copy_state(lbs_solver* h, int b0, int b1, unsigned char* ext, size_t off0, size_t off1,
                             bool to_ext, bool ext_host, const std::vector<int>& sel)
{
    const cudaMemcpyKind kind = to_ext ? (ext_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice)
                                       : (ext_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice);
    for (int part = 0; part < (h->fp32 ? 2 : 1); ++part) {
        const size_t es = part ? 2 : h->esize;
        size_t off = part ? off1 : off0;
        for (int b = b0; b < b1;) {
            auto dev = [&](int e) -> unsigned char* {
                if (part) return reinterpret_cast<unsigned char*>(h->idev[e].L0);
                return static_cast<unsigned char*>(sel[e] ? h->idev[e].F1 : h->idev[e].F0);
            };
            unsigned char* d = dev(b);
            size_t bytes = 0;
            int e = b;
            do {
                bytes += (size_t)h->ih[e].Nz * h->ih[e].Q * es;
                ++e;
            } while (e < b1 && dev(e) == d + bytes);
            if (to_ext) CK(cudaMemcpyAsync(ext + off, d, bytes, kind, h->stream));
            else CK(cudaMemcpyAsync(d, ext + off, bytes, kind, h->stream));
            off += bytes;
            b = e;
        }
    }
    return LBS_OK;
}

// bytes of the deviations d of instances b0 .. b1-1 as stored
static size_t state_d_bytes(const lbs_solver* h, int b0, int b1)
{
    size_t n = 0;
    for (int b = b0; b < b1; ++b) n += (size_t)h->ih[b].Nz * h->ih[b].Q * h->esize;
    return n;
}

lbs_status lbs_get_state(lbs_handle h, int inst, void* dst, int to_host)
{
    if (!h || inst < -1 || inst >= h->ninst) return fail(LBS_ERR_ARG, "invalid handle or instance index");
    if (!dst) return fail(LBS_ERR_ARG, "null destination");
    const int b0 = inst < 0 ? 0 : inst, b1 = inst < 0 ? h->ninst : inst + 1;
    std::vector<int> cur(h->ninst);
    CK(cudaMemcpyAsync(cur.data(), h->cur_all, 4 * (size_t)h->ninst, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    lbs_status s = copy_state(h, b0, b1, static_cast<unsigned char*>(dst), 0, state_d_bytes(h, b0, b1), true,
                              to_host != 0, cur);
    if (s != LBS_OK) return s;
    CK(cudaStreamSynchronize(h->stream));
    return LBS_OK;
}

// A pipelined lbs_set_state copies in up to four groups of instances, of at least 24 MB
// each: a group's analysis (a stage-0 launch and a latency-bound finalisation, about
// 100 us) then hides behind the next group's copy from host memory (about 211 GB/s).
// Smaller or device-resident states are copied whole and analysed once.
static const int kSetStateChunks = 4;
static const size_t kSetStateGroupBytes = size_t(24) << 20;

lbs_status lbs_set_state(lbs_handle h, int inst, const void* src, int from_host)
{
    if (!h || inst < -1 || inst >= h->ninst) return fail(LBS_ERR_ARG, "invalid handle or instance index");
    if (!src) return fail(LBS_ERR_ARG, "null source");
    NvtxRange r("lbs_set_state");
    const int b0 = inst < 0 ? 0 : inst, b1 = inst < 0 ? h->ninst : inst + 1;
    unsigned char* ext = static_cast<unsigned char*>(const_cast<void*>(src));
    const size_t dtot = state_d_bytes(h, b0, b1);
    // the state goes to F0, and F0 becomes the state buffer of those instances
    const std::vector<int> sel(h->ninst, 0);
    CK(cudaMemsetAsync(h->cur_all + b0, 0, 4 * (size_t)(b1 - b0), h->stream));
    const size_t total = dtot + (h->fp32 ? dtot / h->esize * 2 : 0);
    const int K = (int)std::min<size_t>(std::min(kSetStateChunks, b1 - b0), total / kSetStateGroupBytes);
    lbs_status s = h->tiles_full && from_host && K >= 2 ? ensure_stream2(h) : LBS_ERR_ARG;
    if (s != LBS_OK) {
        // one group (or a compacted tile list): copy, then analyse the whole batch
        s = copy_state(h, b0, b1, ext, 0, dtot, false, from_host != 0, sel);
        if (s == LBS_OK) s = analyse(h);
        if (s != LBS_OK) return s;
        return check_status(h);
    }
    // A large state from host memory: the copy runs in groups of instances on the handle's
    // stream, and each group's analysis (stage 0 and its finalisation over the group's
    // tiles and instances) on the second stream as soon as the group has landed, behind
    // the next group's copy.  The copy is bound by the host link, so the analysis (a full
    // read of the state) is hidden but for the last group's.
    const size_t per = (dtot + K - 1) / K;
    size_t doff = 0, roff = 0;  // bytes of d and of residuals of the groups before
    for (int c0 = b0; c0 < b1;) {
        int c1 = c0;
        size_t db = 0;
        do {
            db += (size_t)h->ih[c1].Nz * h->ih[c1].Q * h->esize;
            ++c1;
        } while (c1 < b1 && db < per);
        s = copy_state(h, c0, c1, ext, doff, dtot + roff, false, from_host != 0, sel);
        if (s != LBS_OK) return s;
        doff += db;
        roff += db / h->esize * 2;
        CK(cudaEventRecord(h->ev_fork, h->stream));
        CK(cudaStreamWaitEvent(h->stream2, h->ev_fork, 0));
        {
            // the same launches as analyse() (the fused finalisation counts per instance)
            NvtxRange ra(kStageRange[0]);
            CK(launch_stage_only(h->fp32, h->reduced, h->V, 0, h->d_inst, h->d_tiles + h->tile_first[c0],
                                 h->tile_first[c1] - h->tile_first[c0], h->smem, h->fuse & 1, h->stream2));
            if (!(h->fuse & 1))
                CK(launch_finalize(h->fp32, 0, h->d_inst + c0, c1 - c0, h->maxNz, h->fin_warp, h->nb, h->stream2));
        }
        c0 = c1;
    }
    CK(cudaEventRecord(h->ev_join, h->stream2));
    CK(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    return check_status(h);
}

lbs_status lbs_set_wait_limit(lbs_handle h, unsigned spins)
{
    if (!h) return fail(LBS_ERR_ARG, "invalid handle");
    CK(cudaStreamSynchronize(h->stream));
    for (int b = 0; b < h->ninst; ++b) h->idev[b].wait_limit = spins;
    CK(cudaMemcpyAsync(h->d_inst, h->idev.data(), sizeof(InstDev) * h->ninst, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBS_OK;
}

lbs_status lbs_clear_status(lbs_handle h)
{
    if (!h) return fail(LBS_ERR_ARG, "invalid handle");
    CK(cudaMemsetAsync(h->status_all, 0, 4 * (size_t)h->ninst, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBS_OK;
}

lbs_status lbs_init_from_profiles(lbs_handle h, int inst, const double* prof)
{
    lbs_status s = inst_ok(h, inst);
    if (s != LBS_OK) return s;
    if (!prof) return fail(LBS_ERR_ARG, "null profiles");
    const int Nz = h->ih[inst].Nz;
    // macro[8][Nz] = n, ux, uy, uz, T, qx, qy, qz from the 8 rows of lbs_moments
    std::vector<double> macro(8 * (size_t)Nz, 0.0);
    for (int c = 0; c < Nz; ++c) {
        const double n = prof[c], ux = prof[Nz + c], T = prof[2 * Nz + c];
        const double qx = prof[3 * Nz + c], qz = prof[4 * Nz + c];
        if (!std::isfinite(n) || !std::isfinite(ux) || !std::isfinite(T) || !std::isfinite(qx) ||
            !std::isfinite(qz) || !(n > 0.0) || !(T > 0.0))
            return fail(LBS_ERR_NONFINITE, "profile value not finite or n, T not positive in cell " + std::to_string(c));
        macro[c] = n; macro[Nz + c] = ux; macro[4 * Nz + c] = T; macro[5 * Nz + c] = qx; macro[7 * Nz + c] = qz;
    }
    CK(cudaMemcpyAsync(h->d_macro, macro.data(), macro.size() * 8, cudaMemcpyHostToDevice, h->stream));
    CK(launch_seed(h->fp32, h->d_inst, inst, Nz, h->d_macro, h->stream));
    s = analyse(h);
    if (s != LBS_OK) return s;
    return check_status(h);
}

lbs_status lbs_init_free_molecular(lbs_handle h, int inst)
{
    lbs_status s = inst_ok(h, inst);
    if (s != LBS_OK) return s;
    CK(launch_seed_free_molecular(h->fp32, h->d_inst, inst, h->ih[inst].Nz, h->stream));
    s = analyse(h);
    if (s != LBS_OK) return s;
    return check_status(h);
}

}  // extern "C"
