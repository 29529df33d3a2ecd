// Device code of one RK-3 stage of the mixed-quadrature Shakhov scheme (kernels.cuh).
// Included by kernels.cu (finalisation, seeding, launchers) and by the four
// stage_*.cu translation units, each of which instantiates the stage kernel for
// one storage type and velocity model so that they compile in parallel.
//
// Per stage (Eq. rk3 around Eq. L_def):
//   stage_kernel     one CTA per tile = (instance, z-range of <= 64 cells,
//                    velocity chunk of 128*V velocities).  The rows of F_in
//                    the tile needs (its cells and a 3-cell halo each side) and
//                    its rows of F_l are staged into shared memory by TMA bulk
//                    copies (one cp.async.bulk per row, one mbarrier).  While
//                    they land, the CTA evaluates the per-axis factors of the
//                    truncated Hermite equilibrium (Sec. III) of its cells.
//                    Ghost rows are then built in shared memory: outgoing
//                    populations by the quadratic extrapolation of the
//                    Appendix, incoming ones as n_w times the wall equilibrium;
//                    below a half channel's centre line, cells 0..2 at the
//                    mirrored velocity (bounce-back, Appendix).
//                    Each thread marches up the z-range for its V velocities
//                    with a register window: WENO-5 interface fluxes (Eqs.
//                    weno5_flux - weno_sigma, Table weno), the divergence of
//                    Eq. (flux), relaxation to n G_x G_y G_z (1 + S) and the
//                    Shu-Osher combine; it stores F_out and accumulates the raw
//                    moments of F_out (in FP32 within the CTA and stored per
//                    chunk in FP32 in FP32 mode; in FP64 in FP64 mode).  Tiles
//                    that end at a wall also reduce the outgoing WENO flux of
//                    F_out through the wall.
//   finalisation     per cell: the sum of the chunks' partials (double-float in
//                    FP32 mode, FP64 in FP64 mode), n, u, P, T, q (Eq. qdef),
//                    tau, and the cell record of the next stage; per
//                    instance: the wall densities n_w (zero net mass
//                    flux, Appendix) and, after the third stage, the residual.
//                    Either a launch of its own (finalize_cells, one thread per
//                    cell, or finalize_cells_warp, one warp per cell, in
//                    kernels.cu), or folded into the stage kernel (fuse = 1:
//                    the CTA that ends last among the chunks of a z-tile does
//                    its cells, threadfence tickets).
//
// Template parameter RED: the reduced phi / chi model of Sec. III (j = 0 phi,
// j = 1 chi on a two-node transverse axis), otherwise the full 3D velocity set.
//
// Storage: F[s][k] for interior cells s = 0..Nz-1 (no ghost rows), velocity
// k = ((sg*Qz + m)*Qx + i)*Qy + j fastest, holding f_k / w_k.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "lbs_internal.h"

namespace lbs {

template <typename T> struct Acc { typedef double type; };
template <> struct Acc<float> { typedef float type; };


// ---- PTX helpers: mbarrier and bulk global -> shared copies ------------------
static __device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
static __device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
static __device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
static __device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
static __device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
static __device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// WENO-5 reconstruction of five upwind-ordered values (no advection factor), as the
// correction to the upwind cell's value v2: weno5 = v2 + weno5_corr.  The candidate
// reconstructions are c_q = v2 + e_q / 6 with e_q made of the differences d_j = v_j - v2
// (Eq. weno5_flux), and the smoothness indicators are written in the same differences
// (Eq. weno_sigma), so the correction carries the precision of the differences, not of
// v2, and the divergence of Eq. (flux) can be formed as a difference of cell values plus
// a difference of corrections.  The weights (Eq. weno5_omega) are scale free, so they
// are formed from r_q = sigma_q / max sigma; an r_q below kTiny counts as vanishing and
// the weights of Table (weno) apply (proportional to the ideal weights over the
// vanishing set).
template <typename T>
__device__ __forceinline__ T weno5_corr(T v0, T v1, T v2, T v3, T v4)
{
    const T kTiny = sizeof(T) == 8 ? T(1e-150) : T(1e-18);
    const T d0 = v0 - v2, d1 = v1 - v2, d3 = v3 - v2, d4 = v4 - v2;
    const T e1 = T(2) * d0 - T(7) * d1, e2 = T(2) * d3 - d1, e3 = T(5) * d3 - d4;
    T a = d0 - T(2) * d1, b = d0 - T(4) * d1;
    const T s1 = T(13.0 / 12.0) * a * a + T(0.25) * b * b;
    a = d1 + d3;
    b = d1 - d3;
    const T s2 = T(13.0 / 12.0) * a * a + T(0.25) * b * b;
    a = d4 - T(2) * d3;
    b = d4 - T(4) * d3;
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
    return (w1 * e1 + w2 * e2 + w3 * e3) / (T(6) * (w1 + w2 + w3));
}

static __device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// FP32 form, the same stencils in constant-light operations (the multiples 2, 4, 5, 7 of
// the differences built by additions; two constants in all, which the packed form below
// keeps in registers): 4 sigma_q = 13/3 a_q^2 + b_q^2 and the ideal weights scaled by 10
// to (1, 6, 3), common factors that cancel in the normalised weights.  (4 sigma_q)^2 is
// floored at 1.6e-36 (sigma_q^2 at 1e-37; branch free, hardware reciprocals): as
// sigma_q -> 0 the floor gives exactly the limits of Table (weno), and it changes nothing
// while sigma_q^2 > 1e-30, i.e. for differences above the FP32 resolution of O(1)
// normalised populations.  The rounded weights only multiply the small corrections e_q.
constexpr float kWenoK = 13.f / 3.f, kWenoFloor = 1.6e-36f;
template <>
__device__ __forceinline__ float weno5_corr<float>(float v0, float v1, float v2, float v3, float v4)
{
    const float d0 = v0 - v2, d1 = v1 - v2, d3 = v3 - v2, d4 = v4 - v2;
    const float t = d1 + d1, u = d3 + d3;
    const float a1 = d0 - t, b1 = a1 - t;    // v0-2v1+v2, v0-4v1+3v2
    const float a2 = d1 + d3, b2 = d1 - d3;  // v1-2v2+v3, v1-v3
    const float a3 = d4 - u, b3 = a3 - u;    // v2-2v3+v4, 3v2-4v3+v4
    const float e1 = (a1 + b1) - d1;         // 6 (c1 - v2) = 2 d0 - 7 d1
    const float e2 = u - d1;                 // 6 (c2 - v2) = 2 d3 - d1
    const float e3 = (u + d3) - a3;          // 6 (c3 - v2) = 5 d3 - d4
    const float s1 = fmaf(kWenoK, a1 * a1, b1 * b1);
    const float s2 = fmaf(kWenoK, a2 * a2, b2 * b2);
    const float s3 = fmaf(kWenoK, a3 * a3, b3 * b3);
    const float w1 = rcp_approx(fmaf(s1, s1, kWenoFloor));
    const float w2 = 6.f * rcp_approx(fmaf(s2, s2, kWenoFloor));
    const float w3 = 3.f * rcp_approx(fmaf(s3, s3, kWenoFloor));
    const float inv = rcp_approx(6.f * ((w1 + w2) + w3));
    return fmaf(w1, e1, fmaf(w2, e2, w3 * e3)) * inv;
}

// ---- packed FP32 (two lanes of f32x2 per instruction, each element rounded exactly as
// the scalar operation) ----------------------------------------------------------------
#define LBS_OP2(name, op)                                                                       \
    static __device__ __forceinline__ float2 name(float2 a, float2 b)                           \
    {                                                                                           \
        float2 d;                                                                               \
        asm("{.reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n " op    \
            " rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"                                           \
            : "=f"(d.x), "=f"(d.y)                                                              \
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                          \
        return d;                                                                               \
    }
LBS_OP2(add2, "add.rn.f32x2")
LBS_OP2(sub2, "sub.rn.f32x2")
LBS_OP2(mul2, "mul.rn.f32x2")
#undef LBS_OP2
static __device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{.reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mov.b64 rc, {%6, %7};\n"
        " fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
static __device__ __forceinline__ float2 splat(float a) { return make_float2(a, a); }

// weno5_corr<float> for two velocities at once (the same operations, element by element;
// the reciprocals and the multiplications by the scaled ideal weights stay scalar): about
// half the issued arithmetic of two scalar calls
static __device__ __forceinline__ float2 weno5_corr2(float2 v0, float2 v1, float2 v2, float2 v3, float2 v4)
{
    const float2 d0 = sub2(v0, v2), d1 = sub2(v1, v2), d3 = sub2(v3, v2), d4 = sub2(v4, v2);
    const float2 t = add2(d1, d1), u = add2(d3, d3);
    const float2 a1 = sub2(d0, t), b1 = sub2(a1, t);
    const float2 a2 = add2(d1, d3), b2 = sub2(d1, d3);
    const float2 a3 = sub2(d4, u), b3 = sub2(a3, u);
    const float2 e1 = sub2(add2(a1, b1), d1), e2 = sub2(u, d1), e3 = sub2(add2(u, d3), a3);
    const float2 K = splat(kWenoK), F = splat(kWenoFloor);
    const float2 s1 = fma2(K, mul2(a1, a1), mul2(b1, b1));
    const float2 s2 = fma2(K, mul2(a2, a2), mul2(b2, b2));
    const float2 s3 = fma2(K, mul2(a3, a3), mul2(b3, b3));
    const float2 q1 = fma2(s1, s1, F), q2 = fma2(s2, s2, F), q3 = fma2(s3, s3, F);
    const float2 w1 = make_float2(rcp_approx(q1.x), rcp_approx(q1.y));
    const float2 w2 = make_float2(6.f * rcp_approx(q2.x), 6.f * rcp_approx(q2.y));
    const float2 w3 = make_float2(3.f * rcp_approx(q3.x), 3.f * rcp_approx(q3.y));
    const float2 sw = add2(add2(w1, w2), w3);
    const float2 inv = make_float2(rcp_approx(6.f * sw.x), rcp_approx(6.f * sw.y));
    return mul2(fma2(w1, e1, fma2(w2, e2, mul2(w3, e3))), inv);
}

template <typename T>
__device__ __forceinline__ T weno5(T v0, T v1, T v2, T v3, T v4)
{
    return v2 + weno5_corr<T>(v0, v1, v2, v3, v4);
}

template <typename T>
__device__ __forceinline__ T ld(const void* p, int i) { return static_cast<const T*>(p)[i]; }

// Block-wide FP64 sum (all threads get the result); deterministic order.
static __device__ double block_sum(double v, double* red)
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

// N block sums at once (one pair of barriers for all of them); red holds
// N * (blockDim.x / 32) doubles.  Each sum keeps block_sum's order.
template <int N>
__device__ void block_sum_n(double (&v)[N], double* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) red[i * nw + w] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) {
        double s = 0.0;
        for (int j = 0; j < nw; ++j) s += red[i * nw + j];
        v[i] = s;
    }
    __syncthreads();
}
constexpr int kRedSlots = 8 * (kThreads / 32);  // shared doubles for block_sum_n<8> with 128 threads

// Warp reduce-scatter of 16 values: afterwards lane l holds the warp total of
// value m(l) = 8 b4 + 4 b3 + 2 b2 + b1 (b = bits of l); lanes l, l^1 agree.
// 16 shuffles per lane instead of 16 x 5 for 16 separate butterflies.
template <typename A>
__device__ __forceinline__ A reduce_scatter16(A (&v)[16], int lane)
{
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const bool hi = lane & 16;
        const A send = hi ? v[i] : v[i + 8], keep = hi ? v[i + 8] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool hi = lane & 8;
        const A send = hi ? v[i] : v[i + 4], keep = hi ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool hi = lane & 4;
        const A send = hi ? v[i] : v[i + 2], keep = hi ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const bool hi = lane & 2;
        const A send = hi ? v[0] : v[1], keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// shared-memory layout of a stage CTA (offsets in bytes): the staged rows of the
// step's start state d (cells z0-3 .. z0+zn+2) and the cell records (by bulk copy), the
// per-axis factors of this chunk's nodes, 1/dz, and the per-warp moment sums.  The stage
// input's increment (stages 2 and 3) is read from global memory during the march.
struct StageSmem {
    size_t fin, rec, g, idz, red, total;
};
__host__ __device__ inline size_t pad16(size_t b) { return (b + 15) & ~size_t(15); }
__host__ __device__ inline StageSmem stage_smem(int zn, int KC, int G, int esize, int asize, int rstride)
{
    StageSmem L;
    size_t o = 0;
    L.fin = o; o += (size_t)(zn + 6) * KC * esize;
    L.rec = o; o += (size_t)zn * rstride * esize;
    L.g = o; o += pad16((size_t)zn * G * esize);
    L.idz = o; o += pad16((size_t)zn * esize);
    L.red = o; o += (size_t)zn * (kThreads / 32) * 16 * asize;
    L.total = o;
    return L;
}

// ---- the FP32 state's rounding residual --------------------------------------
// The state d is stored as hi (FP32) plus lo, |lo| <= ulp(hi) / 2, kept as a 16-bit
// integer q = round(lo / ulp(hi) * 2^15).  The RK increment of a step near the steady
// state is far below ulp(hi); added to hi alone it would be rounded away and the state
// would stall at a distance of about eps_32 / (lambda dt) from the steady state
// (lambda the decay rate of its slowest mode).  With lo the increment accumulates in
// lo until it carries into hi; what is lost is below 2^-16 ulp(hi) per step.
// ulp(hi) = 2^(E - 150) for the biased exponent E of a normal hi, so
// lo / ulp(hi) * 2^15 = lo * 2^(165 - E), a power of two built in the exponent field
// from the masked exponent bits of hi (E clamped below at 38; the decoding scale
// 2^(E - 165) is then zero: a hi below 2^-88 keeps no residual).
// Both without int/float conversion instructions: for |x| < 2^22, fma(lo, s, 1.5 2^23)
// holds round-to-nearest-even(lo s) in its low mantissa bits (s is a power of two, so the
// product is exact and rounded once, as __float2int_rn rounds it), and 2^23 + u is exact
// for a 16-bit u, so q = float bits of (2^23 + 2^15 + q) minus (2^23 + 2^15).
static __device__ __forceinline__ unsigned lo_bits(float lo, float hi)  // q in the low 16 bits
{
    const unsigned m = max(__float_as_uint(hi) & 0x7f800000u, 38u << 23);
    const float s = __uint_as_float((292u << 23) - m);  // 2^(165 - E)
    return __float_as_uint(fmaf(lo, s, 12582912.0f));
}
static __device__ __forceinline__ unsigned short lo_encode(float lo, float hi)
{
    return static_cast<unsigned short>(lo_bits(lo, hi));
}
static __device__ __forceinline__ unsigned lo_encode2(float2 lo, float2 hi)  // two residuals, x low
{
    return __byte_perm(lo_bits(lo.x, hi.x), lo_bits(lo.y, hi.y), 0x5410);
}
static __device__ __forceinline__ float lo_decode(unsigned q16, float hi)  // q in the low 16 bits
{
    const unsigned m = max(__float_as_uint(hi) & 0x7f800000u, 38u << 23);
    const float s = __uint_as_float(m - (38u << 23));  // 2^(E - 165), zero for E = 38
    const float q = __uint_as_float((q16 & 0xffffu) ^ 0x4B008000u) - 8421376.0f;  // the int16 q
    return q * s;
}

// ---- double-float arithmetic (an FP32 pair hi + lo, |lo| <= ulp(hi) / 2) for the
// FP32 records' node sums.  On this GPU an FP64 instruction occupies a scheduler's
// FP64 unit for about 70 cycles whatever the number of active lanes, FP32 instructions
// issue every cycle: the error-free transforms below (Knuth's TwoSum, the FMA form of
// TwoProduct, a Fast2Sum renormalisation) cost a few FP32 instructions per term and
// carry about 2^-44 of the largest term, well inside the half ulp of FP32 the factors
// are rounded to.
struct DF {
    float hi, lo;
};
static __device__ __forceinline__ DF df_of(double x)
{
    const float h = __double2float_rn(x);
    return DF{h, __double2float_rn(x - double(h))};
}
static __device__ __forceinline__ void df_add(DF& S, float p, float e)  // S += p + e, |e| << |p|
{
    const float s = S.hi + p, bb = s - S.hi;
    float t = (S.hi - (s - bb)) + (p - bb);  // TwoSum(S.hi, p)
    t += S.lo + e;
    S.hi = s + t;
    S.lo = t - (S.hi - s);  // Fast2Sum
}
static __device__ __forceinline__ void df_fma(DF& S, DF c, float2 h)  // S += c h (h = (hi, lo))
{
    const float p = c.hi * h.x;
    const float e = fmaf(c.hi, h.y, fmaf(c.lo, h.x, fmaf(c.hi, h.x, -p)));
    df_add(S, p, e);
}
static __device__ __forceinline__ void df_add_prod(DF& S, float a, float b)  // S += a b, exact product
{
    const float p = a * b;
    df_add(S, p, fmaf(a, b, -p));
}

// ----------------------------------------------------------------------------
// Cell record of a macroscopic state: the scalars and the per-node factors of the
// truncated Hermite equilibrium (Sec. III, Eqs. fyz, Fmn_def), computed in FP64 (the
// half-range coefficients cancel strongly for N >= 4) and rounded once.  A factor's
// deviation from 1 is sum_l (c_l - r_l) basis_l(node) with the rest state's
// coefficients r: (1, 0, 0, ...) on x and y, (1, 1) on the reduced model's y (factors 1
// and T), (1/2, 0, ...) on each half range of z, for which sum_l r_l basis_l = 1 at every
// node.  R_SCALE makes the discrete equilibrium carry exactly n: in exact arithmetic
// sum_i w_i Gx = 1, sum_j w_j Gy = 1 and the sum over both half ranges of w Gz = 1
// (orthogonality of the bases); with the factors rounded to the storage type the sums
// miss by a few ulps of the same sign every step, which would let FP32 runs drift in
// mass, so the sums are taken over the stored values.  Returns false for a non-finite
// or non-positive state (a neutral state is written instead).
// ----------------------------------------------------------------------------
template <typename T, int NB = kMaxN>
__device__ bool write_record(const InstDev& I, int cell, double n, double in, const double* u, double T_,
                             const double* q)
{
    // in = 1 / n (the callers have it); FP64 divisions are costly here, so 1/T is the
    // only other one before R_SCALE
    bool bad = !(n > 0.0) || !(T_ > 0.0) || !isfinite(n) || !isfinite(T_);
    for (int a = 0; a < 3; ++a) bad |= !isfinite(u[a]) || !isfinite(q[a]);
    const double nn = bad ? 1.0 : n, inn = bad ? 1.0 : in, Tc = bad ? 1.0 : T_;
    const double u0 = bad ? 0.0 : u[0], u1 = bad ? 0.0 : u[1], u2 = bad ? 0.0 : u[2];
    T* rec = static_cast<T*>(I.rec) + (size_t)cell * I.rec_stride;
    const double iT = 1.0 / Tc;
    rec[R_N] = T(nn); rec[R_UX] = T(u0); rec[R_UY] = T(u1); rec[R_UZ] = T(u2); rec[R_T] = T(Tc);
    rec[R_QX] = T(bad ? 0.0 : q[0]); rec[R_QY] = T(bad ? 0.0 : q[1]); rec[R_QZ] = T(bad ? 0.0 : q[2]);
    rec[R_ITAU] = T(inv_relax_time(I.visc_law, I.iKn, I.visc_param, I.isuth, nn, Tc, iT));
    rec[R_CS] = T((1.0 - I.Pr) * inn * iT * iT);
    rec[R_I5T] = T(0.2 * iT);
    const int Qx = I.Qx, Qy = I.Qy, Qz = I.Qz;
    T* dx = rec + R_DX;
    T* dy = dx + Qx;
    T* dz = dy + Qy;
    double c[kMaxN + 1], cm[kMaxN + 1], s[3];
    // x: a_l, l >= 1, against He_l / l!
    full_coeffs<NB>(u0, Tc, I.Nx, c);
    s[0] = 0.0;
    if constexpr (sizeof(T) == 4) {  // FP32 records: the node sums in double-float
        DF cd[NB + 1], sw = {0.f, 0.f};
#pragma unroll
        for (int l = 1; l <= NB; ++l) cd[l] = l <= I.Nx ? df_of(c[l]) : DF{0.f, 0.f};
#pragma unroll 2
        for (int i = 0; i < Qx; ++i) {
            const float2* h = I.Hx2 + i * (I.Nx + 1);
            DF g = {0.f, 0.f};
#pragma unroll
            for (int l = 1; l <= NB; ++l)
                if (l <= I.Nx) df_fma(g, cd[l], h[l]);
            const float v = g.hi + g.lo;
            dx[i] = T(v);
            df_add_prod(sw, ld<float>(I.wx, i), v);
        }
        s[0] = I.sumw_x + (double(sw.hi) + double(sw.lo));  // sum w (1 + v)
    } else {
#pragma unroll 4  // independent nodes: four FP64 chains in flight
        for (int i = 0; i < Qx; ++i) {
            const double* h = I.Hx + i * (I.Nx + 1);
            double g = 0.0;
#pragma unroll
            for (int l = 1; l <= NB; ++l)
                if (l <= I.Nx) g += c[l] * h[l];
            const T v = T(g);
            dx[i] = v;
            s[0] += double(ld<T>(I.wx, i)) * (1.0 + double(v));
        }
    }
    // y: the reduced model's factors 1 and T (phi and chi; its mass is phi's alone)
    s[1] = 0.0;
    if (I.reduced) {
        dy[0] = T(0);
        dy[1] = T(Tc - 1.0);
        s[1] = 1.0;
    } else {
        full_coeffs<NB>(u1, Tc, I.Ny, c);
        if constexpr (sizeof(T) == 4) {
            DF cd[NB + 1], sw = {0.f, 0.f};
#pragma unroll
            for (int l = 1; l <= NB; ++l) cd[l] = l <= I.Ny ? df_of(c[l]) : DF{0.f, 0.f};
#pragma unroll 2
            for (int j = 0; j < Qy; ++j) {
                const float2* h = I.Hy2 + j * (I.Ny + 1);
                DF g = {0.f, 0.f};
#pragma unroll
                for (int l = 1; l <= NB; ++l)
                    if (l <= I.Ny) df_fma(g, cd[l], h[l]);
                const float v = g.hi + g.lo;
                dy[j] = T(v);
                df_add_prod(sw, ld<float>(I.wy, j), v);
            }
            s[1] = I.sumw_y + (double(sw.hi) + double(sw.lo));
        } else {
#pragma unroll 4
            for (int j = 0; j < Qy; ++j) {
                const double* h = I.Hy + j * (I.Ny + 1);
                double g = 0.0;
#pragma unroll
                for (int l = 1; l <= NB; ++l)
                    if (l <= I.Ny) g += c[l] * h[l];
                const T v = T(g);
                dy[j] = v;
                s[1] += double(ld<T>(I.wy, j)) * (1.0 + double(v));
            }
        }
    }
    // z: b_l on each half range against pi_l / h_l, b_0 - 1/2 in place of b_0
    half_coeffs_pm<NB>(u2, Tc, iT, I.Nzq, I.alpha, I.beta, c, cm);
    c[0] -= 0.5;
    cm[0] -= 0.5;
    s[2] = 0.0;
    if constexpr (sizeof(T) == 4) {
        DF bp[NB + 1], bm[NB + 1], sw = {0.f, 0.f};
#pragma unroll
        for (int l = 0; l <= NB; ++l) {
            bp[l] = l <= I.Nzq ? df_of(c[l]) : DF{0.f, 0.f};
            bm[l] = l <= I.Nzq ? df_of(cm[l]) : DF{0.f, 0.f};
        }
        for (int m = 0; m < Qz; ++m) {
            const float2* h = I.Pz2 + m * (I.Nzq + 1);
            DF gp = {0.f, 0.f}, gm = {0.f, 0.f};
#pragma unroll
            for (int l = 0; l <= NB; ++l)
                if (l <= I.Nzq) {
                    df_fma(gp, bp[l], h[l]);
                    df_fma(gm, bm[l], h[l]);
                }
            const float vp = gp.hi + gp.lo, vm = gm.hi + gm.lo;
            dz[m] = T(vp);
            dz[Qz + m] = T(vm);
            const float w = ld<float>(I.wz, m);
            df_add_prod(sw, w, vp);
            df_add_prod(sw, w, vm);
        }
        s[2] = I.sumw_z + (double(sw.hi) + double(sw.lo));  // sum over both half ranges
    } else {
#pragma unroll 2
        for (int m = 0; m < Qz; ++m) {
            const double* h = I.Pz + m * (I.Nzq + 1);
            double gp = 0.0, gm = 0.0;
#pragma unroll
            for (int l = 0; l <= NB; ++l)
                if (l <= I.Nzq) {
                    gp += c[l] * h[l];
                    gm += cm[l] * h[l];
                }
            const T vp = T(gp), vm = T(gm);
            dz[m] = vp;
            dz[Qz + m] = vm;
            s[2] += double(ld<T>(I.wz, m)) * ((1.0 + double(vp)) + (1.0 + double(vm)));
        }
    }
    rec[R_SCALE1] = T(nn / (s[0] * s[1] * s[2]) - 1.0);
    return !bad;
}

// profiles [14][Nz] and W = (n, u_x, T) of a cell; false if any value is not finite
static __device__ __forceinline__ bool store_cell(const InstDev& I, int cell, const CellState& c)
{
    const int Nz = I.Nz;
    const double vals[14] = {c.n, c.u[0], c.u[1], c.u[2], c.T, c.q[0], c.q[1], c.q[2],
                             c.P[0], c.P[1], c.P[2], c.P[3], c.P[4], c.P[5]};
    bool bad = false;
#pragma unroll
    for (int a = 0; a < 14; ++a) {
        I.prof[(size_t)a * Nz + cell] = vals[a];
        bad |= !isfinite(vals[a]);
    }
    I.Wnew[cell] = c.n;
    I.Wnew[Nz + cell] = c.u[0];
    I.Wnew[2 * Nz + cell] = c.T;
    return !bad;
}

// The velocity the stage kernel took its moments about: the u of the cell's record of
// the stage (still in place when the finalisation reads it); 0 for the analysis pass.
template <typename T>
__device__ __forceinline__ void moment_origin(const InstDev& I, int cell, int stage, double* ur)
{
    const T* rc = static_cast<const T*>(I.rec) + (size_t)cell * I.rec_stride;
    ur[0] = stage > 0 ? double(rc[R_UX]) : 0.0;
    ur[1] = stage > 0 ? double(rc[R_UY]) : 0.0;
    ur[2] = stage > 0 ? double(rc[R_UZ]) : 0.0;
}

// The macroscopic state from the partials' moments about ur (sums over the deviations
// d) and the rest state's moments, re-expressed about ur: n, u = ur + the mean of
// p - ur, P, T and q.
static __device__ __forceinline__ void state_about(const InstDev& I, double* mom, const double* ur, CellState& st)
{
    double rest[kNMom];
    shift_moments(I.mrest, ur, rest);
#pragma unroll
    for (int a = 0; a < kNMom; ++a) mom[a] += rest[a];
    cell_state(mom, st);
#pragma unroll
    for (int a = 0; a < 3; ++a) st.u[a] += ur[a];
}

// One cell (one thread): the sum of the per-chunk moment partials (written by other
// CTAs of this launch, hence read past L1; FP32 partials in double-float, FP64 ones in
// FP64), the macroscopic state, the profiles, W for the residual, and the cell record
// of the next stage.
template <typename T, int NB = kMaxN>
__device__ __noinline__ void finalize_cell(const InstDev& I, int cell, int stage)
{
    const int Nz = I.Nz, nch = I.nchunks;
    typedef typename Acc<T>::type A;
    const A* part = static_cast<const A*>(I.partial);
    double mom[kNMom];  // the partials: moments of the deviations about ur
    // chunks in order, four at a time with every load issued before the adds (the
    // partials come from L2: one round trip per four chunks instead of per chunk);
    // FP32 partials summed in double-float (no FP64 instruction per chunk)
    DF md[kNMom];
    for (int a = 0; a < kNMom; ++a) {
        mom[a] = 0.0;
        md[a] = DF{0.f, 0.f};
    }
    for (int c = 0; c < nch; c += 4) {
        A p[4][kNMom];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int a = 0; a < kNMom; ++a)
                p[j][a] = c + j < nch ? __ldcg(part + ((size_t)(c + j) * kNMom + a) * Nz + cell) : A(0);
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int a = 0; a < kNMom; ++a)
                if (c + j < nch) {
                    if constexpr (sizeof(A) == 4) df_add(md[a], p[j][a], 0.f);
                    else mom[a] += p[j][a];
                }
    }
    if constexpr (sizeof(A) == 4)
        for (int a = 0; a < kNMom; ++a) mom[a] = double(md[a].hi) + double(md[a].lo);
    double ur[3];
    moment_origin<T>(I, cell, stage, ur);
    CellState st;
    state_about(I, mom, ur, st);
    bool bad = !store_cell(I, cell, st);
    bad |= !write_record<T, NB>(I, cell, st.n, st.in, st.u, st.T, st.q);
    if (bad) atomicOr(I.status, STATUS_NONFINITE);
}

// ---- one cell per warp: the same record with its FP64 work spread over the lanes.
// FP64 instructions issue at a small fraction of the FP32 rate, so with one thread
// per cell a small batch waits on each cell's long FP64 chain; here lane a sums
// moment a, the two halves of the warp run the x / y coefficient recurrences and
// the p_z > 0 / p_z < 0 half-range tables side by side, within a half lane k
// carries column k of the table J_{l,k} (one shuffle per row instead of the whole
// triangle in one thread), and the nodes' factors are spread over the lanes.  Large
// batches keep one thread per cell, where every lane has a cell of its own.
template <typename T>
__device__ bool write_record_warp(const InstDev& I, int cell, const CellState& st, int lane)
{
    // the half-range recurrence coefficients, loaded ahead of the chain that needs them
    double al[kMaxN], be[kMaxN];
#pragma unroll
    for (int l = 0; l < kMaxN; ++l) {
        al[l] = I.alpha[l];
        be[l] = I.beta[l];
    }
    bool bad = !(st.n > 0.0) || !(st.T > 0.0) || !isfinite(st.n) || !isfinite(st.T);
    for (int a = 0; a < 3; ++a) bad |= !isfinite(st.u[a]) || !isfinite(st.q[a]);
    const double nn = bad ? 1.0 : st.n, inn = bad ? 1.0 : st.in, Tc = bad ? 1.0 : st.T;
    const double u0 = bad ? 0.0 : st.u[0], u1 = bad ? 0.0 : st.u[1], u2 = bad ? 0.0 : st.u[2];
    T* rec = static_cast<T*>(I.rec) + (size_t)cell * I.rec_stride;
    const double iT = 1.0 / Tc;
    if (lane == 0) {
        rec[R_N] = T(nn); rec[R_UX] = T(u0); rec[R_UY] = T(u1); rec[R_UZ] = T(u2); rec[R_T] = T(Tc);
        rec[R_QX] = T(bad ? 0.0 : st.q[0]); rec[R_QY] = T(bad ? 0.0 : st.q[1]); rec[R_QZ] = T(bad ? 0.0 : st.q[2]);
        rec[R_ITAU] = T(inv_relax_time(I.visc_law, I.iKn, I.visc_param, I.isuth, nn, Tc, iT));
        rec[R_CS] = T((1.0 - I.Pr) * inn * iT * iT);
        rec[R_I5T] = T(0.2 * iT);
    }
    const int Qx = I.Qx, Qy = I.Qy, Qz = I.Qz;
    T* dx = rec + R_DX;
    T* dy = dx + Qx;
    T* dz = dy + Qy;
    const int h = lane >> 4, k = lane & 15;  // half of the warp, lane within it
    // x (h = 0) and y (h = 1) coefficients a_l (Eq. fyz), in every lane of the half
    double c[kMaxN + 1];
    const int Nh = h ? I.Ny : I.Nx;
    full_coeffs(h ? u1 : u0, Tc, Nh, c);
    // z: half h = 0 the p_z > 0 range (drift u2), h = 1 the p_z < 0 range written in
    // xi = -p_z >= 0 (drift -u2).  Both share g(0) and one erfc (erfc(x) + erfc(-x) = 2).
    const int K = I.Nzq;
    // 1 / sqrt(2T) straight from T, so that the transcendental chain does not wait for
    // the division 1 / T; with x = |u2| / sqrt(2T): g(0) = exp(-x^2) / sqrt(2 pi T)
    const double r2T = rsqrt(2.0 * Tc), x = fabs(u2) * r2T;
    const double g0 = exp(-x * x) * (r2T * (1.0 / sqrt(M_PI)));
    const double e = erfc_nonneg(x);
    const double us = h ? -u2 : u2;
    const double J00 = (u2 >= 0.0) != (h == 1) ? 1.0 - 0.5 * e : 0.5 * e;  // erfc(-us / sqrt(2T)) / 2
    // J_{0,k}: the half-line Gaussian moments M_k, M_{k+1} = us M_k + k T M_{k-1}
    double mp = J00, mc = us * J00 + Tc * g0;
    double Jc = k == 0 ? J00 : (k == 1 ? mc : 0.0);
#pragma unroll
    for (int kk = 1; kk < kMaxN; ++kk)
        if (kk < K) {
            const double mn = us * mc + kk * Tc * mp;
            mp = mc;
            mc = mn;
            if (k == kk + 1) Jc = mn;
        }
    // rows J_{l+1,k} = J_{l,k+1} - alpha_l J_{l,k} - beta_l J_{l-1,k}; b_l = J_{l,0}.
    // Column k holds a valid entry for k <= K - l; the others never reach column 0.
    double Jp = 0.0, b[kMaxN + 1];
    b[0] = Jc;
#pragma unroll
    for (int l = 0; l < kMaxN; ++l) {
        b[l + 1] = 0.0;
        if (l < K) {
            const double up = __shfl_down_sync(0xffffffffu, Jc, 1, 16);
            const double Jn = up - al[l] * Jc - (l > 0 ? be[l] * Jp : 0.0);
            Jp = Jc;
            Jc = Jn;
            b[l + 1] = Jc;
        }
    }
    // column 0 (lanes 0 and 16) holds the two coefficient sets: give them to every lane,
    // b_0 - 1/2 in place of b_0 (the rest state's coefficient)
    double bp[kMaxN + 1], bm[kMaxN + 1];
#pragma unroll
    for (int l = 0; l <= kMaxN; ++l) {
        bp[l] = __shfl_sync(0xffffffffu, b[l], 0) - (l == 0 ? 0.5 : 0.0);
        bm[l] = __shfl_sync(0xffffffffu, b[l], 16) - (l == 0 ? 0.5 : 0.0);
    }
    // the nodes' factors: x over the lanes of half 0, y over half 1, z over the warp;
    // each lane's terms of the R_SCALE sums
    double sxy = 0.0, sz = 0.0;
    if (h == 0) {
        for (int i = k; i < Qx; i += 16) {
            const double* hb = I.Hx + i * (I.Nx + 1);
            double g = 0.0;
#pragma unroll
            for (int l = 1; l <= kMaxN; ++l)
                if (l <= I.Nx) g += c[l] * hb[l];
            const T v = T(g);
            dx[i] = v;
            sxy += double(ld<T>(I.wx, i)) * (1.0 + double(v));
        }
    } else if (I.reduced) {  // y factors of phi and chi: 1 and T; the mass is phi's alone
        if (k == 0) {
            dy[0] = T(0);
            dy[1] = T(Tc - 1.0);
            sxy = 1.0;
        }
    } else {
        for (int j = k; j < Qy; j += 16) {
            const double* hb = I.Hy + j * (I.Ny + 1);
            double g = 0.0;
#pragma unroll
            for (int l = 1; l <= kMaxN; ++l)
                if (l <= I.Ny) g += c[l] * hb[l];
            const T v = T(g);
            dy[j] = v;
            sxy += double(ld<T>(I.wy, j)) * (1.0 + double(v));
        }
    }
    for (int m = lane; m < Qz; m += 32) {
        const double* hb = I.Pz + m * (I.Nzq + 1);
        double gp = 0.0, gm = 0.0;
#pragma unroll
        for (int l = 0; l <= kMaxN; ++l)
            if (l <= K) {
                gp += bp[l] * hb[l];
                gm += bm[l] * hb[l];
            }
        const T vp = T(gp), vm = T(gm);
        dz[m] = vp;
        dz[Qz + m] = vm;
        sz += double(ld<T>(I.wz, m)) * ((1.0 + double(vp)) + (1.0 + double(vm)));
    }
    // R_SCALE = n / (s_x s_y s_z) (see write_record)
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) sxy += __shfl_xor_sync(0xffffffffu, sxy, o, 16);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sz += __shfl_xor_sync(0xffffffffu, sz, o);
    const double sx = __shfl_sync(0xffffffffu, sxy, 0), sy = __shfl_sync(0xffffffffu, sxy, 16);
    if (lane == 0) rec[R_SCALE1] = T(nn / (sx * sy * sz) - 1.0);
    return !bad;
}

template <typename T>
__device__ __noinline__ void finalize_cell_warp(const InstDev& I, int cell, int lane, int stage)
{
    const int Nz = I.Nz, nch = I.nchunks, am = lane & 15, h = lane >> 4;
    // moment am: lanes am and 16 + am sum the even and the odd chunks (loads four
    // chunks ahead), then add the two halves
    double part = 0.0;
    if (am < kNMom)
        for (int c = h; c < nch; c += 8) {
            double p[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                p[j] = c + 2 * j < nch
                           ? double(__ldcg(static_cast<const typename Acc<T>::type*>(I.partial) +
                                           ((size_t)(c + 2 * j) * kNMom + am) * Nz + cell))
                           : 0.0;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (c + 2 * j < nch) part += p[j];
        }
    part += __shfl_down_sync(0xffffffffu, part, 16);
    double mom[kNMom];
#pragma unroll
    for (int a = 0; a < kNMom; ++a) mom[a] = __shfl_sync(0xffffffffu, part, a);
    double ur[3];
    moment_origin<T>(I, cell, stage, ur);
    CellState st;
    state_about(I, mom, ur, st);
    bool bad = false;
    if (lane == 0) bad = !store_cell(I, cell, st);
    bad |= !write_record_warp<T>(I, cell, st, lane);
    if (bad && lane == 0) atomicOr(I.status, STATUS_NONFINITE);
}

// One instance (whole CTA): wall densities n_w from the outgoing wall fluxes
// (zero net mass flux, Appendix); after stage 3 the residual, the step count
// and retirement; after the analysis pass W_old = W.
static __device__ __noinline__ void finalize_instance(const InstDev& I, int stage, double* red)
{
    // red: kRedSlots doubles.  The wall fluxes and (stage 3) the residual's sums
    // ||W_new - W_old||^2, ||W_old||^2 for n, u_x, T are reduced together.
    const int t = threadIdx.x, Nz = I.Nz;
    double v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = 0.0;
    for (int c = t; c < I.nchunks; c += blockDim.x) {
        v[0] += __ldcg(I.flux_part + 2 * c);
        v[1] += __ldcg(I.flux_part + 2 * c + 1);
    }
    if (stage == 3) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
            for (int s = t; s < Nz; s += blockDim.x) {
                const double wn = __ldcg(I.Wnew + a * Nz + s), wo = I.Wold[a * Nz + s];
                v[2 + 2 * a] += (wn - wo) * (wn - wo);
                v[3 + 2 * a] += wo * wo;
            }
        block_sum_n<8>(v, red);
    } else {
        double w[2] = {v[0], v[1]};
        block_sum_n<2>(w, red);
        v[0] = w[0];
        v[1] = w[1];
    }
    if (t == 0) {  // the partials sum w p_z over the deviations: add the rest state's flux
        I.nw[0] = -(I.frest_bot + v[0]) / I.Dbot;
        I.nw[1] = -(I.frest_top + v[1]) / I.Dtop;
        if (!isfinite(I.nw[0]) || !isfinite(I.nw[1])) atomicOr(I.status, STATUS_NONFINITE);
    }
    if (stage == 3) {
        double R = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a)  // the velocity on the wall speed where u_x is smaller
            R = fmax(R, sqrt(v[2 + 2 * a]) / fmax(sqrt(v[3 + 2 * a]), a == 1 ? I.res_uscale : 1e-30));
        // every W_old read above is complete (block_sum_n ends with a barrier)
        for (int e = t; e < 3 * Nz; e += blockDim.x) I.Wold[e] = __ldcg(I.Wnew + e);
        if (t == 0) {
            *I.res = R;
            *I.steps += 1;
            *I.cur ^= 1;  // the new state was written over the stage-1 increment
            if (!(R == R)) atomicOr(I.status, STATUS_NONFINITE);
            if (I.tol > 0.0 && R < I.tol) *I.active = 0;
        }
    } else if (stage == 0) {
        for (int e = t; e < 3 * Nz; e += blockDim.x) I.Wold[e] = __ldcg(I.Wnew + e);
    }
}

// records from given macroscopic profiles macro[8][Nz] = n, ux, uy, uz, T, qx, qy, qz
template <typename T>
__global__ void records_from_macro(const InstDev* __restrict__ insts, int inst, const double* __restrict__ macro)
{
    const InstDev& I = insts[inst];
    const int Nz = I.Nz, cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= Nz) return;
    const double u[3] = {macro[Nz + cell], macro[2 * Nz + cell], macro[3 * Nz + cell]};
    const double q[3] = {macro[5 * Nz + cell], macro[6 * Nz + cell], macro[7 * Nz + cell]};
    if (!write_record<T>(I, cell, macro[cell], 1.0 / macro[cell], u, macro[4 * Nz + cell], q))
        atomicOr(I.status, STATUS_NONFINITE);
}

// The instance descriptor copied into shared memory by the whole block at once: its
// fields (pointers, orders, wall sums) are then one shared load away instead of an
// L2 round trip each at first use -- in the stage kernel's prologue (pointer, then
// table, then value) and inside the finalisation's FP64 chains.
static __device__ __forceinline__ const InstDev& stage_descriptor(const InstDev* g, InstDev* s)
{
    static_assert(sizeof(InstDev) % 8 == 0, "descriptor copied in 8-byte words");
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(g);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(s);
    for (int e = threadIdx.x; e < (int)(sizeof(InstDev) / 8); e += blockDim.x) dst[e] = src[e];
    __syncthreads();
    return *s;
}

// ----------------------------------------------------------------------------
// stage_kernel<T, V, STAGE, RED>: STAGE 1..3 are the RK stages; STAGE 0 only
// analyses F0 (moments and wall fluxes) without writing F.  RED selects the
// phi / chi model (Sec. III, Eqs. boltz_red, sred_def): j = 0 is phi, j = 1 chi.
// ----------------------------------------------------------------------------
// Minimum resident CTAs per SM requested from the register allocator: the
// per-velocity register window grows with V; the rarely taken finalisation
// path may spill instead of lowering occupancy.
template <typename T, int V> struct MinBlocks {
    // FP32 at V = 4 fits 128 registers (four CTAs, sixteen warps per SM); FP64 values take
    // two registers each and keep three
    static constexpr int value = V == 1 ? 8 : V == 2 ? 6 : sizeof(T) == 4 ? 4 : 3;
};

template <typename T, int V, int STAGE, bool RED>
__global__ void __launch_bounds__(kThreads, MinBlocks<T, V>::value)
stage_kernel(const InstDev* __restrict__ insts, const Tile* __restrict__ tiles, int fuse)
{
    typedef typename Acc<T>::type A;
    constexpr bool kLo = sizeof(T) == 4;  // FP32 storage keeps the rounding residual of d
    constexpr bool kD = STAGE >= 2;       // the stage input is d + an increment
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ double wall_red[kRedSlots];
    __shared__ InstDev sI;
    const Tile tile = tiles[blockIdx.x];
    const InstDev& I = stage_descriptor(insts + tile.inst, &sI);
    if (*I.active == 0) return;
    const int cur = *I.cur;  // which of F0 / F1 holds the step's start state

    const int Nz = I.Nz, Q = I.Q, Qx = I.Qx, Qy = I.Qy, Qz = I.Qz, QxQy = I.QxQy;
    const int z0 = tile.z0, zn = tile.zn;            // cells z0 .. z0+zn-1 (0-based)
    constexpr int KC = kThreads * V;
    // chunks never straddle p_z = 0: this chunk's velocities share the sign of p_z
    const int Qh = Q >> 1, sgc = tile.chunk >= I.nchh;
    const int k0 = sgc * Qh + (tile.chunk - sgc * I.nchh) * KC;
    const int kend = min((sgc + 1) * Qh, k0 + KC), kn = kend - k0;
    const int zm_lo = k0 / QxQy, zm_hi = (kend - 1) / QxQy, nzm = zm_hi - zm_lo + 1;
    const int G = Qx + Qy + nzm;                     // per-cell factors held in smem
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int rstride = I.rec_stride;
    const StageSmem L = stage_smem(zn, KC, G, sizeof(T), sizeof(A), rstride);
    T* Fs = reinterpret_cast<T*>(smem_raw + L.fin);   // d rows: cells z0-3 .. z0+zn+2
    T* recs = reinterpret_cast<T*>(smem_raw + L.rec); // records of cells z0 .. z0+zn-1
    T* gsm = reinterpret_cast<T*>(smem_raw + L.g);
    T* idzs = reinterpret_cast<T*>(smem_raw + L.idz);
    A* red = reinterpret_cast<A*>(smem_raw + L.red);  // per-warp moment sums

    // Buffers (Eq. rk3 in increment form, F_l the step's start state d):
    //   stage 1: d1 = dt L[F_l]                  -> the other of F0 / F1
    //   stage 2: d2 = (d1 + dt L[F_l + d1]) / 4  -> F2
    //   stage 3: F_l + 2/3 (d2 + dt L[F_l + d2]) -> the other of F0 / F1 (over d1)
    const T* Hg = static_cast<const T*>(cur ? I.F1 : I.F0);
    T* Og = static_cast<T*>(cur ? I.F0 : I.F1);
    // the stage input's increment (stages 2, 3) is read from global memory through the
    // read-only path (this launch does not write it), one march step ahead
    const T* __restrict__ Dg = STAGE == 2 ? Og : static_cast<const T*>(I.F2);
    T* Fout = STAGE == 2 ? static_cast<T*>(I.F2) : Og;
    const int s_lo = max(0, z0 - 3), s_hi = min(Nz - 1, z0 + zn + 2);

    // ---- 1. stage the input rows and the cell records (TMA bulk copies; plain loads
    //         if the rows are not 16-byte aligned)
    const T* Rg = static_cast<const T*>(I.rec) + (size_t)z0 * rstride;
    const size_t rec_bytes = (size_t)zn * rstride * sizeof(T);
    if (I.bulk) {
        if (tid == 0) {
            mbar_init(&bar, 1);
            fence_barrier_init();
        }
        __syncthreads();
        if (tid == 0) {
            const uint32_t bytes = kn * sizeof(T);
            uint32_t total = bytes * (s_hi - s_lo + 1);
            if (STAGE > 0) total += rec_bytes;
            mbar_expect_tx(&bar, total);
            for (int s = s_lo; s <= s_hi; ++s)
                bulk_g2s(Fs + (size_t)(s - z0 + 3) * KC, Hg + (size_t)s * Q + k0, bytes, &bar);
            if (STAGE > 0) bulk_g2s(recs, Rg, rec_bytes, &bar);  // records are 16-byte multiples
        }
    } else {
        for (int s = s_lo; s <= s_hi; ++s)
            for (int kl = tid; kl < kn; kl += kThreads) Fs[(size_t)(s - z0 + 3) * KC + kl] = Hg[(size_t)s * Q + k0 + kl];
        if (STAGE > 0)
            for (int e = tid; e < zn * rstride; e += kThreads) recs[e] = Rg[e];
    }
    if (STAGE > 0)
        for (int c = tid; c < zn; c += kThreads) idzs[c] = ld<T>(I.inv_dz, z0 + c);

    // per-velocity constants: p (and |p_z| for the fluxes), the weight w and |p|^2 for the
    // moments (formed from them per cell: fewer registers than 13 weighted monomials)
    // FP32 with an even V: the thread's velocities are adjacent pairs (2 tid, 2 tid + 1,
    // 2 tid + 2 kThreads, ...), so that a pair is one 64-bit word in memory and one
    // operand of the packed FP32 instructions; else tid + v kThreads.  voff(v) is v's
    // offset from the thread's first velocity tbase.
    constexpr bool kPair = sizeof(T) == 4 && V % 2 == 0;
    const int tbase = kPair ? 2 * tid : tid;
    auto voff = [](int v) { return kPair ? (v & 1) + (v >> 1) * 2 * kThreads : v * kThreads; };
    int ii[V], jj[V], zz[V], kl[V];
    T px[V], py[V], pz[V], apz[V];
    A wv[V], yv[V], p2v[V], wm[V];  // weight; p_y for the moments; |p|^2; w of the mass flux
    bool ok[V], chi[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        kl[v] = tbase + voff(v);
        ok[v] = kl[v] < kn;
        const int kc = ok[v] ? k0 + kl[v] : kend - 1;
        jj[v] = kc % Qy;
        ii[v] = (kc / Qy) % Qx;
        zz[v] = kc / QxQy;
        const int sg = zz[v] >= Qz, m = zz[v] - sg * Qz;
        px[v] = ld<T>(I.px, ii[v]);
        py[v] = ld<T>(I.py, jj[v]);
        const T x = ld<T>(I.xi, m);
        pz[v] = sg ? -x : x;
        apz[v] = x;
        wv[v] = ok[v] ? A(ld<T>(I.wx, ii[v]) * ld<T>(I.wy, jj[v]) * ld<T>(I.wz, m)) : A(0);
        const A X = px[v], Y = py[v], Z = pz[v];
        yv[v] = Y;
        p2v[v] = X * X + Y * Y + Z * Z;
        chi[v] = RED && jj[v] == 1;
        wm[v] = chi[v] ? A(0) : wv[v];
        if (RED) {
            // p_y = 0 on both fields.  chi = int p_y^2 f dp_y carries the p_y^2 moments:
            // sum chi -> sum p_y^2 f, sum p_a chi -> sum p_y^2 p_a f (a = x, z), nothing else.
            // py[v] then holds -(the Shakhov offset of Eq. sred_def): -4/5 for phi, -2/5 for chi.
            py[v] = jj[v] ? T(-0.4) : T(-0.8);
        }
    }

    // ---- 3. wait for the copies (bounded).  A CTA whose wait runs out flags the
    //         instance (STATUS_TIMEOUT), then waits a further bounded time for its copies
    //         in flight to land before it leaves, so that none writes shared memory after
    //         the CTA is gone; if that wait runs out too the CTA leaves regardless.
    int late = 0;
    if (I.bulk) {
        for (uint32_t spins = 0;; ++spins) {
            if (spins >= I.wait_limit) { late = 1; break; }
            if (mbar_try_wait(&bar, 0)) break;
        }
    }
    if (__syncthreads_or(late)) {
        if (tid == 0) atomicOr(I.status, STATUS_TIMEOUT);
        uint32_t spins = 0;
        while (!mbar_try_wait(&bar, 0) && ++spins < kDrainLimit) {
        }
        return;
    }

    // ---- 4a. per-cell factors of the truncated Hermite equilibrium (Sec. III) for this
    //          chunk's nodes, as deviations from 1, from the staged records:
    //          dx[i] with R_SCALE applied (R_SCALE (1 + dx) - 1), dy[j], dz[zm]
    if (STAGE > 0) {
        for (int e = tid; e < zn * G; e += kThreads) {
            const int c = e / G, r = e - c * G;
            const T* rc = recs + (size_t)c * rstride;
            T g;
            if (r < Qx) {
                const T s1 = rc[R_SCALE1];
                g = s1 + (T(1) + s1) * rc[R_DX + r];
            } else if (r < Qx + Qy) {
                g = rc[R_DX + r];                               // dy[r - Qx]
            } else {
                g = rc[R_DX + Qx + Qy + zm_lo + r - Qx - Qy];   // dz[zm]
            }
            gsm[e] = g;
        }
    }

    // ---- 4b. ghost rows (each thread fills only its own columns).  A ghost row holds
    //          the whole stage-input value d (+ increment); a cell's row holds d.
    const int rbase = 3 - z0;  // smem row of cell s is s + rbase
    auto rowval = [&](int row, int col) -> T {  // the stage input of a cell's row
        return kD ? Fs[(size_t)row * KC + col] + __ldg(Dg + (size_t)(row - rbase) * Q + k0 + col)
                  : Fs[(size_t)row * KC + col];
    };
#pragma unroll
    for (int v = 0; v < V; ++v) {
        if (!ok[v]) continue;  // columns past the chunk end hold no data
        T* col = Fs + kl[v];
        if (z0 < 3 && I.half) {  // bounce-back on the centre line: ghost -1-s holds cell s
            // at the mirrored velocity (p_z, p_x reversed: other half range, node Qx-1-i;
            // the Gauss nodes are sorted, so p_x[Qx-1-i] = -p_x[i]).  It lies in the other
            // sign's chunk, so it comes from the stage input in global memory.
            const int zm = zz[v] + (sgc ? -Qz : Qz);
            const int kmir = (zm * Qx + (Qx - 1 - ii[v])) * Qy + jj[v];
            for (int s = 0; s < 3; ++s)
                if (-1 - s + rbase >= 0)
                    col[(size_t)(-1 - s + rbase) * KC] =
                        kD ? Hg[(size_t)s * Q + kmir] + Dg[(size_t)s * Q + kmir] : Hg[(size_t)s * Q + kmir];
        } else if (z0 < 3) {
            if (!sgc) {  // incoming at the bottom wall: n_w times the wall equilibrium, minus 1
                const T ax = ld<T>(I.gwx_bot, ii[v]), ay = ld<T>(I.gwy, jj[v]), az = ld<T>(I.gwz, zz[v]);
                const T a = ax + ay + ax * ay, b = a + az + a * az;
                const T g = T(I.nw[0] - 1.0) + T(I.nw[0]) * b;
                for (int s = -3; s <= -1; ++s)
                    if (s + rbase >= 0) col[(size_t)(s + rbase) * KC] = g;
            } else {      // outgoing: quadratic extrapolation (Appendix)
                const T f1 = rowval(0 + rbase, kl[v]), f2 = rowval(1 + rbase, kl[v]), f3 = rowval(2 + rbase, kl[v]);
                const T g0 = T(I.ext_bot[0][0]) * f1 + T(I.ext_bot[0][1]) * f2 + T(I.ext_bot[0][2]) * f3;
                const T g1 = T(I.ext_bot[1][0]) * g0 + T(I.ext_bot[1][1]) * f1 + T(I.ext_bot[1][2]) * f2;
                if (-1 + rbase >= 0) col[(size_t)(-1 + rbase) * KC] = g0;
                if (-2 + rbase >= 0) col[(size_t)(-2 + rbase) * KC] = g1;
                if (-3 + rbase >= 0) col[(size_t)(-3 + rbase) * KC] = g1;  // never read for p_z < 0
            }
        }
        if (z0 + zn + 3 > Nz) {
            const int smax = z0 + zn + 2;
            if (sgc) {
                const T ax = ld<T>(I.gwx_top, ii[v]), ay = ld<T>(I.gwy, jj[v]), az = ld<T>(I.gwz, zz[v]);
                const T a = ax + ay + ax * ay, b = a + az + a * az;
                const T g = T(I.nw[1] - 1.0) + T(I.nw[1]) * b;
                for (int s = Nz; s <= Nz + 2; ++s)
                    if (s <= smax) col[(size_t)(s + rbase) * KC] = g;
            } else {
                const T f1 = rowval(Nz - 1 + rbase, kl[v]), f2 = rowval(Nz - 2 + rbase, kl[v]),
                        f3 = rowval(Nz - 3 + rbase, kl[v]);
                const T g0 = T(I.ext_top[0][0]) * f1 + T(I.ext_top[0][1]) * f2 + T(I.ext_top[0][2]) * f3;
                const T g1 = T(I.ext_top[1][0]) * g0 + T(I.ext_top[1][1]) * f1 + T(I.ext_top[1][2]) * f2;
                if (Nz <= smax) col[(size_t)(Nz + rbase) * KC] = g0;
                if (Nz + 1 <= smax) col[(size_t)(Nz + 1 + rbase) * KC] = g1;
                if (Nz + 2 <= smax) col[(size_t)(Nz + 2 + rbase) * KC] = g1;  // never read for p_z > 0
            }
        }
    }

    __syncthreads();  // per-cell factors complete

    if constexpr (kPair && !RED) {
        // ---- 5 (FP32, full model). The march of section 5 below with the thread's
        // velocities as adjacent pairs: the same operations, two velocities per packed
        // FP32 instruction; rows, increments and outputs move as 64-bit pairs and the two
        // 16-bit residuals of a pair as one 32-bit word.  Q / 2 is even (the host's
        // condition for this layout), so a chunk start k0 and its length kn are even, a
        // pair lies wholly inside or wholly past the chunk, and every pair address is
        // 8-byte aligned.
        constexpr int NP = V / 2;
        const long rstep2 = sgc ? -(long)(KC / 2) : (long)(KC / 2);  // a row, in pairs
        const float2* rp2 = reinterpret_cast<const float2*>(Fs + (sgc ? (size_t)(zn + 5) * KC : 0)) + tid;
        const int sdir = sgc ? -1 : 1;
        const int zw0 = sgc ? z0 + zn + 2 : z0 - 3;  // the cell of window row 0 at step 0
        const float* __restrict__ Dgf = reinterpret_cast<const float*>(Dg);
        // the increments of the cell of a window row (zero for a ghost row)
        auto inc_row2 = [&](int s, float2(&out)[NP]) {
            const bool in = kD && (unsigned)s < (unsigned)Nz;
            const float2* q = reinterpret_cast<const float2*>(Dgf + (long)s * Q + k0) + tid;
#pragma unroll
            for (int p = 0; p < NP; ++p) out[p] = in && ok[2 * p] ? __ldg(q + p * kThreads) : make_float2(0.f, 0.f);
        };
        float2 PX[NP], PY[NP], PZ[NP], NAPZ[NP], WV[NP];  // per pair: p, -|p_z|, weights
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            PX[p] = make_float2(px[2 * p], px[2 * p + 1]);
            PY[p] = make_float2(py[2 * p], py[2 * p + 1]);
            PZ[p] = make_float2(pz[2 * p], pz[2 * p + 1]);
            NAPZ[p] = make_float2(-apz[2 * p], -apz[2 * p + 1]);
            WV[p] = make_float2(wv[2 * p], wv[2 * p + 1]);
        }
        float2 W[NP][6], CM[NP], DN[NP], DIN[NP];
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            inc_row2(zw0 + d * sdir, DN);
#pragma unroll
            for (int p = 0; p < NP; ++p) W[p][d] = add2(rp2[d * rstep2 + p * kThreads], DN[p]);
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) CM[p] = weno5_corr2(W[p][0], W[p][1], W[p][2], W[p][3], W[p][4]);
        int sn = zw0 + 6 * sdir;
        inc_row2(sn, DN);
        // the increments' row of cell sn as a running offset in pairs (one add per march
        // step instead of the row's product; a pointer is formed only inside the channel)
        const float2* __restrict__ dbase = reinterpret_cast<const float2*>(Dgf + k0) + tid;
        long doff = (long)sn * (Q / 2);
        const long dstep = sdir * (long)(Q / 2);
        const float2 DT = splat(float(I.dt));
        const long ostep2 = sgc ? -(long)(Q / 2) : (long)(Q / 2);
        const size_t orow0 = (size_t)(sgc ? z0 + zn - 1 : z0) * Q + k0 + tbase;
        float2* outp = reinterpret_cast<float2*>(reinterpret_cast<float*>(Fout) + orow0);
        const float2* __restrict__ dop = kD ? reinterpret_cast<const float2*>(Dgf + orow0) : nullptr;
        unsigned* lop = kLo && STAGE == 3 ? reinterpret_cast<unsigned*>(I.L0 + orow0) : nullptr;
        unsigned LQN[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            LQN[p] = kLo && STAGE == 3 && ok[2 * p] ? __ldcg(lop + p * kThreads) : 0u;
            DIN[p] = kD && ok[2 * p] ? __ldg(dop + p * kThreads) : make_float2(0.f, 0.f);
        }
        // stage 1 unrolled by two steps (the window's shift halves; 80 vs 86 us on 64 x C2);
        // stages 2 and 3, with their increment and residual streams, lose by unrolling
#pragma unroll(STAGE == 1 ? 2 : 1)
        for (int c = 0; c < zn; ++c) {
            unsigned LQC[NP];
            float2 DC[NP], DIC[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                LQC[p] = LQN[p];
                if (kLo && STAGE == 3 && ok[2 * p] && c + 1 < zn) LQN[p] = __ldcg(lop + ostep2 + p * kThreads);
                DIC[p] = DIN[p];
                if (kD && ok[2 * p] && c + 1 < zn) DIN[p] = __ldg(dop + ostep2 + p * kThreads);
                DC[p] = DN[p];
            }
            if (kD && c + 1 < zn) {
                sn += sdir;
                doff += dstep;
                const bool in = (unsigned)sn < (unsigned)Nz;
#pragma unroll
                for (int p = 0; p < NP; ++p)
                    DN[p] = in && ok[2 * p] ? __ldg(dbase + doff + p * kThreads) : make_float2(0.f, 0.f);
            }
            const int cc = sgc ? zn - 1 - c : c;
            const float* sc = reinterpret_cast<const float*>(recs) + (size_t)cc * rstride;
            const float* gc = reinterpret_cast<const float*>(gsm) + cc * G;
            const float2* rn2 = rp2 + (c + 6) * rstep2;
            const float2* own2 = reinterpret_cast<const float2*>(Fs + (size_t)(cc + 3) * KC) + tid;
            float2 UX, UY, UZ, QX, QY, QZ, NITAU, CS, I5T, IDZ;
            if (STAGE > 0) {
                UX = splat(sc[R_UX]); UY = splat(sc[R_UY]); UZ = splat(sc[R_UZ]);
                QX = splat(sc[R_QX]); QY = splat(sc[R_QY]); QZ = splat(sc[R_QZ]);
                NITAU = splat(-sc[R_ITAU]); CS = splat(sc[R_CS]); I5T = splat(sc[R_I5T]);
                IDZ = splat(float(idzs[cc]));
            }
            float2 S2[kNMom];  // the thread's moment sums, one lane per velocity of a pair
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int v0 = 2 * p, v1 = v0 + 1;
                const float2 f = W[p][3];
                float2 out = f, X = PX[p], Y = PY[p], Z = PZ[p], P2;
                if (STAGE > 0) {
                    const float2 cp = weno5_corr2(W[p][1], W[p][2], W[p][3], W[p][4], W[p][5]);
                    // the Shakhov target's deviation from 1, (1 + dx)(1 + dy)(1 + dz)(1 + S) - 1
                    X = sub2(PX[p], UX);
                    Y = sub2(PY[p], UY);
                    Z = sub2(PZ[p], UZ);
                    P2 = fma2(Z, Z, fma2(Y, Y, mul2(X, X)));
                    const float2 xq = fma2(Z, QZ, fma2(Y, QY, mul2(X, QX)));
                    const float2 S = mul2(mul2(CS, fma2(P2, I5T, splat(-1.f))), xq);
                    const float2 DXf = make_float2(gc[ii[v0]], gc[ii[v1]]);
                    const float2 DYf = make_float2(gc[Qx + jj[v0]], gc[Qx + jj[v1]]);
                    const float2 DZf = make_float2(gc[Qx + Qy + zz[v0] - zm_lo], gc[Qx + Qy + zz[v1] - zm_lo]);
                    const float2 a = fma2(DXf, DYf, add2(DXf, DYf));
                    const float2 b = fma2(a, DZf, add2(a, DZf));
                    const float2 tgt = fma2(b, S, add2(b, S));
                    // the departure from the target from its parts (see section 5)
                    float2 h = f, dinc = make_float2(0.f, 0.f), lo = make_float2(0.f, 0.f);
                    if (STAGE >= 2) {
                        h = own2[p * kThreads];
                        dinc = DIC[p];
                    }
                    if constexpr (kLo && STAGE == 3)
                        lo = make_float2(lo_decode(LQC[p], h.x), lo_decode(LQC[p] >> 16, h.y));
                    const float2 dep = STAGE >= 2 ? add2(add2(sub2(h, tgt), dinc), lo) : sub2(f, tgt);
                    // Eq. (flux) and the relaxation: -|p_z| div / dz - dep / tau
                    const float2 div = add2(sub2(W[p][3], W[p][2]), sub2(cp, CM[p]));
                    const float2 Lv = fma2(dep, NITAU, mul2(mul2(NAPZ[p], div), IDZ));
                    float2 st;
                    if (STAGE == 1) {
                        st = mul2(DT, Lv);
                        out = add2(f, st);
                    } else if (STAGE == 2) {
                        st = mul2(splat(0.25f), fma2(DT, Lv, dinc));
                        out = add2(h, st);
                    } else {
                        const float2 inc = mul2(splat(float(2.0 / 3.0)), fma2(DT, Lv, dinc));
                        if constexpr (kLo) {
                            const float2 t = add2(lo, inc);
                            const float2 h2 = add2(h, t);
                            const float2 lo2 = sub2(t, sub2(h2, h));
                            if (ok[v0]) __stcg(lop + p * kThreads, lo_encode2(lo2, h2));
                            st = h2;
                        } else {
                            st = add2(h, inc);
                        }
                        out = st;
                    }
                    if (ok[v0]) __stcg(outp + p * kThreads, st);
                    CM[p] = cp;
                } else {
                    P2 = fma2(Z, Z, fma2(Y, Y, mul2(X, X)));
                }
#pragma unroll
                for (int d = 0; d < 5; ++d) W[p][d] = W[p][d + 1];
                W[p][5] = kD ? add2(rn2[p * kThreads], DC[p]) : rn2[p * kThreads];
                // the moments about the record's u (section 5): w f times 1, xi_a,
                // xi_a xi_b, |xi|^2 xi_a; pairs past the chunk contribute zero
                const float2 o = ok[v0] ? mul2(out, WV[p]) : make_float2(0.f, 0.f);
                const float2 oX = mul2(o, X), oY = mul2(o, Y), oZ = mul2(o, Z), oP = mul2(o, P2);
                if (p == 0) {
                    S2[0] = o; S2[1] = oX; S2[2] = oY; S2[3] = oZ;
                    S2[4] = mul2(oX, X); S2[5] = mul2(oY, Y); S2[6] = mul2(oZ, Z);
                    S2[7] = mul2(oX, Y); S2[8] = mul2(oX, Z); S2[9] = mul2(oY, Z);
                    S2[10] = mul2(oP, X); S2[11] = mul2(oP, Y); S2[12] = mul2(oP, Z);
                } else {
                    S2[0] = add2(S2[0], o); S2[1] = add2(S2[1], oX); S2[2] = add2(S2[2], oY);
                    S2[3] = add2(S2[3], oZ);
                    S2[4] = fma2(oX, X, S2[4]); S2[5] = fma2(oY, Y, S2[5]); S2[6] = fma2(oZ, Z, S2[6]);
                    S2[7] = fma2(oX, Y, S2[7]); S2[8] = fma2(oX, Z, S2[8]); S2[9] = fma2(oY, Z, S2[9]);
                    S2[10] = fma2(oP, X, S2[10]); S2[11] = fma2(oP, Y, S2[11]); S2[12] = fma2(oP, Z, S2[12]);
                }
            }
            float acc[16];
#pragma unroll
            for (int a = 0; a < kNMom; ++a) acc[a] = S2[a].x + S2[a].y;
#pragma unroll
            for (int a = kNMom; a < 16; ++a) acc[a] = 0.f;
            const float tot = reduce_scatter16<float>(acc, lane);
            const int m = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
            if ((lane & 1) == 0) red[((size_t)cc * (kThreads / 32) + warp) * 16 + m] = tot;
            outp += ostep2;
            if (kD) dop += ostep2;
            if (kLo && STAGE == 3) lop += ostep2;
        }
    } else {
    // ---- 5. march through the z-range in the upwind direction of the chunk: up
    // (p_z > 0) from z0, down (p_z < 0) from z0+zn-1.  At march step c the register
    // window holds the cells s-3 .. s+2 seen from upwind (s+3 .. s-2 going down), so
    // both directions use one stencil: the flux through the interface ahead is
    // |p_z| weno5(w1 .. w5), the one behind was formed at the previous step, and the
    // divergence of Eq. (flux) is (ahead - behind) / dz for the signed p_z either way.
    const long rstep = sgc ? -(long)KC : (long)KC;
    const T* rp = Fs + (sgc ? (size_t)(zn + 5) * KC : 0);  // window row d at step c: rp + (c + d) rstep
    // stages 2, 3: the increment of the cell of each window row, read from global memory
    // through the read-only path (this launch does not write it).  Window row cd at step c
    // holds cell zw0 + (c + cd) sdir; a ghost row (a cell outside 0 .. Nz-1) takes zero,
    // its shared-memory value being the whole stage input.  Thread-based pointers: the
    // thread's velocity v sits at + voff(v).
    const int sdir = sgc ? -1 : 1;
    const int zw0 = sgc ? z0 + zn + 2 : z0 - 3;
    const T* __restrict__ dq = Dg + k0 + tbase;
    auto inc_row = [&](int s, T(&out)[V]) {
        const bool in = kD && (unsigned)s < (unsigned)Nz;
        const T* p = dq + (long)s * Q;
#pragma unroll
        for (int v = 0; v < V; ++v) out[v] = in && ok[v] ? __ldg(p + voff(v)) : T(0);
    };
    // cm: the WENO correction of the interface behind (its flux is |p_z| (w2 + cm))
    T w[V][6], cm[V], dn[V];
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        inc_row(zw0 + d * sdir, dn);
#pragma unroll
        for (int v = 0; v < V; ++v) w[v][d] = rp[d * rstep + kl[v]] + dn[v];
    }
#pragma unroll
    for (int v = 0; v < V; ++v) cm[v] = weno5_corr<T>(w[v][0], w[v][1], w[v][2], w[v][3], w[v][4]);
    int sn = zw0 + 6 * sdir;  // the cell of the row the next step loads
    inc_row(sn, dn);
    const T dt = T(I.dt);
    const long ostep = sgc ? -(long)Q : (long)Q;
    const size_t orow0 = (size_t)(sgc ? z0 + zn - 1 : z0) * Q + k0 + tbase;  // the first cell, thread's column
    T* outp = Fout + orow0;
    const T* __restrict__ dop = kD ? Dg + orow0 : nullptr;  // the increment of the cell
    unsigned short* lop = kLo && STAGE == 3 ? I.L0 + orow0 : nullptr;
    // stage 3 (FP32): the residuals of the next cell are loaded one march step ahead, so
    // that their global-memory latency overlaps a step's arithmetic
    // the increments of the next cell (stages 2, 3) likewise
    unsigned short lqn[V];
    T din[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        lqn[v] = kLo && STAGE == 3 && ok[v] ? __ldcg(lop + voff(v)) : 0;
        din[v] = kD && ok[v] ? __ldg(dop + voff(v)) : T(0);
    }
    constexpr bool kPack = sizeof(T) == 4 && V % 2 == 0;  // moments of two velocities per packed op
#pragma unroll 1  // unrolling the z-march only adds instruction-cache misses
    for (int c = 0; c < zn; ++c) {
        unsigned short lqc[V];
        T dc[V], dic[V];  // increments of the window row this step loads and of the cell
#pragma unroll
        for (int v = 0; v < V; ++v) {
            lqc[v] = lqn[v];
            if (kLo && STAGE == 3 && ok[v] && c + 1 < zn) lqn[v] = __ldcg(lop + ostep + voff(v));
            dic[v] = din[v];
            if (kD && ok[v] && c + 1 < zn) din[v] = __ldg(dop + ostep + voff(v));
            dc[v] = dn[v];
        }
        if (kD && c + 1 < zn) {
            sn += sdir;
            inc_row(sn, dn);
        }
        const int cc = sgc ? zn - 1 - c : c;  // the cell within the tile
        const T* sc = recs + (size_t)cc * rstride;
        const T* gc = gsm + cc * G;
        const T* rn = rp + (c + 6) * rstep;
        const T* own = Fs + (size_t)(cc + 3) * KC;  // the cell's row of d
        T ux = 0, uy = 0, uz = 0, i5T = 0, qx = 0, qy = 0, qz = 0, itau = 0, cS = 0, idz = 0;
        if (STAGE > 0) {
            ux = sc[R_UX]; uy = sc[R_UY]; uz = sc[R_UZ];
            qx = sc[R_QX]; qy = sc[R_QY]; qz = sc[R_QZ];
            itau = sc[R_ITAU]; cS = sc[R_CS]; i5T = sc[R_I5T]; idz = idzs[cc];
        }
        // WENO corrections of the interfaces ahead, two velocities per packed FP32
        // instruction where the storage is FP32
        T cpv[V];
        if (STAGE > 0) {
            if constexpr (kPack) {
#pragma unroll
                for (int p2 = 0; p2 < V / 2; ++p2) {
                    const float2 r = weno5_corr2(make_float2(w[2 * p2][1], w[2 * p2 + 1][1]),
                                                 make_float2(w[2 * p2][2], w[2 * p2 + 1][2]),
                                                 make_float2(w[2 * p2][3], w[2 * p2 + 1][3]),
                                                 make_float2(w[2 * p2][4], w[2 * p2 + 1][4]),
                                                 make_float2(w[2 * p2][5], w[2 * p2 + 1][5]));
                    cpv[2 * p2] = r.x;
                    cpv[2 * p2 + 1] = r.y;
                }
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) cpv[v] = weno5_corr<T>(w[v][1], w[v][2], w[v][3], w[v][4], w[v][5]);
            }
        }
        // ---- per velocity: the update, its store, and the moment variables
        A ov[V], mx[V], my[V], mz[V], m2[V];  // value; the monomials' factors (p or p - u_r); |.|^2
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const unsigned short lq = lqc[v];
            const T wn = rn[kl[v]] + dc[v];
            T out = w[v][3];  // the value whose moments are taken
            T ex = 0, ey = 0, ez = 0, xi2 = 0;  // xi = p - u of the cell's record
            if (STAGE > 0) {
                const T cp = cpv[v];
                const T f = w[v][3];
                // Shakhov target n Gx Gy Gz (1 + S), S = cS (xi^2/(5T) - 1) xi.q; in the
                // phi / chi model (Eq. sred_def) S = cS ((xi_x^2 + xi_z^2)/(5T) - 4/5 or 2/5) xi.q
                // with u_y = q_y = 0, and Gy = 1 (phi) or T (chi) from the record
                T S;
                ex = px[v] - ux;
                ez = pz[v] - uz;
                if (RED) {
                    xi2 = ex * ex + ez * ez;
                    S = cS * (xi2 * i5T + py[v]) * (ex * qx + ez * qz);
                } else {
                    ey = py[v] - uy;
                    xi2 = ex * ex + ey * ey + ez * ez;
                    const T xq = ex * qx + ey * qy + ez * qz;
                    S = cS * (xi2 * i5T - T(1)) * xq;
                }
                // the target's deviation from 1: (1 + dx)(1 + dy)(1 + dz)(1 + S) - 1
                const T dx = gc[ii[v]], dy = gc[Qx + jj[v]], dz = gc[Qx + Qy + zz[v] - zm_lo];
                const T a = dx + dy + dx * dy, b = a + dz + a * dz, tgt = b + S + b * S;
                // the departure from the target, f - tgt: from the cell's d, increment and
                // (stage 3, FP32) residual separately, (d - tgt) + increment + residual,
                // so that its rounding is relative to the departure, which in the
                // collision-dominated regime is much smaller than f itself
                T h = f, dinc = T(0), lo = T(0);
                if (STAGE >= 2) {
                    h = own[kl[v]];
                    dinc = dic[v];
                }
                if constexpr (kLo && STAGE == 3) lo = lo_decode(lq, h);
                const T dep = STAGE >= 2 ? ((h - tgt) + dinc) + lo : f - tgt;
                // Eq. (flux): (|p_z| (w3 + cp) - |p_z| (w2 + cm)) / dz, formed from the
                // difference of the two upwind cells and of the two corrections, so that
                // its rounding is relative to the divergence rather than to d.  The
                // advection and relaxation increments nearly cancel near a steady state:
                // combine them first.
                const T Lv = -apz[v] * ((w[v][3] - w[v][2]) + (cp - cm[v])) * idz - dep * itau;
                T st;  // the value stored
                if (STAGE == 1) {
                    st = dt * Lv;
                    out = f + st;
                } else if (STAGE == 2) {
                    st = T(0.25) * (dinc + dt * Lv);
                    out = h + st;
                } else {
                    // Shu-Osher combine in increment form: F_l + 2/3 (d2 + dt L), added to the
                    // state with its rounding residual carried (FP32)
                    const T inc = T(2.0 / 3.0) * (dinc + dt * Lv);
                    if constexpr (kLo) {
                        const T t = lo + inc;
                        const T h2 = h + t;
                        const T lo2 = t - (h2 - h);
                        if (ok[v]) __stcg(lop + voff(v), lo_encode(lo2, h2));
                        st = h2;
                    } else {
                        st = h + inc;
                    }
                    out = st;
                }
                if (ok[v]) __stcg(outp + voff(v), st);
                cm[v] = cp;
            }
#pragma unroll
            for (int d = 0; d < 5; ++d) w[v][d] = w[v][d + 1];
            w[v][5] = wn;
            // the moments: of psi(p - u_r) about the velocity u_r of the cell's record
            // (stage 0, which has no record: of psi(p)), so that the third moments are
            // close to the heat flux itself instead of its sum with terms of size u |p|^2
            // that cancel it (160-fold in config C1), and the Shakhov factor's xi and
            // |xi|^2 serve as the monomials' factors; the finalisation adds the rest
            // state's moments about u_r.  Columns past the chunk hold no data (their
            // shared memory is never written) and contribute zero.
            ov[v] = ok[v] ? A(out) * wv[v] : A(0);
            if (STAGE > 0) {
                mx[v] = A(ex); my[v] = A(ey); mz[v] = A(ez); m2[v] = A(xi2);
            } else {
                mx[v] = A(px[v]); my[v] = yv[v]; mz[v] = A(pz[v]); m2[v] = p2v[v];
            }
        }
        // ---- the 13 weighted monomials summed over the thread's velocities: w f times
        // 1, p_a, p_a p_b, |p|^2 p_a (RED: chi carries the p_y^2 parts: sum chi, sum chi p_x,
        // sum chi p_z)
        A acc[16];
#pragma unroll
        for (int a = kNMom; a < 16; ++a) acc[a] = A(0);
        if constexpr (kPack && !RED) {
            float2 s2[kNMom];
#pragma unroll
            for (int p2 = 0; p2 < V / 2; ++p2) {
                const int v0 = 2 * p2, v1 = v0 + 1;
                const float2 o = make_float2(ov[v0], ov[v1]), X = make_float2(mx[v0], mx[v1]),
                             Y = make_float2(my[v0], my[v1]), Z = make_float2(mz[v0], mz[v1]),
                             P = make_float2(m2[v0], m2[v1]);
                const float2 oX = mul2(o, X), oY = mul2(o, Y), oZ = mul2(o, Z), oP = mul2(o, P);
                if (p2 == 0) {
                    s2[0] = o; s2[1] = oX; s2[2] = oY; s2[3] = oZ;
                    s2[4] = mul2(oX, X); s2[5] = mul2(oY, Y); s2[6] = mul2(oZ, Z);
                    s2[7] = mul2(oX, Y); s2[8] = mul2(oX, Z); s2[9] = mul2(oY, Z);
                    s2[10] = mul2(oP, X); s2[11] = mul2(oP, Y); s2[12] = mul2(oP, Z);
                } else {
                    s2[0] = add2(s2[0], o); s2[1] = add2(s2[1], oX); s2[2] = add2(s2[2], oY);
                    s2[3] = add2(s2[3], oZ);
                    s2[4] = fma2(oX, X, s2[4]); s2[5] = fma2(oY, Y, s2[5]); s2[6] = fma2(oZ, Z, s2[6]);
                    s2[7] = fma2(oX, Y, s2[7]); s2[8] = fma2(oX, Z, s2[8]); s2[9] = fma2(oY, Z, s2[9]);
                    s2[10] = fma2(oP, X, s2[10]); s2[11] = fma2(oP, Y, s2[11]); s2[12] = fma2(oP, Z, s2[12]);
                }
            }
#pragma unroll
            for (int a = 0; a < kNMom; ++a) acc[a] = s2[a].x + s2[a].y;
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                A t[kNMom];
                const A o = ov[v], X = mx[v], Y = my[v], Z = mz[v], P = m2[v];
                if (RED) {  // phi: p_y = 0; chi: the p_y^2 parts
                    const A oc = chi[v] ? o : A(0), op = o - oc;
                    const A oX = op * X, oZ = op * Z, r3 = op * P + oc;
                    t[0] = op; t[1] = oX; t[2] = A(0); t[3] = oZ;
                    t[4] = oX * X; t[5] = oc; t[6] = oZ * Z; t[7] = A(0); t[8] = oX * Z;
                    t[9] = A(0); t[10] = r3 * X; t[11] = A(0); t[12] = r3 * Z;
                } else {
                    const A oX = o * X, oY = o * Y, oZ = o * Z, oP = o * P;
                    t[0] = o; t[1] = oX; t[2] = oY; t[3] = oZ;
                    t[4] = oX * X; t[5] = oY * Y; t[6] = oZ * Z;
                    t[7] = oX * Y; t[8] = oX * Z; t[9] = oY * Z;
                    t[10] = oP * X; t[11] = oP * Y; t[12] = oP * Z;
                }
#pragma unroll
                for (int a = 0; a < kNMom; ++a) acc[a] = v == 0 ? t[a] : acc[a] + t[a];
            }
        }
        const A tot = reduce_scatter16<A>(acc, lane);
        const int m = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
        if ((lane & 1) == 0) red[((size_t)cc * (kThreads / 32) + warp) * 16 + m] = tot;
        outp += ostep;
        if (kD) dop += ostep;
        if (kLo && STAGE == 3) lop += ostep;
    }
    }  // the scalar march
    __syncthreads();
    // the chunk's partial of each cell: the warps' sums added and stored in the
    // accumulation type (FP32 storage: no FP64 instruction here; the finalisation sums
    // the chunks exactly enough in double-float)
    for (int e = tid; e < zn * kNMom; e += kThreads) {
        const int c = e / kNMom, a = e - c * kNMom;
        A s = red[(size_t)c * (kThreads / 32) * 16 + a];
#pragma unroll
        for (int q = 1; q < kThreads / 32; ++q) s += red[((size_t)c * (kThreads / 32) + q) * 16 + a];
        static_cast<A*>(I.partial)[((size_t)tile.chunk * kNMom + a) * Nz + z0 + c] = s;
    }

    // ---- 6. outgoing WENO flux of the stage output through the wall interfaces (for
    // n_w), as a sum over the deviations (the rest state's flux is added by the
    // finalisation).  Each thread re-reads the outputs it wrote itself: the new d after
    // stage 3, d + the increment after stages 1 and 2 (STAGE 0: its input rows).
    auto outval = [&](int v, int cell) -> T {
        const T* row = Fs + (size_t)(cell + rbase) * KC;
        if (STAGE == 0) return row[kl[v]];
        const T o = Fout[(size_t)cell * Q + k0 + kl[v]];
        return STAGE == 3 ? o : row[kl[v]] + o;
    };
    if (z0 == 0) {  // bottom: p_z < 0 leaves through s = -1/2
        double fl = 0.0;
#pragma unroll
        for (int v = 0; v < V; ++v)
            if (ok[v] && sgc && !I.half) {  // no wall below a half channel
                const T f1 = outval(v, 0), f2 = outval(v, 1), f3 = outval(v, 2);
                const T g0 = T(I.ext_bot[0][0]) * f1 + T(I.ext_bot[0][1]) * f2 + T(I.ext_bot[0][2]) * f3;
                const T g1 = T(I.ext_bot[1][0]) * g0 + T(I.ext_bot[1][1]) * f1 + T(I.ext_bot[1][2]) * f2;
                fl += double(wm[v]) * double(pz[v] * weno5<T>(f3, f2, f1, g0, g1));
            }
        fl = block_sum(fl, wall_red);
        if (tid == 0) I.flux_part[tile.chunk * 2 + 0] = fl;
    }
    if (z0 + zn == Nz) {  // top: p_z > 0 leaves through s = Nz - 1/2
        double fl = 0.0;
#pragma unroll
        for (int v = 0; v < V; ++v)
            if (ok[v] && !sgc) {
                const T f1 = outval(v, Nz - 1), f2 = outval(v, Nz - 2), f3 = outval(v, Nz - 3);
                const T g0 = T(I.ext_top[0][0]) * f1 + T(I.ext_top[0][1]) * f2 + T(I.ext_top[0][2]) * f3;
                const T g1 = T(I.ext_top[1][0]) * g0 + T(I.ext_top[1][1]) * f1 + T(I.ext_top[1][2]) * f2;
                fl += double(wm[v]) * double(pz[v] * weno5<T>(f3, f2, f1, g0, g1));
            }
        fl = block_sum(fl, wall_red);
        if (tid == 0) I.flux_part[tile.chunk * 2 + 1] = fl;
    }

    // ---- 7. (fuse != 0) finalisation without extra launches (threadfence tickets): the CTA
    // that finishes last among the chunks of this z-tile finalises the tile's
    // cells; the one that finalises the instance's last z-tile does the walls
    // and the residual.  Counters are reset by their last user.
    if (!fuse) return;  // finalize_cells follows as a separate launch
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(I.zcount + tile.zt, 1) == I.nchunks - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (I.fin_warp) {
        for (int c = tid >> 5; c < zn; c += kThreads / 32) finalize_cell_warp<T>(I, z0 + c, tid & 31, STAGE);
    } else if (tid < zn) {
        finalize_cell<T>(I, z0 + tid, STAGE);
    }
    if (tid == 0) I.zcount[tile.zt] = 0;
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(I.icount, 1) == I.nzt - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (tid == 0) *I.icount = 0;
    finalize_instance(I, STAGE, wall_red);
}

// ---- host-side launch of one stage-kernel instantiation ----------------------
template <typename T, int V, int STAGE, bool RED>
static cudaError_t launch_stage_t(const InstDev* d_inst, const Tile* d_tiles, int ntiles, size_t smem,
                                  int fuse, cudaStream_t st)
{
    auto kfn = stage_kernel<T, V, STAGE, RED>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kfn<<<ntiles, kThreads, smem, st>>>(d_inst, d_tiles, fuse);
    return cudaGetLastError();
}

template <typename T, int V, bool RED>
static cudaError_t launch_stage_r(int stage, const InstDev* d, const Tile* t, int n, size_t smem, int fuse,
                                  cudaStream_t st)
{
    switch (stage) {
        case 0: return launch_stage_t<T, V, 0, RED>(d, t, n, smem, fuse, st);
        case 1: return launch_stage_t<T, V, 1, RED>(d, t, n, smem, fuse, st);
        case 2: return launch_stage_t<T, V, 2, RED>(d, t, n, smem, fuse, st);
        default: return launch_stage_t<T, V, 3, RED>(d, t, n, smem, fuse, st);
    }
}

template <typename T, bool RED>
static cudaError_t launch_stage_m(int V, int stage, const InstDev* d, const Tile* t, int n, size_t smem, int fuse,
                                  cudaStream_t st)
{
    if (V == 1) return launch_stage_r<T, 1, RED>(stage, d, t, n, smem, fuse, st);
    if (V == 2) return launch_stage_r<T, 2, RED>(stage, d, t, n, smem, fuse, st);
    return launch_stage_r<T, 4, RED>(stage, d, t, n, smem, fuse, st);
}

// per (storage type, model) launchers of the stage kernel, one translation unit each
cudaError_t launch_stage_f32_full(int V, int stage, const InstDev* d, const Tile* t, int n, size_t smem, int fuse,
                                  cudaStream_t st);
cudaError_t launch_stage_f32_red(int V, int stage, const InstDev* d, const Tile* t, int n, size_t smem, int fuse,
                                 cudaStream_t st);
cudaError_t launch_stage_f64_full(int V, int stage, const InstDev* d, const Tile* t, int n, size_t smem, int fuse,
                                  cudaStream_t st);
cudaError_t launch_stage_f64_red(int V, int stage, const InstDev* d, const Tile* t, int n, size_t smem, int fuse,
                                 cudaStream_t st);

}  // namespace lbs
