// lbs_moments_static: the profiles of a caller-supplied distribution, computed
// without allocating any device memory.
//
// Some callers cannot call cudaMalloc at the point where they need moments:
// code that runs under another framework's device-memory budget (a caching
// allocator that owns the whole pool), or a latency-critical loop in which the
// device-wide synchronisation of cudaMalloc/cudaFree is not acceptable.  This
// entry point serves them: it reduces the moments of a distribution the caller
// already holds in device memory into profiles the caller also provides, and
// its only scratch (the per-chunk partial sums of the moment reduction) is the
// file-scope array below.  It is a variant of the solver's analysis pass (the
// stage kernel without an update, followed by the per-cell finalise); the paper
// has no counterpart.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lbs.h"
#include "lbs_internal.h"

namespace lbs {

// 2 MiB of partial sums: ceil(Q / kStaticChunk) * Nz * kNMom doubles at most.
constexpr int kStaticChunk = 512;
constexpr size_t kStaticScratch = size_t(1) << 18;  // doubles

// Shared by every call on a device and kept until the process exits.  Each
// call overwrites every entry it later reads, so nothing needs clearing, but
// calls that overlap on the GPU (different streams, or different host threads
// on one device) race on it.
static __device__ __align__(256) double g_static_partial[kStaticScratch];

// per (velocity chunk, cell): raw moments sum_k w_k f_k psi(p_k), FP64 sums, of the
// populations f_k = w_k (1 + d_k) given as their deviations d_k (the solver's state form)
template <typename T>
__global__ void __launch_bounds__(128) static_partials(const InstDev* __restrict__ insts, int inst,
                                                      const T* __restrict__ f, double* __restrict__ partial)
{
    const InstDev& I = insts[inst];
    const int chunk = blockIdx.x, cell = blockIdx.y;
    const int Q = I.Q, Qx = I.Qx, Qy = I.Qy, Qz = I.Qz, QxQy = I.QxQy;
    const int k0 = chunk * kStaticChunk, k1 = min(Q, k0 + kStaticChunk);
    double acc[kNMom];
    for (int a = 0; a < kNMom; ++a) acc[a] = 0.0;
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const int j = k % Qy, i = (k / Qy) % Qx, zm = k / QxQy, sg = zm >= Qz, m = zm - sg * Qz;
        const double X = static_cast<const T*>(I.px)[i], Y = static_cast<const T*>(I.py)[j];
        const double xi = static_cast<const T*>(I.xi)[m], Z = sg ? -xi : xi;
        const double w = double(static_cast<const T*>(I.wx)[i]) * double(static_cast<const T*>(I.wy)[j]) *
                         double(static_cast<const T*>(I.wz)[m]);
        const double g = w * (1.0 + double(f[(size_t)cell * Q + k]));  // f_k = w_k (1 + d_k)
        if (I.reduced && j == 1) {  // chi = int p_y^2 f dp_y: the p_y^2 moments only
            acc[5] += g;
            acc[10] += g * X;
            acc[12] += g * Z;
            continue;
        }
        const double p2 = X * X + Y * Y + Z * Z;
        acc[0] += g;
        acc[1] += g * X; acc[2] += g * Y; acc[3] += g * Z;
        acc[4] += g * X * X; acc[5] += g * Y * Y; acc[6] += g * Z * Z;
        acc[7] += g * X * Y; acc[8] += g * X * Z; acc[9] += g * Y * Z;
        acc[10] += g * p2 * X; acc[11] += g * p2 * Y; acc[12] += g * p2 * Z;
    }
    __shared__ double red[kNMom][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int a = 0; a < kNMom; ++a) {
        double v = acc[a];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[a][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < kNMom) {
        const int a = threadIdx.x;
        partial[((size_t)chunk * I.Nz + cell) * kNMom + a] = red[a][0] + red[a][1] + red[a][2] + red[a][3];
    }
}

// per cell: sum the chunks and form the 14 profiles (layout of lbs_profiles)
__global__ void static_profiles(const InstDev* __restrict__ insts, int inst, int nchunks,
                                const double* __restrict__ partial, double* __restrict__ prof)
{
    const InstDev& I = insts[inst];
    const int cell = blockIdx.x * blockDim.x + threadIdx.x, Nz = I.Nz;
    if (cell >= Nz) return;
    double mom[kNMom];
    for (int a = 0; a < kNMom; ++a) {
        double s = 0.0;
        for (int c = 0; c < nchunks; ++c) s += partial[((size_t)c * Nz + cell) * kNMom + a];
        mom[a] = s;
    }
    CellState c;  // the solver's own raw -> central moment map (NaN profiles if n = 0)
    cell_state(mom, c);
    const double vals[14] = {c.n, c.u[0], c.u[1], c.u[2], c.T, c.q[0], c.q[1], c.q[2],
                             c.P[0], c.P[1], c.P[2], c.P[3], c.P[4], c.P[5]};
    for (int a = 0; a < 14; ++a) prof[(size_t)a * Nz + cell] = vals[a];
}

// device address of g_static_partial, looked up once per device
static std::mutex g_mu;
static double* g_addr[64];

static int scratch_address(int device, double** out)
{
    if (device < 0 || device >= 64) return record_error(LBS_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_partial);
        if (e != cudaSuccess || !p)
            return record_error(LBS_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
        g_addr[device] = static_cast<double*>(p);
    }
    *out = g_addr[device];
    return LBS_OK;
}

}  // namespace lbs

extern "C" lbs_status lbs_moments_static(lbs_handle h, int inst, const void* f_dev, double* prof_dev)
{
    using namespace lbs;
    HandleView v;
    int st = handle_view(h, inst, &v);
    if (st != LBS_OK) return static_cast<lbs_status>(st);
    if (!f_dev || !prof_dev) return static_cast<lbs_status>(record_error(LBS_ERR_ARG, "null device pointer"));
    const int nchunks = (v.inst.Q + kStaticChunk - 1) / kStaticChunk;
    if ((size_t)nchunks * v.inst.Nz * kNMom > kStaticScratch)
        return static_cast<lbs_status>(record_error(
            LBS_ERR_ARG, "instance too large for the 2 MiB static scratch: need ceil(Q/512) * Nz <= 20164"));
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess)
        return static_cast<lbs_status>(record_error(LBS_ERR_CUDA, "cudaGetDevice failed"));
    if (cur != v.device && cudaSetDevice(v.device) != cudaSuccess)
        return static_cast<lbs_status>(record_error(LBS_ERR_CUDA, "cudaSetDevice failed"));
    double* scratch = nullptr;
    st = scratch_address(v.device, &scratch);
    cudaStream_t s = static_cast<cudaStream_t>(v.stream);
    if (st == LBS_OK) {
        dim3 g1(nchunks, v.inst.Nz);
        if (v.fp32)
            static_partials<float><<<g1, 128, 0, s>>>(v.d_inst, inst, static_cast<const float*>(f_dev), scratch);
        else
            static_partials<double><<<g1, 128, 0, s>>>(v.d_inst, inst, static_cast<const double*>(f_dev), scratch);
        static_profiles<<<(v.inst.Nz + 127) / 128, 128, 0, s>>>(v.d_inst, inst, nchunks, scratch, prof_dev);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = record_error(LBS_ERR_CUDA, cudaGetErrorString(e));
    }
    if (cur != v.device) cudaSetDevice(cur);
    return static_cast<lbs_status>(st);
}
