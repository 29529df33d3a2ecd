// Finalisation and seeding kernels and the launchers of every kernel of the
// scheme (the device code shared with the stage kernel is in kernels.cuh; the
// stage kernel's instantiations are in the stage_*.cu translation units).
#include "kernels.cuh"

namespace lbs {

// ---- separate finalisation launches (used when the stage kernel does not fuse them).
// NB bounds the expansion orders of the batch (the unrolled coefficient loops of the
// record run to NB, not to the largest order kMaxN).
template <typename T, int NB>
__global__ void __launch_bounds__(32) finalize_cells(const InstDev* __restrict__ insts, int stage)
{
    __shared__ double red[kRedSlots];
    __shared__ int last;
    __shared__ InstDev sI;
    const InstDev& I = stage_descriptor(insts + blockIdx.y, &sI);
    const int nblk = (I.Nz + 31) >> 5;
    if (blockIdx.x >= nblk || *I.active == 0) return;
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell < I.Nz) finalize_cell<T, NB>(I, cell, stage);
    // the instance's last block to finish (threadfence ticket) forms n_w and, after
    // stage 3, the residual; the counter is reset by its last user
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(I.icount, 1) == nblk - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) *I.icount = 0;
    finalize_instance(I, stage, red);
}

// the same with one warp per cell (4 cells per block of 128 threads)
template <typename T>
__global__ void __launch_bounds__(128) finalize_cells_warp(const InstDev* __restrict__ insts, int stage)
{
    __shared__ double red[kRedSlots];
    __shared__ int last;
    __shared__ InstDev sI;
    const InstDev& I = stage_descriptor(insts + blockIdx.y, &sI);
    const int nblk = (I.Nz + 3) >> 2;
    if (blockIdx.x >= nblk || *I.active == 0) return;
    const int cell = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (cell < I.Nz) finalize_cell_warp<T>(I, cell, threadIdx.x & 31, stage);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(I.icount, 1) == nblk - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) *I.icount = 0;
    finalize_instance(I, stage, red);
}

// ---- seed a cell from its record: d_k = f_k / w_k - 1 = R_SCALE Gx Gy Gz (1 + S) - 1,
// formed from the factors' deviations as in the stage kernel; the rounding residual
// (FP32 storage) starts at zero.  Written into whichever buffer holds the state.
template <typename T>
__global__ void __launch_bounds__(128) seed_cells(const InstDev* __restrict__ insts, int inst)
{
    const InstDev& I = insts[inst];
    const int cell = blockIdx.x;
    const T* rc = static_cast<const T*>(I.rec) + (size_t)cell * I.rec_stride;
    T* F = static_cast<T*>(*I.cur ? I.F1 : I.F0) + (size_t)cell * I.Q;
    for (int k = threadIdx.x; k < I.Q; k += blockDim.x) {
        const int j = k % I.Qy, i = (k / I.Qy) % I.Qx, zm = k / I.QxQy;
        const int sg = zm >= I.Qz, m = zm - sg * I.Qz;
        const T gx = rc[R_SCALE1] + (T(1) + rc[R_SCALE1]) * rc[R_DX + i];
        const T gy = rc[R_DX + I.Qx + j], gz = rc[R_DX + I.Qx + I.Qy + zm];
        const T x = ld<T>(I.xi, m);
        const T ex = ld<T>(I.px, i) - rc[R_UX], ey = ld<T>(I.py, j) - rc[R_UY], ez = (sg ? -x : x) - rc[R_UZ];
        const T S = I.reduced ? rc[R_CS] * ((ex * ex + ez * ez) * rc[R_I5T] - (j ? T(0.4) : T(0.8))) *
                                    (ex * rc[R_QX] + ez * rc[R_QZ])
                              : rc[R_CS] * ((ex * ex + ey * ey + ez * ez) * rc[R_I5T] - T(1)) *
                    (ex * rc[R_QX] + ey * rc[R_QY] + ez * rc[R_QZ]);
        const T a = gx + gy + gx * gy, b = a + gz + a * gz;
        F[k] = b + S + b * S;
        if (I.L0) I.L0[(size_t)cell * I.Q + k] = 0;
    }
}

// ---- seed a cell with the free-molecular state of the channel: each velocity carries the
// discrete equilibrium of the wall it left (Appendix, with n_w = 1: p_z > 0 the bottom
// wall, p_z < 0 the top wall; the incoming ghosts' formula), then the cell is rescaled to
// unit density.  The collisionless limit of Couette flow between diffuse walls; a start
// for strongly rarefied instances.  One block per cell; residual 0.
template <typename T>
__global__ void __launch_bounds__(128) seed_free_molecular(const InstDev* __restrict__ insts, int inst)
{
    __shared__ double red[kRedSlots];
    const InstDev& I = insts[inst];
    const int cell = blockIdx.x;
    T* F = static_cast<T*>(*I.cur ? I.F1 : I.F0) + (size_t)cell * I.Q;
    double m = 0.0;  // the cell's density sum w (1 + d), phi's alone in the reduced model
    for (int k = threadIdx.x; k < I.Q; k += blockDim.x) {
        const int j = k % I.Qy, i = (k / I.Qy) % I.Qx, zm = k / I.QxQy;
        const int sg = zm >= I.Qz, mz = zm - sg * I.Qz;
        const T ax = ld<T>(sg ? I.gwx_top : I.gwx_bot, i), ay = ld<T>(I.gwy, j), az = ld<T>(I.gwz, zm);
        const T a = ax + ay + ax * ay, b = a + az + a * az;
        F[k] = b;
        if (!(I.reduced && j == 1))
            m += double(ld<T>(I.wx, i)) * double(ld<T>(I.wy, j)) * double(ld<T>(I.wz, mz)) * (1.0 + double(b));
    }
    m = block_sum(m, red);
    const T c = T(1.0 / m - 1.0);  // (1 + d) / m - 1 = d + c (1 + d)
    for (int k = threadIdx.x; k < I.Q; k += blockDim.x) {
        const T d = F[k];
        F[k] = d + c * (T(1) + d);
        if (I.L0) I.L0[(size_t)cell * I.Q + k] = 0;
    }
}

// The eight profile rows that lbs_moments reports (n, u_x, T, q_x, q_z, P_xx, P_xz, P_zz:
// rows 0, 1, 4, 5, 7, 8, 12, 10 of the [14][Nz] profiles, one nibble each) of every
// instance, packed [8][Nz] per instance in instance order, so that a whole-batch read is
// one device-to-host copy.  The profiles sit back to back (14 Nz doubles per instance),
// so an instance's offset in out is 8/14 of its offset in prof_all.  Block (b, r) copies
// row r of instance b.
__global__ void __launch_bounds__(128) gather_moment_rows(const InstDev* __restrict__ insts,
                                                          const double* __restrict__ prof_all,
                                                          double* __restrict__ out)
{
    const InstDev& I = insts[blockIdx.x];
    const int r = blockIdx.y, row = (0xAC875410u >> (4 * r)) & 0xFu;
    const long before = (long)(I.prof - prof_all) / 14;  // cells of the instances before b
    const double* __restrict__ src = I.prof + (long)row * I.Nz;
    double* __restrict__ dst = out + 8 * before + (long)r * I.Nz;
    for (int c = threadIdx.x; c < I.Nz; c += blockDim.x) dst[c] = src[c];
}

// ---- host launchers ---------------------------------------------------------
cudaError_t launch_gather_moments(const InstDev* d_inst, int ninst, const double* prof_all, double* out,
                                  cudaStream_t st)
{
    gather_moment_rows<<<dim3(ninst, 8), 128, 0, st>>>(d_inst, prof_all, out);
    return cudaGetLastError();
}

size_t stage_smem_bytes(int fp32, int V, int zn, int G, int stage, int rstride)
{
    const int KC = kThreads * V;
    (void)stage;
    // element and accumulator sizes from the kernel's own types, so that the host's
    // dynamic shared-memory size always covers the kernel's layout
    return stage_smem(zn, KC, G, fp32 ? (int)sizeof(float) : (int)sizeof(double),
                      fp32 ? (int)sizeof(Acc<float>::type) : (int)sizeof(Acc<double>::type), rstride)
        .total;
}

// Finalisation launches carry the device's highest priority: when the batch's halves step
// on two streams, the block scheduler then dispatches one half's finalisation blocks as soon
// as the other half's stage CTAs free room on an SM, instead of after all of them.  (The
// attribute is kept by CUDA-graph capture.)
static int highest_priority()
{
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    return greatest;
}
template <typename K>
static cudaError_t launch_first(K kernel, dim3 g, dim3 b, cudaStream_t st, const InstDev* d_inst, int stage)
{
    static const int prio = highest_priority();
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = prio;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, d_inst, stage);
}

template <typename T>
static cudaError_t launch_finalize_t(int stage, const InstDev* d_inst, int ninst, int maxNz, int fin_warp,
                                     int nb, cudaStream_t st)
{
    const dim3 g((maxNz + 31) / 32, ninst);
    if (fin_warp) return launch_first(finalize_cells_warp<T>, dim3((maxNz + 3) / 4, ninst), dim3(128), st, d_inst, stage);
    if (nb <= 4) return launch_first(finalize_cells<T, 4>, g, dim3(32), st, d_inst, stage);
    if (nb <= 6) return launch_first(finalize_cells<T, 6>, g, dim3(32), st, d_inst, stage);
    return launch_first(finalize_cells<T, kMaxN>, g, dim3(32), st, d_inst, stage);
}

// the stage kernel alone
cudaError_t launch_stage_only(int fp32, int red, int V, int stage, const InstDev* d_inst, const Tile* d_tiles,
                              int ntiles, size_t smem, int fuse, cudaStream_t st)
{
    if (ntiles <= 0) return cudaSuccess;  // a split half whose instances have all retired
    if (fp32)
        return red ? launch_stage_f32_red(V, stage, d_inst, d_tiles, ntiles, smem, fuse, st)
                   : launch_stage_f32_full(V, stage, d_inst, d_tiles, ntiles, smem, fuse, st);
    return red ? launch_stage_f64_red(V, stage, d_inst, d_tiles, ntiles, smem, fuse, st)
               : launch_stage_f64_full(V, stage, d_inst, d_tiles, ntiles, smem, fuse, st);
}

// the separate finalisation launches of an unfused stage
cudaError_t launch_finalize(int fp32, int stage, const InstDev* d_inst, int ninst, int maxNz, int fin_warp,
                            int nb, cudaStream_t st)
{
    return fp32 ? launch_finalize_t<float>(stage, d_inst, ninst, maxNz, fin_warp, nb, st)
                : launch_finalize_t<double>(stage, d_inst, ninst, maxNz, fin_warp, nb, st);
}

// one RK stage (stage 1..3) or the analysis pass (stage 0); without fusion the
// finalisation follows as two more launches
cudaError_t launch_stage(int fp32, int red, int V, int stage, const InstDev* d_inst, const Tile* d_tiles,
                         int ntiles, size_t smem, int fuse, int ninst, int maxNz, int fin_warp, int nb,
                         cudaStream_t st)
{
    cudaError_t e = launch_stage_only(fp32, red, V, stage, d_inst, d_tiles, ntiles, smem, fuse, st);
    if (e != cudaSuccess || fuse) return e;
    return launch_finalize(fp32, stage, d_inst, ninst, maxNz, fin_warp, nb, st);
}

cudaError_t launch_seed_free_molecular(int fp32, const InstDev* d_inst, int inst, int Nz, cudaStream_t st)
{
    if (fp32) seed_free_molecular<float><<<Nz, 128, 0, st>>>(d_inst, inst);
    else seed_free_molecular<double><<<Nz, 128, 0, st>>>(d_inst, inst);
    return cudaGetLastError();
}

cudaError_t launch_seed(int fp32, const InstDev* d_inst, int inst, int Nz, const double* d_macro,
                        cudaStream_t st)
{
    const int g = (Nz + 63) / 64;
    if (fp32) records_from_macro<float><<<g, 64, 0, st>>>(d_inst, inst, d_macro);
    else records_from_macro<double><<<g, 64, 0, st>>>(d_inst, inst, d_macro);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (fp32) seed_cells<float><<<Nz, 128, 0, st>>>(d_inst, inst);
    else seed_cells<double><<<Nz, 128, 0, st>>>(d_inst, inst);
    return cudaGetLastError();
}

}  // namespace lbs
