// lbs_probe_fma_rate: the device's sustained FMA rate in FP64 and FP32, measured with
// CUDA events on a kernel of independent fused multiply-add chains.  It is the peak
// against which the FP64 solver (bound by the FP64 pipe, not by HBM) is reported.
// Not part of the scheme.
#include <cuda_runtime.h>

#include <string>

#include "../../include/lbs.h"
#include "lbs_internal.h"

namespace lbs {

// kChains independent chains per thread, iters multiply-adds each; the operands stay
// in registers.  a * x + b with |a| < 1 keeps every value finite.
constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_chains(T* out, T a, T b, int iters)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
#pragma unroll 4
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == T(-1)) out[blockIdx.x] = s;  // never true; keeps the chains live
}

template <typename T>
static lbs_status rate(double* flops, std::string& err)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8;
    const int iters = sizeof(T) == 8 ? 4096 : 65536;  // tens of milliseconds either way
    T* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(T) * blocks);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0);
        fma_chains<T><<<blocks, 256>>>(out, T(0.999), T(1e-4), iters);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;  // the first launch warms up
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        err = cudaGetErrorString(e);
        return LBS_ERR_CUDA;
    }
    *flops = 2.0 * kChains * (double)iters * 256.0 * blocks / (best * 1e-3);
    return LBS_OK;
}

}  // namespace lbs

extern "C" lbs_status lbs_probe_fma_rate(double* fp64_flops, double* fp32_flops)
{
    using namespace lbs;
    if (!fp64_flops || !fp32_flops) return static_cast<lbs_status>(record_error(LBS_ERR_ARG, "null output"));
    std::string err;
    lbs_status s = rate<double>(fp64_flops, err);
    if (s == LBS_OK) s = rate<float>(fp32_flops, err);
    if (s != LBS_OK) return static_cast<lbs_status>(record_error(s, ("FMA rate probe: " + err).c_str()));
    return LBS_OK;
}
