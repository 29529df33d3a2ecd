// Warm-start network: a 3-layer perceptron (n_in -> H -> H -> n_out, GELU) that
// maps the parameters of a Couette problem to its steady profiles.  Matrix
// products run on the tensor cores in BF16 with FP32 accumulation
// (mma.sync.m16n8k16): every product operand is rounded to BF16 when it is
// staged into shared memory; biases, GELU, the loss, the gradients' elementwise
// parts and Adam are FP32, with FP32 master weights and BF16 working copies.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbs.h"
#include "lbs_internal.h"

namespace lbs {
namespace mlp {

constexpr int kTM = 64, kTN = 64, kTK = 16;  // CTA tile; 4 warps of 32 x 32
enum { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2 };

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// C[m][n] = sum_k A(m, k) B(k, n) (+ bias[n], + GELU), A(m, k) = A[m sAm + k sAk],
// B(k, n) = B[k sBk + n sBn]: the strides cover the transposed products of the
// backward pass.  EPI_BIAS_GELU stores z = acc + bias in C and gelu(z) in H.
template <typename TA, typename TB, int EPI>
__global__ void __launch_bounds__(128) gemm_bf16(int M, int N, int K, const TA* __restrict__ A, long sAm,
                                                long sAk, const TB* __restrict__ B, long sBk, long sBn,
                                                float* __restrict__ C, long ldc, const float* __restrict__ bias,
                                                float* __restrict__ H)
{
    __shared__ __align__(16) __nv_bfloat16 As[kTM][kTK + 8];  // [m][k]
    __shared__ __align__(16) __nv_bfloat16 Bs[kTN][kTK + 8];  // [n][k] (k contiguous for the B fragment)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;  // warp tile origin
    const int g = lane >> 2, t = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

    for (int k0 = 0; k0 < K; k0 += kTK) {
        for (int e = tid; e < kTM * kTK; e += 128) {
            const int m = e / kTK, k = e % kTK, gm = m0 + m, gk = k0 + k;
            const float v = (gm < M && gk < K) ? to_f(A[gm * sAm + gk * sAk]) : 0.f;
            As[m][k] = __float2bfloat16_rn(v);
        }
        for (int e = tid; e < kTN * kTK; e += 128) {
            const int n = e / kTK, k = e % kTK, gn = n0 + n, gk = k0 + k;
            const float v = (gn < N && gk < K) ? to_f(B[gk * sBk + gn * sBn]) : 0.f;
            Bs[n][k] = __float2bfloat16_rn(v);
        }
        __syncthreads();
        uint32_t a[2][4], b[4][2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r = wm + 16 * i + g;
            a[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][2 * t]);
            a[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][2 * t]);
            a[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][2 * t + 8]);
            a[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][2 * t + 8]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = wn + 8 * j + g;
            b[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[n][2 * t]);
            b[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[n][2 * t + 8]);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                    "{%8,%9}, {%0,%1,%2,%3};"
                    : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                    : "r"(a[i][0]), "r"(a[i][1]), "r"(a[i][2]), "r"(a[i][3]), "r"(b[j][0]), "r"(b[j][1]));
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = m0 + wm + 16 * i + g + (r >= 2 ? 8 : 0);
                const int n = n0 + wn + 8 * j + 2 * t + (r & 1);
                if (m >= M || n >= N) continue;
                float v = acc[i][j][r];
                if (EPI != EPI_STORE) v += bias[n];
                C[m * ldc + n] = v;
                if (EPI == EPI_BIAS_GELU) H[m * ldc + n] = gelu(v);
            }
}

// dy = 2 (y - t) / (B n_out); the squared error is summed into *loss (FP64)
__global__ void mse_grad(const float* __restrict__ y, const float* __restrict__ tgt, float* __restrict__ dy,
                         long n, float scale, double* loss)
{
    __shared__ double red[8];
    double s = 0.0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const float d = y[e] - tgt[e];
        dy[e] = 2.f * d * scale;
        s += double(d) * double(d);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(loss, t);
    }
}

// dz = dh * gelu'(z)
__global__ void gelu_backward(const float* __restrict__ dh, const float* __restrict__ z, float* __restrict__ dz,
                              long n)
{
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        dz[e] = dh[e] * gelu_grad(z[e]);
}

// db[n] = sum over the batch of d[b][n]
__global__ void colsum(const float* __restrict__ d, int B, int N, float* __restrict__ db)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += d[(long)b * N + n];
    db[n] = s;
}

// Adam (bias corrected) on the FP32 masters, then refresh the BF16 weight copies
__global__ void adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                     float* __restrict__ v, long n, float lr, float b1, float b2, float eps, float c1, float c2,
                     __nv_bfloat16* __restrict__ pb, const unsigned char* __restrict__ is_w)
{
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const float gg = g[e];
        const float mm = b1 * m[e] + (1.f - b1) * gg;
        const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
        m[e] = mm;
        v[e] = vv;
        const float w = p[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
        p[e] = w;
        if (is_w[e]) pb[e] = __float2bfloat16_rn(w);
    }
}

__global__ void to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ pb, long n)
{
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        pb[e] = __float2bfloat16_rn(p[e]);
}

}  // namespace mlp
}  // namespace lbs

using namespace lbs;
using namespace lbs::mlp;

struct lbs_mlp {
    int I, H, O, maxB;
    long nW1, nb1, nW2, nb2, nW3, nb3, P;
    long oW1, ob1, oW2, ob2, oW3, ob3;  // offsets into the packed parameter vector
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    unsigned char* mem = nullptr;
    float *p, *g, *m, *v;                 // [P] masters, gradients, Adam moments
    __nv_bfloat16* pb;                    // [P] BF16 copies (weights; biases unused)
    unsigned char* is_w;                  // [P] 1 where the entry is a weight
    float *z1, *h1, *z2, *h2, *y, *dy, *dh, *dz;  // activations and gradients, max batch
    double* loss;
    long step = 0;
};

#define MCK(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return static_cast<lbs_status>(record_error(LBS_ERR_CUDA, cudaGetErrorString(e_))); \
    } while (0)

static lbs_status merr(lbs_status s, const char* m) { return static_cast<lbs_status>(record_error(s, m)); }

template <typename TA, typename TB, int EPI>
static cudaError_t gemm(cudaStream_t st, int M, int N, int K, const TA* A, long sAm, long sAk, const TB* B, long sBk,
                        long sBn, float* C, long ldc, const float* bias = nullptr, float* H = nullptr)
{
    dim3 grid((N + kTN - 1) / kTN, (M + kTM - 1) / kTM);
    gemm_bf16<TA, TB, EPI><<<grid, 128, 0, st>>>(M, N, K, A, sAm, sAk, B, sBk, sBn, C, ldc, bias, H);
    return cudaGetLastError();
}

static int blocks(long n) { return (int)std::min<long>((n + 255) / 256, 4096); }

// forward pass for a batch already on the device; y may be h->y
static lbs_status forward(lbs_mlp* h, const float* x, int B, float* y)
{
    const __nv_bfloat16* W1 = h->pb + h->oW1;
    const __nv_bfloat16* W2 = h->pb + h->oW2;
    const __nv_bfloat16* W3 = h->pb + h->oW3;
    MCK((gemm<float, __nv_bfloat16, EPI_BIAS_GELU>(h->stream, B, h->H, h->I, x, h->I, 1, W1, 1, h->I, h->z1, h->H,
                                                   h->p + h->ob1, h->h1)));
    MCK((gemm<float, __nv_bfloat16, EPI_BIAS_GELU>(h->stream, B, h->H, h->H, h->h1, h->H, 1, W2, 1, h->H, h->z2, h->H,
                                                   h->p + h->ob2, h->h2)));
    MCK((gemm<float, __nv_bfloat16, EPI_BIAS>(h->stream, B, h->O, h->H, h->h2, h->H, 1, W3, 1, h->H, y, h->O,
                                              h->p + h->ob3)));
    return LBS_OK;
}

extern "C" {

lbs_status lbs_mlp_create(lbs_mlp_handle* out, int n_in, int n_hidden, int n_out, int max_batch, void* stream)
{
    if (!out || n_in < 1 || n_hidden < 1 || n_out < 1 || max_batch < 1 || n_in > 4096 || n_hidden > 4096 ||
        n_out > 4096 || max_batch > (1 << 20))
        return merr(LBS_ERR_ARG, "network sizes must lie in 1..4096 and the batch in 1..2^20");
    lbs_mlp* h = new lbs_mlp();
    h->I = n_in; h->H = n_hidden; h->O = n_out; h->maxB = max_batch;
    h->nW1 = (long)n_hidden * n_in; h->nb1 = n_hidden;
    h->nW2 = (long)n_hidden * n_hidden; h->nb2 = n_hidden;
    h->nW3 = (long)n_out * n_hidden; h->nb3 = n_out;
    h->oW1 = 0; h->ob1 = h->oW1 + h->nW1; h->oW2 = h->ob1 + h->nb1; h->ob2 = h->oW2 + h->nW2;
    h->oW3 = h->ob2 + h->nb2; h->ob3 = h->oW3 + h->nW3; h->P = h->ob3 + h->nb3;
    if (stream) {
        h->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return merr(LBS_ERR_CUDA, "cudaStreamCreate failed");
        }
        h->own_stream = true;
    }
    const long P = h->P, BH = (long)max_batch * n_hidden, BO = (long)max_batch * n_out;
    const long wide = std::max(BH, BO);
    size_t bytes = 4 * P * 4 + 2 * P + P + (4 * BH + 2 * BO + 2 * wide) * 4 + 8 + 16 * 16;  // + alignment slack
    void* mem = nullptr;
    if (cudaMalloc(&mem, bytes) != cudaSuccess) {
        if (h->own_stream) cudaStreamDestroy(h->stream);
        delete h;
        return merr(LBS_ERR_CUDA, "cudaMalloc of the network's buffers failed");
    }
    h->mem = static_cast<unsigned char*>(mem);
    size_t o = 0;
    auto take = [&](size_t n) { size_t r = o; o = (o + n + 15) & ~size_t(15); return h->mem + r; };
    h->p = reinterpret_cast<float*>(take(P * 4));
    h->g = reinterpret_cast<float*>(take(P * 4));
    h->m = reinterpret_cast<float*>(take(P * 4));
    h->v = reinterpret_cast<float*>(take(P * 4));
    h->pb = reinterpret_cast<__nv_bfloat16*>(take(P * 2));
    h->is_w = take(P);
    h->z1 = reinterpret_cast<float*>(take(BH * 4));
    h->h1 = reinterpret_cast<float*>(take(BH * 4));
    h->z2 = reinterpret_cast<float*>(take(BH * 4));
    h->h2 = reinterpret_cast<float*>(take(BH * 4));
    h->y = reinterpret_cast<float*>(take(BO * 4));
    h->dy = reinterpret_cast<float*>(take(BO * 4));
    h->dh = reinterpret_cast<float*>(take(wide * 4));
    h->dz = reinterpret_cast<float*>(take(wide * 4));
    h->loss = reinterpret_cast<double*>(take(8));
    std::vector<unsigned char> isw(P, 0);
    for (long e = h->oW1; e < h->oW1 + h->nW1; ++e) isw[e] = 1;
    for (long e = h->oW2; e < h->oW2 + h->nW2; ++e) isw[e] = 1;
    for (long e = h->oW3; e < h->oW3 + h->nW3; ++e) isw[e] = 1;
    cudaError_t e1 = cudaMemcpyAsync(h->is_w, isw.data(), P, cudaMemcpyHostToDevice, h->stream);
    cudaError_t e2 = cudaMemsetAsync(h->mem, 0, 4 * P * 4, h->stream);
    cudaError_t e3 = cudaStreamSynchronize(h->stream);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        lbs_mlp_destroy(h);
        return merr(LBS_ERR_CUDA, "initialising the network's buffers failed");
    }
    *out = h;
    return LBS_OK;
}

lbs_status lbs_mlp_destroy(lbs_mlp_handle h)
{
    if (!h) return LBS_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->mem) cudaFree(h->mem);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return LBS_OK;
}

lbs_status lbs_mlp_num_params(lbs_mlp_handle h, long* out)
{
    if (!h || !out) return merr(LBS_ERR_ARG, "invalid handle or null output");
    *out = h->P;
    return LBS_OK;
}

lbs_status lbs_mlp_set_params(lbs_mlp_handle h, const float* host_params)
{
    if (!h || !host_params) return merr(LBS_ERR_ARG, "invalid handle or null parameters");
    for (long e = 0; e < h->P; ++e)
        if (!std::isfinite(host_params[e])) return merr(LBS_ERR_NONFINITE, "parameter not finite");
    MCK(cudaMemcpyAsync(h->p, host_params, h->P * 4, cudaMemcpyHostToDevice, h->stream));
    MCK(cudaMemsetAsync(h->m, 0, h->P * 4, h->stream));
    MCK(cudaMemsetAsync(h->v, 0, h->P * 4, h->stream));
    to_bf16<<<blocks(h->P), 256, 0, h->stream>>>(h->p, h->pb, h->P);
    MCK(cudaGetLastError());
    MCK(cudaStreamSynchronize(h->stream));
    h->step = 0;
    return LBS_OK;
}

lbs_status lbs_mlp_get_params(lbs_mlp_handle h, float* host_params)
{
    if (!h || !host_params) return merr(LBS_ERR_ARG, "invalid handle or null output");
    MCK(cudaMemcpyAsync(host_params, h->p, h->P * 4, cudaMemcpyDeviceToHost, h->stream));
    MCK(cudaStreamSynchronize(h->stream));
    return LBS_OK;
}

lbs_status lbs_mlp_forward(lbs_mlp_handle h, const float* x_dev, int B, float* y_dev)
{
    if (!h || !x_dev || !y_dev || B < 1 || B > h->maxB) return merr(LBS_ERR_ARG, "invalid arguments or batch too large");
    return forward(h, x_dev, B, y_dev);
}

lbs_status lbs_mlp_loss_grad(lbs_mlp_handle h, const float* x_dev, const float* t_dev, int B, double* loss_out,
                             float* grad_host)
{
    if (!h || !x_dev || !t_dev || B < 1 || B > h->maxB) return merr(LBS_ERR_ARG, "invalid arguments or batch too large");
    lbs_status s = forward(h, x_dev, B, h->y);
    if (s != LBS_OK) return s;
    const int I = h->I, H = h->H, O = h->O;
    cudaStream_t st = h->stream;
    MCK(cudaMemsetAsync(h->loss, 0, 8, st));
    const long BO = (long)B * O, BH = (long)B * H;
    mse_grad<<<blocks(BO), 256, 0, st>>>(h->y, t_dev, h->dy, BO, 1.f / float(BO), h->loss);
    MCK(cudaGetLastError());
    const __nv_bfloat16* W2 = h->pb + h->oW2;
    const __nv_bfloat16* W3 = h->pb + h->oW3;
    // layer 3: dW3 = dy^T h2, db3 = sum dy, dh2 = dy W3
    MCK((gemm<float, float, EPI_STORE>(st, O, H, B, h->dy, 1, O, h->h2, H, 1, h->g + h->oW3, H)));
    colsum<<<(O + 127) / 128, 128, 0, st>>>(h->dy, B, O, h->g + h->ob3);
    MCK((gemm<float, __nv_bfloat16, EPI_STORE>(st, B, H, O, h->dy, O, 1, W3, H, 1, h->dh, H)));
    gelu_backward<<<blocks(BH), 256, 0, st>>>(h->dh, h->z2, h->dz, BH);
    // layer 2: dW2 = dz2^T h1, db2 = sum dz2, dh1 = dz2 W2
    MCK((gemm<float, float, EPI_STORE>(st, H, H, B, h->dz, 1, H, h->h1, H, 1, h->g + h->oW2, H)));
    colsum<<<(H + 127) / 128, 128, 0, st>>>(h->dz, B, H, h->g + h->ob2);
    MCK((gemm<float, __nv_bfloat16, EPI_STORE>(st, B, H, H, h->dz, H, 1, W2, H, 1, h->dh, H)));
    gelu_backward<<<blocks(BH), 256, 0, st>>>(h->dh, h->z1, h->dz, BH);
    // layer 1: dW1 = dz1^T x, db1 = sum dz1
    MCK((gemm<float, float, EPI_STORE>(st, H, I, B, h->dz, 1, H, x_dev, I, 1, h->g + h->oW1, I)));
    colsum<<<(H + 127) / 128, 128, 0, st>>>(h->dz, B, H, h->g + h->ob1);
    MCK(cudaGetLastError());
    if (loss_out || grad_host) {
        double L = 0.0;
        MCK(cudaMemcpyAsync(&L, h->loss, 8, cudaMemcpyDeviceToHost, st));
        if (grad_host) MCK(cudaMemcpyAsync(grad_host, h->g, h->P * 4, cudaMemcpyDeviceToHost, st));
        MCK(cudaStreamSynchronize(st));
        if (loss_out) *loss_out = L / double(BO);
    }
    return LBS_OK;
}

lbs_status lbs_mlp_adam(lbs_mlp_handle h, float lr, float beta1, float beta2, float eps)
{
    if (!h || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return merr(LBS_ERR_ARG, "Adam needs lr > 0, 0 <= beta < 1, eps > 0");
    h->step += 1;
    const float c1 = 1.f - powf(beta1, float(h->step)), c2 = 1.f - powf(beta2, float(h->step));
    adam<<<blocks(h->P), 256, 0, h->stream>>>(h->p, h->g, h->m, h->v, h->P, lr, beta1, beta2, eps, c1, c2, h->pb,
                                              h->is_w);
    MCK(cudaGetLastError());
    return LBS_OK;
}

lbs_status lbs_mlp_get_stream(lbs_mlp_handle h, void** out)
{
    if (!h || !out) return merr(LBS_ERR_ARG, "invalid handle or null output");
    *out = static_cast<void*>(h->stream);
    return LBS_OK;
}

}  // extern "C"
