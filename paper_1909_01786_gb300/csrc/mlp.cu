// Training of the learned decision heuristic (not in the paper): a 16-64-1
// MLP, ReLU hidden layer, logistic output, trained by minibatch SGD with
// momentum on binary cross-entropy.  Each minibatch is spread over many
// CTAs, one sample per thread: gradients are reduced across the warp with
// shuffles, summed into shared memory, then added to a global gradient; a
// second kernel applies the momentum step.  The solver evaluates the trained
// network with bf16 weights and fp32 accumulation (solver.cuh, mlp_score).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "aspgpu.h"
#include "device.cuh"
#include "mlp.cuh"

namespace aspgpu {

int internal_fail(int code, const char *msg);

namespace {

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Gradient of the mean binary cross-entropy over samples [i0, i1), added to
// g.  One sample per thread (grid-stride); every warp runs the same number
// of iterations so the shuffles see all 32 lanes.
__global__ void __launch_bounds__(256) mlp_grad_kernel(const float *X, const float *Y, int i0, int i1, const float *W,
                                                       float *g)
{
    __shared__ float w[MLP_PARAMS], gs[MLP_PARAMS];
    const int tid = threadIdx.x, lane = tid & 31;
    for (int p = tid; p < MLP_PARAMS; p += blockDim.x) { w[p] = W[p]; gs[p] = 0.0f; }
    __syncthreads();
    const float *W1 = w, *b1 = w + N_FEATURES * N_HIDDEN, *w2 = b1 + N_HIDDEN, *b2 = w2 + N_HIDDEN;
    const float inv = 1.0f / (float)(i1 - i0);
    const int stride = gridDim.x * blockDim.x;
    for (int base = i0 + blockIdx.x * blockDim.x + (tid & ~31); base < i1; base += stride) {
        const int i = base + lane;
        const bool ok = i < i1;
        float x[N_FEATURES];
#pragma unroll
        for (int q = 0; q < N_FEATURES; q++) x[q] = ok ? X[(size_t)i * N_FEATURES + q] : 0.0f;
        float logit = b2[0];
        for (int k = 0; k < N_HIDDEN; k++) {
            float a = b1[k];
#pragma unroll
            for (int q = 0; q < N_FEATURES; q++) a = fmaf(W1[k * N_FEATURES + q], x[q], a);
            logit = fmaf(w2[k], fmaxf(a, 0.0f), logit);
        }
        const float p = 1.0f / (1.0f + expf(-logit));
        const float d = ok ? (p - Y[i]) * inv : 0.0f;        // dLoss/dlogit
        const float gb2 = warp_sum(d);
        if (lane == 0) atomicAdd(&gs[MLP_PARAMS - 1], gb2);
        for (int k = 0; k < N_HIDDEN; k++) {
            float a = b1[k];
#pragma unroll
            for (int q = 0; q < N_FEATURES; q++) a = fmaf(W1[k * N_FEATURES + q], x[q], a);
            const float h = fmaxf(a, 0.0f);
            const float dh = a > 0.0f ? d * w2[k] : 0.0f;
            const float gw2 = warp_sum(d * h);
            const float gb1 = warp_sum(dh);
            if (lane == 0) {
                atomicAdd(&gs[N_FEATURES * N_HIDDEN + N_HIDDEN + k], gw2);
                atomicAdd(&gs[N_FEATURES * N_HIDDEN + k], gb1);
            }
#pragma unroll
            for (int q = 0; q < N_FEATURES; q++) {
                const float gw = warp_sum(dh * x[q]);
                if (lane == 0) atomicAdd(&gs[k * N_FEATURES + q], gw);
            }
        }
    }
    __syncthreads();
    for (int p = tid; p < MLP_PARAMS; p += blockDim.x)
        if (gs[p] != 0.0f) atomicAdd(&g[p], gs[p]);
}

// SGD with momentum: v = momentum v + g, W -= lr v; the gradient is cleared.
__global__ void mlp_update_kernel(float *W, float *g, float *v, float lr, float momentum)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= MLP_PARAMS) return;
    v[p] = momentum * v[p] + g[p];
    W[p] -= lr * v[p];
    g[p] = 0.0f;
}

// Inference with the solver's arithmetic: bf16 weights, fp32 accumulation.
__global__ void mlp_score_kernel(const uint16_t *Wb, const float *X, int n, float *out)
{
    __shared__ __nv_bfloat16 w[MLP_PARAMS];
    for (int p = threadIdx.x; p < MLP_PARAMS; p += blockDim.x) w[p] = __ushort_as_bfloat16(Wb[p]);
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float x[N_FEATURES];
#pragma unroll
        for (int q = 0; q < N_FEATURES; q++) x[q] = X[(size_t)i * N_FEATURES + q];
        out[i] = mlp_score(w, x);
    }
}

// Static prior of heuristic 3: feature 0 + log sigmoid(MLP) per row.
__global__ void mlp_prior_kernel(const uint16_t *Wb, const float *X, int n, float *out)
{
    __shared__ __nv_bfloat16 w[MLP_PARAMS];
    for (int p = threadIdx.x; p < MLP_PARAMS; p += blockDim.x) w[p] = __ushort_as_bfloat16(Wb[p]);
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float x[N_FEATURES];
#pragma unroll
        for (int q = 0; q < N_FEATURES; q++) x[q] = X[(size_t)i * N_FEATURES + q];
        const float z = mlp_score(w, x);
        const float log_p = z >= 0.0f ? -log1pf(__expf(-z)) : z - log1pf(__expf(z));
        out[i] = x[0] + log_p;
    }
}

}  // namespace

// Per-rule prior of heuristic 3 on the device: features uploaded from the
// host, bf16 weights already on the device, result left in d_out.
int mlp_prior(const uint16_t *d_w, const std::vector<float> &features, int64_t n, float *d_out, cudaStream_t st)
{
    if (n <= 0) return ASP_OK;
    float *dX = nullptr;
    const size_t bx = (size_t)n * N_FEATURES * sizeof(float);
    if (cudaMalloc(&dX, bx) != cudaSuccess) { cudaGetLastError(); return internal_fail(ASP_E_OOM, "device allocation failed (prior)"); }
    cudaError_t e = cudaMemcpyAsync(dX, features.data(), bx, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        mlp_prior_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, st>>>(d_w, dX, (int)n, d_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dX);
    if (e != cudaSuccess) return internal_fail(ASP_E_CUDA, cudaGetErrorString(e));
    return ASP_OK;
}

}  // namespace aspgpu

extern "C" int asp_mlp_score(const float *weights, const float *features, int64_t n, float *scores)
{
    using namespace aspgpu;
    if (!weights || !features || !scores || n <= 0 || n > (1ll << 30)) return internal_fail(ASP_E_ARG, "bad argument");
    std::vector<uint16_t> wb(MLP_PARAMS);
    for (int i = 0; i < MLP_PARAMS; i++) {
        uint32_t u;
        std::memcpy(&u, weights + i, 4);
        wb[i] = (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
    }
    uint16_t *dW = nullptr;
    float *dX = nullptr, *dO = nullptr;
    const size_t bx = (size_t)n * N_FEATURES * sizeof(float), bo = (size_t)n * sizeof(float);
    if (cudaMalloc(&dW, MLP_PARAMS * 2) != cudaSuccess || cudaMalloc(&dX, bx) != cudaSuccess ||
        cudaMalloc(&dO, bo) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dW); cudaFree(dX); cudaFree(dO);
        return internal_fail(ASP_E_OOM, "device allocation failed");
    }
    cudaError_t e = cudaMemcpy(dW, wb.data(), MLP_PARAMS * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dX, features, bx, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        mlp_score_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 1024), 256>>>(dW, dX, (int)n, dO);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(scores, dO, bo, cudaMemcpyDeviceToHost);
    cudaFree(dW); cudaFree(dX); cudaFree(dO);
    if (e != cudaSuccess) return internal_fail(ASP_E_CUDA, cudaGetErrorString(e));
    return ASP_OK;
}

extern "C" int asp_train_mlp(const float *features, const float *labels, int64_t n, int32_t epochs,
                             float learning_rate, float *weights)
{
    using namespace aspgpu;
    if (!features || !labels || !weights || n <= 0 || n > (1ll << 30) || epochs < 0)
        return internal_fail(ASP_E_ARG, "bad argument");
    float *dX = nullptr, *dY = nullptr, *dW = nullptr;
    const size_t bx = (size_t)n * N_FEATURES * sizeof(float), by = (size_t)n * sizeof(float);
    const size_t bw = (size_t)MLP_PARAMS * sizeof(float);
    // dW holds the weights, then the gradient and the momentum
    if (cudaMalloc(&dX, bx) != cudaSuccess || cudaMalloc(&dY, by) != cudaSuccess ||
        cudaMalloc(&dW, 3 * bw) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dX); cudaFree(dY); cudaFree(dW);
        return internal_fail(ASP_E_OOM, "device allocation failed (training data)");
    }
    float *dG = dW + MLP_PARAMS, *dV = dW + 2 * MLP_PARAMS;
    cudaError_t e = cudaMemcpy(dX, features, bx, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dY, labels, by, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dW, weights, bw, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dG, 0, 2 * bw);
    // minibatches of 4096 samples, one sample per thread: 16 CTAs of 256
    const int batch = 4096, threads = 256;
    const int updates = (MLP_PARAMS + 255) / 256;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ep++) {
        for (int64_t b0 = 0; b0 < n && e == cudaSuccess; b0 += batch) {
            const int b1 = (int)std::min<int64_t>(b0 + batch, n);
            const int ctas = (b1 - (int)b0 + threads - 1) / threads;
            mlp_grad_kernel<<<ctas, threads>>>(dX, dY, (int)b0, b1, dW, dG);
            mlp_update_kernel<<<updates, 256>>>(dW, dG, dV, learning_rate, 0.9f);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(weights, dW, bw, cudaMemcpyDeviceToHost);
    cudaFree(dX); cudaFree(dY); cudaFree(dW);
    if (e != cudaSuccess) return internal_fail(ASP_E_CUDA, cudaGetErrorString(e));
    return ASP_OK;
}
