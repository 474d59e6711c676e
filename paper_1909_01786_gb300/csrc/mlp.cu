// Training of the learned decision heuristic (not in the paper): a 16-64-1
// MLP, ReLU hidden layer, logistic output, trained by minibatch SGD with
// momentum on binary cross-entropy, in one CTA.  One lane holds one sample;
// gradients are reduced across the warp with shuffles and summed into shared
// memory.  The solver evaluates the trained network with bf16 weights and
// fp32 accumulation (solver.cuh, mlp_score).
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

__global__ void __launch_bounds__(1024, 1) mlp_train_kernel(const float *X, const float *Y, int n, int epochs,
                                                            int batch, float lr, float momentum, float *W)
{
    __shared__ float w[MLP_PARAMS], g[MLP_PARAMS], v[MLP_PARAMS];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    float *W1 = w, *b1 = w + N_FEATURES * N_HIDDEN, *w2 = b1 + N_HIDDEN, *b2 = w2 + N_HIDDEN;
    for (int p = tid; p < MLP_PARAMS; p += blockDim.x) { w[p] = W[p]; v[p] = 0.0f; }
    __syncthreads();
    for (int ep = 0; ep < epochs; ep++) {
        for (int b0 = 0; b0 < n; b0 += batch) {
            const int b1i = b0 + batch < n ? b0 + batch : n;
            const float inv = 1.0f / (float)(b1i - b0);
            for (int p = tid; p < MLP_PARAMS; p += blockDim.x) g[p] = 0.0f;
            __syncthreads();
            for (int s0 = b0 + wid * 32; s0 < b1i; s0 += nw * 32) {
                const int i = s0 + lane;
                const bool ok = i < b1i;
                float x[N_FEATURES];
#pragma unroll
                for (int q = 0; q < N_FEATURES; q++) x[q] = ok ? X[(size_t)i * N_FEATURES + q] : 0.0f;
                // forward
                float logit = b2[0];
                for (int k = 0; k < N_HIDDEN; k++) {
                    float a = b1[k];
#pragma unroll
                    for (int q = 0; q < N_FEATURES; q++) a = fmaf(W1[k * N_FEATURES + q], x[q], a);
                    logit = fmaf(w2[k], fmaxf(a, 0.0f), logit);
                }
                const float p = 1.0f / (1.0f + expf(-logit));
                const float d = ok ? (p - Y[i]) * inv : 0.0f;        // dLoss/dlogit
                // backward, reduced over the warp's 32 samples
                const float gb2 = warp_sum(d);
                if (lane == 0) atomicAdd(&g[MLP_PARAMS - 1], gb2);
                for (int k = 0; k < N_HIDDEN; k++) {
                    float a = b1[k];
#pragma unroll
                    for (int q = 0; q < N_FEATURES; q++) a = fmaf(W1[k * N_FEATURES + q], x[q], a);
                    const float h = fmaxf(a, 0.0f);
                    const float dh = a > 0.0f ? d * w2[k] : 0.0f;
                    const float gw2 = warp_sum(d * h);
                    const float gb1 = warp_sum(dh);
                    if (lane == 0) {
                        atomicAdd(&g[N_FEATURES * N_HIDDEN + N_HIDDEN + k], gw2);
                        atomicAdd(&g[N_FEATURES * N_HIDDEN + k], gb1);
                    }
#pragma unroll
                    for (int q = 0; q < N_FEATURES; q++) {
                        const float gw = warp_sum(dh * x[q]);
                        if (lane == 0) atomicAdd(&g[k * N_FEATURES + q], gw);
                    }
                }
            }
            __syncthreads();
            for (int p = tid; p < MLP_PARAMS; p += blockDim.x) {
                v[p] = momentum * v[p] + g[p];
                w[p] -= lr * v[p];
            }
            __syncthreads();
        }
    }
    for (int p = tid; p < MLP_PARAMS; p += blockDim.x) W[p] = w[p];
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
    if (cudaMalloc(&dX, bx) != cudaSuccess || cudaMalloc(&dY, by) != cudaSuccess || cudaMalloc(&dW, bw) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dX); cudaFree(dY); cudaFree(dW);
        return internal_fail(ASP_E_OOM, "device allocation failed (training data)");
    }
    cudaError_t e = cudaMemcpy(dX, features, bx, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dY, labels, by, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dW, weights, bw, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        mlp_train_kernel<<<1, 1024>>>(dX, dY, (int)n, epochs, 4096, learning_rate, 0.9f, dW);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(weights, dW, bw, cudaMemcpyDeviceToHost);
    cudaFree(dX); cudaFree(dY); cudaFree(dW);
    if (e != cudaSuccess) return internal_fail(ASP_E_CUDA, cudaGetErrorString(e));
    return ASP_OK;
}
