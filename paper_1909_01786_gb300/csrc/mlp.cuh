// Forward pass of the learned decision heuristic's MLP, shared by the
// solver's Decision step and the standalone scoring kernel.
#pragma once
#include <cuda_bf16.h>

#include "device.cuh"

namespace aspgpu {

// 16 -> 64 (ReLU) -> 1 with bf16 weights W1[64][16], b1[64], w2[64], b2 and
// fp32 accumulation
__device__ __forceinline__ float mlp_score(const __nv_bfloat16 *W, const float *x)
{
    const __nv_bfloat16 *b1 = W + N_FEATURES * N_HIDDEN, *w2 = b1 + N_HIDDEN;
    float y = __bfloat162float(w2[N_HIDDEN]);
    for (int k = 0; k < N_HIDDEN; k++) {
        float a = __bfloat162float(b1[k]);
#pragma unroll
        for (int i = 0; i < N_FEATURES; i++) a = fmaf(__bfloat162float(W[k * N_FEATURES + i]), x[i], a);
        y = fmaf(__bfloat162float(w2[k]), fmaxf(a, 0.0f), y);
    }
    return y;
}

}  // namespace aspgpu
