// The propagate-and-check sweep alone, for timing it in isolation (device
// code in solver.cuh).
#include "solver.cuh"

namespace aspgpu {

// One sweep over the static store without claiming (timing the sweep kernel
// in isolation): counts unit nogoods in acc->flag, conflicts in acc->ckey.
// Same partition, views and classification as the solver's sweep.
__global__ void __launch_bounds__(768, 1) sweep_kernel(Dev D, Acc *acc, uint32_t passes)
{
    extern __shared__ unsigned long long smem_raw[];
    uint32_t *vbase = reinterpret_cast<uint32_t *>(smem_raw + D.WW + 32) + 16;
    const View V = make_view(D, vbase, blockIdx.x);
    view_reload(D, V, 0u);
    unit_table(D, blockIdx.x);
    cta_sync();
    for (uint32_t pass = 0; pass < (passes ? passes : 1u); pass++) {
        SweepCtx X{&D, V, 0u, 1u, 0u, acc, false, true, 0xFFFFFFFFu, blockIdx.x,
                   (blockIdx.x * blockDim.x + threadIdx.x) >> 5, (gridDim.x * blockDim.x) >> 5};
        sweep<0>(X, 0u, true, 0u, 0u, pass);
    }
}

cudaError_t sweep_configure()
{
    return cudaFuncSetAttribute(sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
}

cudaError_t launch_sweep(const Dev &D, Acc *acc, int grid, int block, size_t smem, cudaStream_t st,
                         uint32_t passes)
{
    sweep_kernel<<<grid, block, smem, st>>>(D, acc, passes);
    return cudaGetLastError();
}

}  // namespace aspgpu
