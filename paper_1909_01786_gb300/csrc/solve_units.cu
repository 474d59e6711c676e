// The single-program solver with the frontier by units (kernel in
// kernels.cuh).
#include "kernels.cuh"

namespace aspgpu {

cudaError_t solve_units_configure(int block, size_t smem, int *blocks_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(solve_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, solve_kernel<true>, block, smem);
}

cudaError_t launch_solve_units(const Dev &D, int grid, int block, size_t smem, cudaStream_t st)
{
    Dev copy = D;
    void *args[] = {(void *)&copy};
    return cudaLaunchCooperativeKernel((void *)solve_kernel<true>, dim3(grid), dim3(block), args, smem, st);
}

}  // namespace aspgpu
