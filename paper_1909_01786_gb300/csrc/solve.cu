// The single-program solver without the frontier by units (kernel in
// kernels.cuh), and the dispatch to solve_units.cu.
#include "kernels.cuh"

namespace aspgpu {

cudaError_t sweep_configure();

cudaError_t solve_units_configure(int block, size_t smem, int *blocks_per_sm);
cudaError_t launch_solve_units(const Dev &D, int grid, int block, size_t smem, cudaStream_t st);

// Both solve kernels (without and with the frontier by units): the CTAs per
// SM the smaller of the two allows.
cudaError_t solve_configure(int block, size_t smem, int *blocks_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(solve_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    if (e != cudaSuccess) return e;
    e = sweep_configure();
    if (e != cudaSuccess) return e;
    int a = 0, b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, solve_kernel<false>, block, smem);
    if (e == cudaSuccess) e = solve_units_configure(block, smem, &b);
    *blocks_per_sm = a < b ? a : b;
    return e;
}

cudaError_t solve_attributes(cudaFuncAttributes *a) { return cudaFuncGetAttributes(a, solve_kernel<false>); }

cudaError_t launch_solve(const Dev &D, int grid, int block, size_t smem, cudaStream_t st)
{
    if (D.frontier >= 2u) return launch_solve_units(D, grid, block, smem, st);
    Dev copy = D;
    void *args[] = {(void *)&copy};
    return cudaLaunchCooperativeKernel((void *)solve_kernel<false>, dim3(grid), dim3(block), args, smem, st);
}

}  // namespace aspgpu
