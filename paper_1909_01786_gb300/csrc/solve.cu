// The single-program solver: one persistent cooperative kernel over the
// whole grid runs Algorithm 1 (device code in solver.cuh).
#include "solver.cuh"

namespace aspgpu {

__global__ void __launch_bounds__(768, 1) solve_kernel(Dev D)
{
    extern __shared__ unsigned long long smem_raw[];
    const Smem S = make_smem(D, smem_raw);
    const View V = make_view(D, S.misc + 16, blockIdx.x);
    solver_loop<false>(D, S, V, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, blockIdx.x == 0,
                       blockIdx.x == 0 && threadIdx.x == 0, blockIdx.x);
}

cudaError_t sweep_configure();

cudaError_t solve_configure(int block, size_t smem, int *blocks_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    if (e != cudaSuccess) return e;
    e = sweep_configure();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, solve_kernel, block, smem);
}

cudaError_t solve_attributes(cudaFuncAttributes *a) { return cudaFuncGetAttributes(a, solve_kernel); }

cudaError_t launch_solve(const Dev &D, int grid, int block, size_t smem, cudaStream_t st)
{
    Dev copy = D;
    void *args[] = {(void *)&copy};
    return cudaLaunchCooperativeKernel((void *)solve_kernel, dim3(grid), dim3(block), args, smem, st);
}

}  // namespace aspgpu
