// One instantiation of the batch kernel (kernels.cuh) per compilation:
// BATCH_CONFIG 0 = 256 threads, 3 CTAs per SM; 1 = 128 threads, 6 per SM;
// BATCH_UNITS 1 = with the frontier by units.  The build compiles this file
// four times, so the instantiations compile in parallel.
#include "kernels.cuh"

#ifndef BATCH_CONFIG
#error "BATCH_CONFIG must be 0 or 1"
#endif
#ifndef BATCH_UNITS
#error "BATCH_UNITS must be 0 or 1"
#endif

#define ASP_CAT4(a, b, c, d) a##b##c##d
#define ASP_NAME(a, b, c, d) ASP_CAT4(a, b, c, d)

namespace aspgpu {

constexpr int THREADS = BATCH_CONFIG == 1 ? 128 : 256;
constexpr int MIN_BLOCKS = BATCH_CONFIG == 1 ? 6 : 3;
#define KERNEL batch_kernel<THREADS, MIN_BLOCKS, (BATCH_UNITS != 0)>

cudaError_t ASP_NAME(batch_configure_c, BATCH_CONFIG, _u, BATCH_UNITS)(size_t smem, int *blocks_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, KERNEL, THREADS, smem);
}

cudaError_t ASP_NAME(launch_batch_c, BATCH_CONFIG, _u, BATCH_UNITS)(const Dev *devs, const uint32_t *order, uint32_t n,
                                                                     unsigned int *queue, int grid, size_t smem,
                                                                     cudaStream_t st)
{
    KERNEL<<<grid, THREADS, smem, st>>>(devs, order, n, queue);
    return cudaGetLastError();
}

#undef KERNEL

}  // namespace aspgpu
