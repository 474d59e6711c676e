// Batched solving: many programs in one launch, one CTA per program.  The
// kernel (kernels.cuh) is compiled once per configuration and frontier mode
// in batch_kernel.cu; this unit dispatches to those instantiations.
#include <cuda_runtime.h>

#include "device.cuh"

namespace aspgpu {

// Batch kernel configurations the autotuner chooses from: threads per CTA
// and the CTAs per SM the register budget is compiled for.
//   0: 256 threads, 3 per SM (programs up to ~70 KB of view)
//   1: 128 threads, 6 per SM (twice the programs in flight, ~34 KB views)
int batch_threads(int config) { return config == 1 ? 128 : 256; }

// batch_kernel.cu, compiled with BATCH_CONFIG = c and BATCH_UNITS = u
#define ASP_BATCH_DECL(c, u)                                                                                  \
    cudaError_t batch_configure_c##c##_u##u(size_t smem, int *blocks_per_sm);                                   \
    cudaError_t launch_batch_c##c##_u##u(const Dev *devs, const uint32_t *order, uint32_t n, unsigned int *queue, \
                                         int grid, size_t smem, cudaStream_t st);
ASP_BATCH_DECL(0, 0)
ASP_BATCH_DECL(0, 1)
ASP_BATCH_DECL(1, 0)
ASP_BATCH_DECL(1, 1)
#undef ASP_BATCH_DECL

// units: the kernels compiled with the frontier by units
cudaError_t batch_configure(int config, bool units, size_t smem, int *blocks_per_sm)
{
    if (config == 1) return units ? batch_configure_c1_u1(smem, blocks_per_sm) : batch_configure_c1_u0(smem, blocks_per_sm);
    return units ? batch_configure_c0_u1(smem, blocks_per_sm) : batch_configure_c0_u0(smem, blocks_per_sm);
}

cudaError_t launch_batch(int config, bool units, const Dev *devs, const uint32_t *order, uint32_t n,
                         unsigned int *queue, int grid, size_t smem, cudaStream_t st)
{
    if (config == 1)
        return units ? launch_batch_c1_u1(devs, order, n, queue, grid, smem, st)
                     : launch_batch_c1_u0(devs, order, n, queue, grid, smem, st);
    return units ? launch_batch_c0_u1(devs, order, n, queue, grid, smem, st)
                 : launch_batch_c0_u0(devs, order, n, queue, grid, smem, st);
}

}  // namespace aspgpu
