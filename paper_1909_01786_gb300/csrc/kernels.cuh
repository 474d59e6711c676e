// The solver kernels (device code in solver.cuh), instantiated per
// translation unit: solve.cu and batch.cu without the frontier by units,
// solve_units.cu and batch_units.cu with it.
#pragma once
#include "solver.cuh"

namespace aspgpu {

// The single-program solver: one persistent cooperative kernel over the
// whole grid runs Algorithm 1.
template <bool UNITS>
__global__ void __launch_bounds__(768, 1) solve_kernel(Dev D)
{
    extern __shared__ unsigned long long smem_raw[];
    const Smem S = make_smem(D, smem_raw);
    const View V = make_view(D, S.misc + 16, blockIdx.x);
    solver_loop<false, UNITS>(D, S, V, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, blockIdx.x == 0,
                       blockIdx.x == 0 && threadIdx.x == 0, blockIdx.x);
}

// Batched solving: each CTA takes programs from a queue (the host orders it
// largest first) and solves each alone, with the whole program's assignment
// view in its shared memory and a CTA barrier as the phase barrier.
template <int THREADS, int MIN_BLOCKS, bool UNITS>
__global__ void __launch_bounds__(THREADS, MIN_BLOCKS) batch_kernel(const Dev *devs, const uint32_t *order, uint32_t n,
                                                                    unsigned int *queue)
{
    extern __shared__ unsigned long long smem_raw[];
    __shared__ Dev sD;
    __shared__ uint32_t s_item;
    for (;;) {
        if (threadIdx.x == 0) {
            uint32_t i = atomicAdd(queue, 1u);
            s_item = i < n ? __ldg(order + i) : 0xFFFFFFFFu;
            if (s_item != 0xFFFFFFFFu) sD = devs[s_item];
        }
        cta_sync();
        if (s_item == 0xFFFFFFFFu) break;
        const Dev &D = sD;
        // reset this program's search state
        for (uint32_t w = threadIdx.x; w <= D.asg_words; w += blockDim.x) D.asg[w] = 0u;
        for (uint32_t v = threadIdx.x; v < D.nv; v += blockDim.x) D.dl[v] = 0;
        for (uint32_t j = threadIdx.x; j <= D.J; j += blockDim.x) D.act[j] = 0u;
        if (D.frontier >= 2u)
            for (uint32_t w = threadIdx.x; w < 2u * D.dirty_words; w += blockDim.x) D.dirty[w] = 0u;
        if (threadIdx.x == 0) {
            Ctl c;
            memset(&c, 0, sizeof(c));
            c.op = OP_INIT;
            c.cdl = 1;
            c.lfill = D.lits_static;
            D.ctl[0] = c;
            memset(&c, 0, sizeof(c));
            D.ctl[1] = c;
            Acc a;
            a.ckey = NO_KEY; a.cslot[0] = a.cslot[1] = a.cslot[2] = NO_KEY; a.dkey = 0; a.nclaim = 0; a.flag = 0; a.minU = 0xFFFFFFFFu; a.nlits = 0; a.checks = 0; a.visits = 0; a.tbusy = 0; a.tsweep = 0; a.tlong = 0; a.tbuck = 0;
            for (int i = 0; i < 4; i++) D.acc[i] = a;
            memset(D.stats, 0, sizeof(DevStats));
            memset(D.bar, 0, sizeof(Barrier));   // unused here, read by the final error check
        }
        cta_sync();
        const Smem S = make_smem(D, smem_raw);
        const View V = make_view(D, S.misc + 16, 0);
        solver_loop<true, UNITS>(D, S, V, threadIdx.x, blockDim.x, true, threadIdx.x == 0, 0);
        cta_sync();
    }
}

}  // namespace aspgpu
