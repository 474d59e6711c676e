// Allocation-free unit propagation (asp_propagate_noalloc).
//
// Some callers cannot allocate device memory on the path where they need
// propagation: real-time loops that must not enter the allocator (an
// allocation can block on the driver or trigger a synchronising free of
// cached blocks), and processes whose device memory is handed out up front
// by a pool or a framework that owns all of it.  This entry point computes the
// same closure as asp_debug_propagate, but all of its working memory (the
// assignment codes, the round counters and the grid barrier) lives in one
// fixed static device array defined below.  It reads the program's nogood
// store (created earlier by asp_load_ground) and the caller's device buffers,
// and allocates nothing.
//
// The array is shared by every call in the process: calls that overlap on
// the GPU (two streams, or two host threads) race on it and give wrong
// results.  Each call re-initialises what must start at zero.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "aspgpu.h"
#include "device.cuh"
#include "store.h"

namespace aspgpu {

constexpr uint32_t NOALLOC_CTL_WORDS = 64;
// largest program the static array serves: 2^20 variables (4-bit codes)
constexpr uint32_t NOALLOC_MAX_VARS = 1u << 20;
constexpr uint32_t NOALLOC_WORDS = NOALLOC_CTL_WORDS + NOALLOC_MAX_VARS / 8u;

// 512 KB of codes + 256 B of control words; every GPU that loads the
// library holds it until the process exits.
static __device__ __align__(256) uint32_t g_noalloc_scratch[NOALLOC_WORDS];

namespace {

struct NaCtl {                 // first words of the scratch array
    unsigned int count, gen, err, pad;
    unsigned int nclaim[3];
    unsigned int conflict;
};

__device__ __forceinline__ unsigned long long na_timer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t na_ld_acquire(const unsigned int *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// grid barrier on the scratch control words; bounded wait (~20 s)
__device__ bool na_sync(NaCtl *c)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (gridDim.x > 1) {
            unsigned g = na_ld_acquire(&c->gen);
            __threadfence();
            if (atomicAdd(&c->count, 1u) == gridDim.x - 1) {
                atomicExch(&c->count, 0u);
                __threadfence();
                atomicAdd(&c->gen, 1u);
            } else {
                unsigned long long t0 = na_timer();
                unsigned spins = 0;
                while (na_ld_acquire(&c->gen) == g) {
                    if (na_ld_acquire(&c->err)) { ok = 0; break; }
                    if ((++spins & 1023u) == 0 && na_timer() - t0 > 20000000000ull) {
                        atomicExch(&c->err, 1u);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
        if (na_ld_acquire(&c->err)) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// value of variable v with claims of the current round (fresh bit) unseen
__device__ __forceinline__ uint32_t na_val(const uint32_t *asg, uint32_t v, uint32_t fresh)
{
    uint32_t c = (__ldcg(asg + (v >> 3)) >> ((v & 7u) * 4u)) & 0xFu;
    return (c & fresh) ? 0u : (c & 3u);
}

// claim the complement of literal l; conflict flag on a clash
__device__ __forceinline__ void na_claim(uint32_t *asg, NaCtl *c, uint32_t l, uint32_t fresh, uint32_t slot)
{
    const uint32_t v = l >> 1, valbit = (l & 1u) ? V_T : V_F, sh = (v & 7u) * 4u;
    const uint32_t old = (atomicOr(asg + (v >> 3), (valbit | fresh) << sh) >> sh) & 3u;
    if (old == 0u) atomicAdd(&c->nclaim[slot], 1u);
    else if (!(old & valbit)) atomicExch(&c->conflict, 1u);
}

__global__ void __launch_bounds__(768, 1) noalloc_propagate_kernel(Dev D, const int8_t *partial, int8_t *closure,
                                                                   int32_t *conflict_out, uint32_t *scratch)
{
    NaCtl *c = reinterpret_cast<NaCtl *>(scratch);
    uint32_t *asg = scratch + NOALLOC_CTL_WORDS;
    const uint32_t nth = gridDim.x * blockDim.x, gt = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31u, gw = gt >> 5, nw = nth >> 5;
    const uint32_t words = (D.nv + 7u) >> 3;
    // the caller's partial assignment, committed (no fresh bits)
    for (uint32_t w = gt; w < words; w += nth) {
        uint32_t m = 0;
        for (uint32_t q = 0; q < 8u; q++) {
            uint32_t v = 8u * w + q;
            if (v < D.nv && partial[v]) m |= (partial[v] > 0 ? V_T : V_F) << (4u * q);
        }
        asg[w] = m;
    }
    if (!na_sync(c)) return;
    // round 0 applies the unit nogoods; later rounds sweep the store
    for (uint32_t r = 0;; r++) {
        const uint32_t fresh = 4u << (r & 1u), slot = r % 3u;
        // clear the fresh bits of round r-1 (the other parity)
        const uint32_t old_fresh = 4u << ((r + 1u) & 1u);
        const uint32_t clear = ~(old_fresh * 0x11111111u);
        if (r > 0)
            for (uint32_t w = gt; w < words; w += nth) atomicAnd(asg + w, clear);
        if (gt == 0) c->nclaim[(r + 1u) % 3u] = 0u;
        if (r == 0) {
            for (uint32_t i = gt; i < D.n_units; i += nth) {
                const uint32_t l = __ldg(D.lits + D.units_base + i) & ~END_BIT;
                const uint32_t v = na_val(asg, l >> 1, fresh);
                if (v == 0u) na_claim(asg, c, l, fresh, slot);
                else if (v == ((l & 1u) ? V_F : V_T)) atomicExch(&c->conflict, 1u);
            }
        } else {
            // buckets: one lane per nogood
            for (uint32_t L = 2; L <= (uint32_t)BUCKET_MAX; L++) {
                const uint32_t n = D.bk_n[L];
                const uint32_t *base = D.lits + D.bk_base[L];
                for (uint32_t k = gt; k < n; k += nth) {
                    bool sat = false;
                    uint32_t n_un = 0, ul = 0;
                    for (uint32_t q = 0; q < L && !sat; q++) {
                        const uint32_t l = __ldg(base + (size_t)q * n + k);
                        const uint32_t v = na_val(asg, l >> 1, fresh);
                        if (v == ((l & 1u) ? V_T : V_F)) sat = true;
                        else if (v == 0u) { n_un++; ul = l; }
                    }
                    if (sat || n_un > 1u) continue;
                    if (n_un == 0u) atomicExch(&c->conflict, 1u);
                    else na_claim(asg, c, ul, fresh, slot);
                }
            }
            // long nogoods: one warp per nogood, lanes over literals
            for (uint32_t i = gw; i < D.n_long; i += nw) {
                const uint32_t id = __ldg(D.long_ids + i);
                bool sat = false;
                uint32_t n_un = 0, ul = 0;
                for (uint32_t off = id;; off += 32u) {
                    const uint32_t w = __ldg(D.lits + off + lane);
                    const unsigned Bend = __ballot_sync(0xFFFFFFFFu, (w & END_BIT) != 0u);
                    const unsigned valid = Bend ? ((2u << (__ffs(Bend) - 1)) - 1u) : 0xFFFFFFFFu;
                    const uint32_t l = w & ~END_BIT;
                    const bool mine = (valid >> lane) & 1u;
                    const uint32_t v = mine ? na_val(asg, l >> 1, fresh) : 0u;
                    const unsigned Bopp = __ballot_sync(0xFFFFFFFFu, mine && v == ((l & 1u) ? V_T : V_F));
                    const unsigned Bun = __ballot_sync(0xFFFFFFFFu, mine && v == 0u);
                    const uint32_t first = __shfl_sync(0xFFFFFFFFu, l, Bun ? __ffs(Bun) - 1 : 0);
                    if (Bun && n_un == 0) ul = first;
                    n_un += (uint32_t)__popc(Bun);
                    if (Bopp) { sat = true; break; }
                    if (Bend || n_un > 1u) break;
                }
                if (lane == 0 && !sat) {
                    if (n_un == 0u) atomicExch(&c->conflict, 1u);
                    else if (n_un == 1u) na_claim(asg, c, ul, fresh, slot);
                }
            }
        }
        if (!na_sync(c)) break;
        // every thread sees the same counters after the barrier
        const uint32_t claims = __ldcg(&c->nclaim[slot]);
        const uint32_t conf = __ldcg(&c->conflict);
        if (conf || (r > 0 && claims == 0u)) break;
        if (!na_sync(c)) break;   // nobody may reset a slot still being read
    }
    for (uint32_t v = gt; v < D.nv; v += nth) {
        const uint32_t code = (__ldcg(asg + (v >> 3)) >> ((v & 7u) * 4u)) & 3u;
        closure[v] = code == V_T ? 1 : code == V_F ? -1 : code == 3u ? 2 : 0;
    }
    if (gt == 0) *conflict_out = __ldcg(&c->conflict) ? 1 : (__ldcg(&c->err) ? -1 : 0);
}

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[128];
int g_noalloc_grid[128];

}  // namespace

const Dev *internal_dev(const asp_prog *p);
cudaStream_t internal_stream(const asp_prog *p);
int internal_device(const asp_prog *p);
int internal_fail(int code, const char *msg);

}  // namespace aspgpu

extern "C" int asp_propagate_noalloc(const asp_prog *p, const int8_t *d_partial, int8_t *d_closure,
                                     int32_t *d_conflict)
{
    using namespace aspgpu;
    if (!p || !d_partial || !d_closure || !d_conflict) return internal_fail(ASP_E_ARG, "null argument");
    const Dev *D = internal_dev(p);
    if (D->nv > NOALLOC_MAX_VARS)
        return internal_fail(ASP_E_CAPACITY, "program has more than 2^20 variables, the static working array's limit");
    // the program's stream and store belong to the device it was loaded on;
    // the static array's address is looked up on the current device, so the
    // two must agree
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return internal_fail(ASP_E_CUDA, "no current device");
    if (dev != internal_device(p))
        return internal_fail(ASP_E_ARG, "the current device is not the device the program was loaded on");
    void *scratch = nullptr;
    int grid = 0;
    {
        // once per device, with that device current: the device address of
        // the static array (its host-side name is only a stand-in)
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr)
                return internal_fail(ASP_E_CUDA, "cudaGetSymbolAddress of the static working array failed");
            int sms = 0, per_sm = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
                return internal_fail(ASP_E_CUDA, "reading the multiprocessor count failed");
            // The kernel is compiled for one 768-thread block per SM
            // (__launch_bounds__(768, 1)), so a grid of one CTA per SM always
            // fits a cooperative launch; the occupancy query confirms that
            // at least one block is resident per SM.
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, noalloc_propagate_kernel, 768, 0) != cudaSuccess ||
                per_sm < 1)
                return internal_fail(ASP_E_CUDA, "the propagation kernel cannot be resident on an SM");
            g_noalloc_grid[dev] = sms;
            g_noalloc_ptr[dev] = ptr;
        }
        scratch = g_noalloc_ptr[dev];
        grid = g_noalloc_grid[dev];
    }
    cudaStream_t st = internal_stream(p);
    // the control words start at zero on every call
    if (cudaMemsetAsync(scratch, 0, NOALLOC_CTL_WORDS * sizeof(uint32_t), st) != cudaSuccess)
        return internal_fail(ASP_E_CUDA, "clearing the counters failed");
    Dev copy = *D;
    uint32_t *s = static_cast<uint32_t *>(scratch);
    void *args[] = {(void *)&copy, (void *)&d_partial, (void *)&d_closure, (void *)&d_conflict, (void *)&s};
    if (cudaLaunchCooperativeKernel((void *)noalloc_propagate_kernel, dim3(grid), dim3(768), args, 0, st) != cudaSuccess)
        return internal_fail(ASP_E_CUDA, "launch failed");
    return ASP_OK;
}
