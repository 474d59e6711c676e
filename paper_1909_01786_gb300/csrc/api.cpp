// C ABI of libaspgpu: program loading, device memory, launches, results.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "aspgpu.h"
#include "device.cuh"
#include "store.h"

namespace aspgpu {
cudaError_t solve_configure(int block, size_t smem, int *blocks_per_sm);
cudaError_t launch_solve(const Dev &D, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t solve_attributes(cudaFuncAttributes *a);
cudaError_t launch_sweep(const Dev &D, Acc *acc, int grid, int block, size_t smem, cudaStream_t st,
                         uint32_t passes);
int batch_threads(int config);
int mlp_prior(const uint16_t *d_w, const std::vector<float> &features, int64_t n, float *d_out, cudaStream_t st);
cudaError_t batch_configure(int config, bool units, size_t smem, int *blocks_per_sm);
cudaError_t launch_batch(int config, bool units, const Dev *devs, const uint32_t *order, uint32_t n, unsigned int *queue, int grid,
                         size_t smem, cudaStream_t st);
}  // namespace aspgpu

using namespace aspgpu;

static thread_local std::string g_err;

static int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

namespace aspgpu {
int internal_fail(int code, const char *msg) { return fail(code, msg); }
}  // namespace aspgpu

static int cuda_fail(cudaError_t e, const char *what)
{
    return fail(ASP_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// device arrays of a frontier by units (see unit_lists)
struct UnitLists {
    const uint32_t *ubase = nullptr, *uoff = nullptr, *unit = nullptr;
    uint32_t *dirty = nullptr;
    uint32_t words = 0;
    bool built = false;
};

struct asp_prog {
    asp_options opt{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int n_sms = 0;
    struct Buf { void *p; size_t bytes; };
    std::vector<Buf> bufs;
    Dev D{};
    int grid = 1, block = 1024;
    size_t smem = 0;
    // the same program as one CTA solves it in a batch, for each batch
    // kernel configuration (256 threads, 3 per SM; 128 threads, 6 per SM)
    Dev D1[2]{};
    UnitLists batch_units;              // frontier by units in batches
    size_t smem1[2] = {0, 0};
    int64_t n_nogoods = 0, n_literals = 0, n_units = 0, n_long = 0, store_bytes = 0;
    bool empty_nogood = false;
    // internal buffers for the blocking entry points
    long long *d_result = nullptr;
    unsigned long long *d_models = nullptr;
    int64_t d_models_rows = 0;
    Acc *d_sweep_acc = nullptr;
};

namespace aspgpu {
// for entry points defined in other translation units
const Dev *internal_dev(const asp_prog *p) { return &p->D; }
cudaStream_t internal_stream(const asp_prog *p) { return p->stream; }
int internal_device(const asp_prog *p) { return p->device; }
int internal_fail(int code, const char *msg);
}  // namespace aspgpu

// test-only: the n-th device allocation from now on fails (0 = none)
static std::atomic<int64_t> g_alloc_fail_in{0};

static void *dalloc(asp_prog *p, size_t bytes)
{
    bytes = std::max<size_t>(bytes, 16);
    void *ptr = nullptr;
    if (g_alloc_fail_in.load() > 0 && g_alloc_fail_in.fetch_sub(1) == 1) return nullptr;
    if (p->opt.dev_alloc) {
        ptr = p->opt.dev_alloc(bytes, p->opt.alloc_ctx);
    } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
    }
    if (ptr) p->bufs.push_back({ptr, bytes});
    return ptr;
}

static void release_all(asp_prog *p)
{
    if (p->stream) cudaStreamSynchronize(p->stream);
    else cudaDeviceSynchronize();
    for (auto &b : p->bufs) {
        if (p->opt.dev_free) p->opt.dev_free(b.p, b.bytes, p->opt.alloc_ctx);
        else cudaFree(b.p);
    }
    p->bufs.clear();
}

template <class T>
static T *upload(asp_prog *p, const std::vector<T> &v, int &rc)
{
    T *d = (T *)dalloc(p, v.size() * sizeof(T));
    if (!d) { rc = fail(ASP_E_OOM, "device allocation failed"); return nullptr; }
    if (!v.empty()) {
        cudaError_t e = cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, p->stream);
        if (e != cudaSuccess) { rc = cuda_fail(e, "upload"); return nullptr; }
    }
    return d;
}

// shared memory for the heuristic's bf16 weights, after the view
constexpr size_t MLP_SMEM_BYTES = ((2 * MLP_PARAMS + 15) / 16) * 16;

// The buckets' literals rewritten for the view of the CTA that owns each
// nogood: (entry << 2) | (3 if false), with entry = v for an atom and
// aux_base + (v - alo[c]) for an auxiliary variable of the CTA's slice.
// False if some literal names a variable outside the owner's view.
static bool translate_buckets(const Dev &D, const HostStore &H, const std::vector<uint32_t> &boff,
                              uint32_t G, const std::vector<uint32_t> &alo, const std::vector<uint32_t> &an,
                              uint32_t aux_base, std::vector<uint32_t> &out)
{
    const uint32_t G1 = G + 1u;
    out.assign((size_t)D.bk_base[BUCKET_MAX] + (size_t)BUCKET_MAX * D.bk_n[BUCKET_MAX], 0u);
    for (int L = 2; L <= BUCKET_MAX; L++) {
        const std::vector<uint32_t> &rows = H.bucket_rows[L];
        const size_t n = D.bk_n[L];
        for (uint32_t c = 0; c < G; c++) {
            for (uint32_t k = boff[L * G1 + c]; k < boff[L * G1 + c + 1]; k++) {
                for (int q = 0; q < L; q++) {
                    const uint32_t l = rows[(size_t)k * L + q], v = l >> 1;
                    uint32_t e;
                    if (v < D.na) e = v;
                    else if (v - alo[c] < an[c]) e = aux_base + (v - alo[c]);
                    else return false;
                    out[D.bk_base[L] + (size_t)q * n + k] = (e << 2) | ((l & 1u) ? 3u : 0u);
                }
            }
        }
    }
    return true;
}

// View of G CTAs with auxiliary slices (alo, an) in `budget` bytes of
// shared memory after `base` bytes: the widest mode allowed by the options
// that fits (and whose literals translate), else PLAIN with atoms read from
// global memory if they do not fit either.  Sets view_mode, view_atoms,
// view_words and vlits; may clear an[] (PLAIN without auxiliary slice).
static int choose_view(asp_prog *p, const HostStore &H, Dev &D, const std::vector<uint32_t> &boff,
                       const std::vector<uint32_t> &alo, std::vector<uint32_t> &an, size_t base, size_t budget)
{
    uint32_t max_an = 0;
    for (uint32_t x : an) max_an = std::max(max_an, x);
    const uint32_t want = p->opt.view_mode > 0 ? (uint32_t)p->opt.view_mode : (uint32_t)VIEW_BYTES;
    const size_t aux_base = ((size_t)D.na + 15u) / 16u * 16u;
    const size_t bytes_words = (aux_base + max_an + 3u) / 4u;
    const size_t packed_words = aux_base / 16u + (max_an + 15u) / 16u;
    uint32_t mode = VIEW_PLAIN;
    if (want >= VIEW_BYTES && base + 4 * bytes_words <= budget) mode = VIEW_BYTES;
    else if (want >= VIEW_PACKED && base + 4 * packed_words <= budget) mode = VIEW_PACKED;
    std::vector<uint32_t> vl;
    if (mode != VIEW_PLAIN && !translate_buckets(D, H, boff, D.G, alo, an, (uint32_t)aux_base, vl)) mode = VIEW_PLAIN;
    D.view_mode = mode;
    D.vlits = nullptr;
    if (mode != VIEW_PLAIN) {
        D.view_atoms = D.na;
        D.view_words = (uint32_t)(mode == VIEW_BYTES ? bytes_words : packed_words);
        int rc = ASP_OK;
        D.vlits = upload(p, vl, rc);
        return rc;
    }
    size_t atoms_words = (D.na + 15u) / 16u;
    size_t aux_words = (max_an + 15u) / 16u;
    D.view_atoms = D.na;
    if (base + 4 * (atoms_words + aux_words) > budget) {
        // too big for shared memory: keep the auxiliary slice, read atoms globally
        D.view_atoms = 0;
        atoms_words = 0;
        if (base + 4 * aux_words > budget) {
            std::fill(an.begin(), an.end(), 0u);
            aux_words = 0;
        }
    }
    D.view_words = (uint32_t)(atoms_words + aux_words);
    return ASP_OK;
}

// Frontier by units (frontier = 2) over a static partition of G CTAs
// (bucket L's nogoods [boff[L*(G+1)+g], boff[L*(G+1)+g+1]) belong to CTA
// g): the sweep units numbered globally (CTA g's units are [ubase[g],
// ubase[g+1]), in the order the device's unit table gives them: bucket by
// bucket, unit_groups(L) groups of 32 nogoods each), for every variable the
// units whose nogoods hold it, and the two dirty bitmaps.  Sets *built =
// false (and allocates nothing) if the partition has more than max_units.

static int unit_lists(asp_prog *p, const HostStore &H, const std::vector<uint32_t> &boff, uint32_t G,
                      uint64_t max_units, UnitLists &out)
{
    const Dev &D = p->D;
    const uint32_t G1 = G + 1u;
    std::vector<uint32_t> ubase(G1, 0u), lbase((size_t)G * (BUCKET_MAX + 1), 0u);
    for (uint32_t c = 0; c < G; c++) {
        uint32_t acc = 0;
        for (int L = 2; L <= BUCKET_MAX; L++) {
            lbase[(size_t)c * (BUCKET_MAX + 1) + L] = acc;
            const uint32_t n = boff[L * G1 + c + 1] - boff[L * G1 + c];
            const uint32_t groups = (n + 31u) >> 5, per = unit_groups((uint32_t)L);
            acc += (groups + per - 1u) / per;
        }
        ubase[c + 1] = ubase[c] + acc;
    }
    const uint32_t total = ubase[G];
    out.built = false;
    if (total > max_units) return ASP_OK;
    // every (variable, unit) pair once: nogoods are visited in unit order,
    // so a repeat of a pair is always adjacent to its first visit
    std::vector<uint32_t> off((size_t)D.nv + 1, 0u), last((size_t)D.nv, 0xFFFFFFFFu), occ;
    for (int pass = 0; pass < 2; pass++) {
        std::fill(last.begin(), last.end(), 0xFFFFFFFFu);
        std::vector<uint32_t> fill;
        if (pass == 1) {
            for (uint32_t v = 0; v < D.nv; v++) off[v + 1] += off[v];
            occ.resize(off[D.nv]);
            fill.assign(off.begin(), off.end() - 1);
        }
        for (uint32_t c = 0; c < G; c++) {
            for (int L = 2; L <= BUCKET_MAX; L++) {
                const std::vector<uint32_t> &rows = H.bucket_rows[L];
                const uint32_t k0 = boff[L * G1 + c], k1 = boff[L * G1 + c + 1];
                const uint32_t first = ubase[c] + lbase[(size_t)c * (BUCKET_MAX + 1) + L];
                const uint32_t per = unit_groups((uint32_t)L) * 32u;
                for (uint32_t k = k0; k < k1; k++) {
                    const uint32_t u = first + (k - k0) / per;
                    for (int q = 0; q < L; q++) {
                        const uint32_t v = rows[(size_t)k * L + q] >> 1;
                        if (last[v] == u) continue;
                        last[v] = u;
                        if (pass == 0) off[v + 1]++;
                        else occ[fill[v]++] = u;
                    }
                }
            }
        }
    }
    int rc = ASP_OK;
    out.ubase = upload(p, ubase, rc);
    if (rc == ASP_OK) out.uoff = upload(p, off, rc);
    if (rc == ASP_OK) out.unit = upload(p, occ, rc);
    if (rc != ASP_OK) return rc;
    out.words = (total + 31u) / 32u + 1u;
    out.dirty = (uint32_t *)dalloc(p, (size_t)out.words * 2 * 4);
    if (!out.dirty) return fail(ASP_E_OOM, "device allocation failed (dirty bitmaps)");
    cudaError_t e = cudaMemsetAsync(out.dirty, 0, (size_t)out.words * 2 * 4, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "clear dirty bitmaps");
    out.built = true;
    return ASP_OK;
}

// (a partition without lists sweeps everything; one with lists keeps the
// requested unit mode, 2 or 3)
static void use_unit_lists(Dev &D, const UnitLists &U)
{
    D.frontier = U.built ? (D.frontier >= 2u ? D.frontier : 2u) : 0u;
    D.cta_ubase = U.ubase;
    D.occ_uoff = U.uoff;
    D.occ_unit = U.unit;
    D.dirty = U.dirty;
    D.dirty_words = U.words;
}

// Grid size, the static partition of the buckets over the CTAs along groups
// (an atom with its rules; a constraint), each CTA's slice of auxiliary
// variables kept in shared memory, and the shared-memory layout.
static int plan_grid(asp_prog *p, const HostStore &H)
{
    Dev &D = p->D;
    const size_t max_smem = 220 * 1024;
    const size_t base_smem = 8ull * D.WW + 8ull * 32 + 4ull * 16 + MLP_SMEM_BYTES;
    int per_sm = 0;
    cudaError_t e = solve_configure(p->block, max_smem, &per_sm);
    if (e != cudaSuccess) return cuda_fail(e, "kernel configuration");
    if (per_sm < 1) return fail(ASP_E_CUDA, "solver kernel cannot be resident with this block size");
    const int max_grid = p->n_sms * per_sm;
    uint64_t total = 0;
    for (uint64_t x : H.group_lits) total += x;
    // every SM for any real store; one CTA for tiny programs
    int64_t want = (int64_t)(total / 2048) + 1;
    int g = (int)std::max<int64_t>(1, std::min<int64_t>(want, max_grid));
    if (p->opt.grid_ctas > 0) g = std::min(p->opt.grid_ctas, max_grid);
    p->grid = g;
    D.G = (uint32_t)g;
    // groups [glo[i], glo[i+1]) for CTA i, balanced by literal count
    const uint32_t ng = (uint32_t)H.n_groups;
    std::vector<uint32_t> glo(g + 1, ng);
    glo[0] = 0;
    {
        uint64_t acc = 0;
        int next = 1;
        for (uint32_t gi = 0; gi < ng && next < g; gi++) {
            acc += H.group_lits[gi];
            while (next < g && acc * (uint64_t)g >= total * (uint64_t)next) glo[next++] = gi + 1;
        }
        while (next < g) glo[next++] = ng;
    }
    const uint32_t G1 = (uint32_t)g + 1;
    std::vector<uint32_t> boff(16 * (size_t)G1, 0);
    for (int L = 2; L <= BUCKET_MAX; L++) {
        const std::vector<uint32_t> &grp = H.bucket_group[L];
        for (int i = 0; i <= g; i++)
            boff[L * G1 + i] = (uint32_t)(std::lower_bound(grp.begin(), grp.end(), glo[i]) - grp.begin());
    }
    // rules of atom p are [first[p], first[p+1]); their auxiliary variables
    // are na + 3j .. na + 3j + 2
    std::vector<uint32_t> first((size_t)D.na + 1, 0);
    for (uint32_t j = 0; j < D.J; j++) first[H.rule_head[j] + 1]++;
    for (uint32_t a = 0; a < D.na; a++) first[a + 1] += first[a];
    std::vector<uint32_t> alo(g), an(g);
    for (int i = 0; i < g; i++) {
        uint32_t a0 = std::min(glo[i], D.na), a1 = std::min(glo[i + 1], D.na);
        uint32_t j0 = first[a0], j1 = first[a1];
        alo[i] = D.na + 3 * j0;
        an[i] = 3 * (j1 - j0);
    }
    int rc = choose_view(p, H, D, boff, alo, an, base_smem, max_smem);
    if (rc != ASP_OK) return rc;
    p->smem = base_smem + 4 * D.view_words;
    if (D.frontier >= 2) {
        UnitLists U;
        rc = unit_lists(p, H, boff, D.G, ~0ull, U);
        if (rc != ASP_OK) return rc;
        use_unit_lists(D, U);
    }
    D.cta_boff = upload(p, boff, rc);
    if (rc == ASP_OK) D.cta_auxlo = upload(p, alo, rc);
    if (rc == ASP_OK) D.cta_auxn = upload(p, an, rc);
    if (rc != ASP_OK) return rc;
    e = solve_configure(p->block, p->smem, &per_sm);
    if (e != cudaSuccess) return cuda_fail(e, "kernel configuration");
    if (per_sm < 1) return fail(ASP_E_CUDA, "solver kernel cannot be resident");
    return ASP_OK;
}

// Single-CTA layout of the program for batched solving: the whole store is
// the CTA's range, and the view holds every atom and auxiliary variable if
// they fit in the per-CTA shared-memory budget of the batch kernel
// configuration (3 or 6 CTAs in an SM's 228 KB, less reserved and static
// shared memory).
constexpr size_t BATCH_SMEM_BUDGET[2] = {72 * 1024 - 1024, 34 * 1024};
// frontier by units in batches: the unit lists of a program's single-CTA
// partition are built for programs of at most this many sweep units (about
// 20k atoms at 4 rules per atom), whatever the program's own frontier option,
// so that the batch autotuner can choose between full sweeps and the unit
// frontier
constexpr uint64_t BATCH_MAX_UNITS = 1u << 14;

static int plan_batch(asp_prog *p, const HostStore &H, int config)
{
    Dev D1 = p->D;
    std::vector<uint32_t> boff(32, 0), alo(1), an(1);
    for (int L = 2; L <= BUCKET_MAX; L++) boff[L * 2 + 1] = (uint32_t)H.bucket_group[L].size();
    alo[0] = D1.na;
    an[0] = 3 * D1.J;
    const size_t base = 8ull * D1.WW + 8ull * 32 + 4ull * 16 + MLP_SMEM_BYTES;
    D1.G = 1;
    int rc = choose_view(p, H, D1, boff, alo, an, base, BATCH_SMEM_BUDGET[config]);
    if (rc != ASP_OK) return rc;
    D1.cta_boff = upload(p, boff, rc);
    if (rc == ASP_OK) D1.cta_auxlo = upload(p, alo, rc);
    if (rc == ASP_OK) D1.cta_auxn = upload(p, an, rc);
    if (rc == ASP_OK) {
        // one program per CTA: the units of the whole store (the same for
        // both configurations), for programs small enough for batches.  The
        // descriptor keeps the program's own choice (the unit frontier if
        // it asked for it and the lists exist, no chaining in batches); a
        // batch's autotuner may switch every program with lists to it
        if (config == 0) rc = unit_lists(p, H, boff, 1u, BATCH_MAX_UNITS, p->batch_units);
        if (rc == ASP_OK) {
            const uint32_t own = D1.frontier;
            use_unit_lists(D1, p->batch_units);
            D1.frontier = own >= 2u ? (p->batch_units.built ? 2u : 0u) : own;
        }
    }
    p->D1[config] = D1;
    p->smem1[config] = base + 4 * D1.view_words;
    return rc;
}

// A batch prepared for repeated solving: per-program descriptors of the
// chosen kernel configuration in device memory, and the launch (queue reset
// + batch kernel) captured in a CUDA graph.
struct asp_batch {
    std::vector<asp_prog *> progs;
    std::vector<int64_t> caps;
    int64_t max_models_each = 0;
    int config = 0, grid = 0;
    bool units = false;                 // the unit-frontier kernels (programs with unit lists use them)
    size_t smem = 0;
    // autotuner trial times per program: configurations 0 and 1 with full
    // sweeps, then with the unit frontier (0 = not tried, < 0 = cannot run)
    double trial_ns[4] = {0.0, 0.0, 0.0, 0.0};
    uint32_t queued = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

// autotuner trials solve each sampled program with at most this many
// conflicts and this much device time (the same short work for every
// configuration)
constexpr long long TRIAL_CONFLICTS = 8, TRIAL_TIME_NS = 500000000ll;

// descriptors of every program of the batch for kernel configuration
// `config` (trial: the autotuner's shortened budgets)
std::vector<Dev> batch_descriptors(const asp_batch *b, int config, bool trial = false)
{
    std::vector<Dev> devs(b->progs.size());
    for (size_t i = 0; i < b->progs.size(); i++) {
        asp_prog *p = b->progs[i];
        Dev d = p->D1[config];
        // the batch's propagation schedule: the unit frontier for programs
        // with lists, or no unit frontier at all
        if (b->units && p->batch_units.built) d.frontier = 2u;
        else if (!b->units && d.frontier >= 2u) d.frontier = 0u;
        d.mode = MODE_SOLVE;
        d.max_models = b->max_models_each;
        d.models_cap = b->caps[i];
        d.models = p->d_models;
        d.result = p->d_result;
        d.conflict_budget = p->opt.conflict_budget;
        d.time_budget_ns = p->opt.time_budget_ms > 0 ? p->opt.time_budget_ms * 1000000ll : 0;
        if (trial) {
            d.conflict_budget = d.conflict_budget > 0 ? std::min(d.conflict_budget, TRIAL_CONFLICTS) : TRIAL_CONFLICTS;
            d.time_budget_ns = d.time_budget_ns > 0 ? std::min(d.time_budget_ns, TRIAL_TIME_NS) : TRIAL_TIME_NS;
            d.max_models = 1;
        }
        devs[i] = d;
    }
    return devs;
}

// Upload the descriptors of configuration `config` and the queue `order`
// (device scratch: descriptors | order | queue) and size the grid.
int batch_prepare(asp_batch *b, int config, const std::vector<uint32_t> &order, bool trial = false)
{
    const size_t n = b->progs.size();
    size_t smem = 0;
    for (asp_prog *p : b->progs) smem = std::max(smem, p->smem1[config]);
    int per_sm = 0;
    cudaError_t e = batch_configure(config, b->units, smem, &per_sm);
    if (e != cudaSuccess) return cuda_fail(e, "batch configuration");
    if (per_sm < 1) return fail(ASP_E_CUDA, "batch kernel cannot be resident");
    const std::vector<Dev> devs = batch_descriptors(b, config, trial);
    Dev *d_devs = (Dev *)b->scratch;
    uint32_t *d_order = (uint32_t *)((char *)b->scratch + sizeof(Dev) * n);
    e = cudaMemcpyAsync(d_devs, devs.data(), sizeof(Dev) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_order, order.data(), 4 * order.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);     // host vectors go out of scope
    if (e != cudaSuccess) return cuda_fail(e, "batch descriptors");
    b->config = config;
    b->grid = (int)std::min<int64_t>((int64_t)b->progs[0]->n_sms * per_sm, (int64_t)order.size());
    b->smem = smem;
    b->queued = (uint32_t)order.size();
    return ASP_OK;
}

// enqueue one batch launch as prepared: reset the queue counter, launch
cudaError_t batch_enqueue(asp_batch *b)
{
    const size_t n = b->progs.size();
    Dev *d_devs = (Dev *)b->scratch;
    uint32_t *d_order = (uint32_t *)((char *)b->scratch + sizeof(Dev) * n);
    unsigned int *d_queue = (unsigned int *)((char *)d_order + 4 * n);
    cudaError_t e = cudaMemsetAsync(d_queue, 0, 64, b->stream);
    if (e == cudaSuccess) e = launch_batch(b->config, b->units, d_devs, d_order, b->queued, d_queue, b->grid, b->smem, b->stream);
    return e;
}

// autotuner trial: configuration `config` on the programs `sample`, device
// time per program in ns (< 0 if the configuration cannot run)
double batch_trial(asp_batch *b, int config, const std::vector<uint32_t> &sample)
{
    if (batch_prepare(b, config, sample, true) != ASP_OK) { g_err.clear(); return -1.0; }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.0f;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
    if (e == cudaSuccess) e = batch_enqueue(b);
    if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) { cudaGetLastError(); return -1.0; }
    return (double)ms * 1e6 / (double)sample.size();
}

}  // namespace

extern "C" {

void asp_default_options(asp_options *opt)
{
    if (opt) std::memset(opt, 0, sizeof(*opt));
}

const char *asp_last_error(void) { return g_err.c_str(); }

int asp_load_ground(int32_t n_atoms, int32_t n_rules, const int32_t *head,
                    const int64_t *pos_off, const int32_t *pos,
                    const int64_t *neg_off, const int32_t *neg,
                    const asp_options *opt, asp_prog **out)
{
    g_err.clear();
    if (!out) return fail(ASP_E_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(ASP_E_NODEVICE, "no CUDA device");
    }
    HostStore H;
    std::string err;
    int rc = build_store(n_atoms, n_rules, head, pos_off, pos, neg_off, neg, H, err,
                         opt && opt->compact != 0);
    if (rc != ASP_OK) return fail(rc, err);

    asp_prog *p = new asp_prog();
    if (opt) p->opt = *opt;
    p->stream = (cudaStream_t)p->opt.cuda_stream;
    cudaGetDevice(&p->device);
    cudaDeviceGetAttribute(&p->n_sms, cudaDevAttrMultiProcessorCount, p->device);
    p->block = p->opt.block_threads > 0 ? std::min(768, (p->opt.block_threads + 31) / 32 * 32) : 768;

    Dev &D = p->D;
    D.na = (uint32_t)H.n_atoms;
    D.J = (uint32_t)H.n_headed;
    D.nv = (uint32_t)H.n_vars;
    D.asg_words = (D.nv + 7u) / 8u;
    D.n_long = (uint32_t)H.long_rel.size();
    D.n_units = (uint32_t)H.units.size();
    // literal array: buckets (structure-of-arrays) | long CSR | units | learned
    std::vector<uint32_t> lits;
    unsigned long long bucket_lits = 0, bucket_ngs = 0;
    for (int L = 2; L <= BUCKET_MAX; L++) {
        const std::vector<uint32_t> &rows = H.bucket_rows[L];
        const uint32_t n = (uint32_t)H.bucket_group[L].size();
        D.bk_base[L] = (uint32_t)lits.size();
        D.bk_n[L] = n;
        for (int q = 0; q < L; q++)
            for (uint32_t k = 0; k < n; k++) lits.push_back(rows[(size_t)k * L + q]);
        bucket_lits += (unsigned long long)L * n;
        bucket_ngs += n;
    }
    std::vector<uint32_t> long_ids(H.long_rel.size());
    const uint32_t long_base = (uint32_t)lits.size();
    for (size_t i = 0; i < H.long_rel.size(); i++) long_ids[i] = long_base + H.long_rel[i];
    lits.insert(lits.end(), H.long_lits.begin(), H.long_lits.end());
    D.units_base = (uint32_t)lits.size();
    for (uint32_t u : H.units) lits.push_back(u | END_BIT);
    D.lits_static = (uint32_t)lits.size();
    D.static_checks = bucket_lits;
    D.static_nogoods = bucket_ngs;
    int64_t lcap = p->opt.learned_capacity > 0 ? p->opt.learned_capacity
                                               : std::min<int64_t>(std::max<int64_t>(1 << 24, 8 * (int64_t)lits.size()), 1 << 28);
    if ((int64_t)D.lits_static + lcap + 128 >= (int64_t)0xFFFFFF00ll) lcap = (int64_t)0xFFFFFF00ll - D.lits_static - 128;
    D.lits_cap = (uint32_t)(D.lits_static + lcap);
    D.learned_ng_cap = (uint32_t)std::min<int64_t>(lcap / 2 + 1024, 1 << 28);
    int levels = p->opt.deps_levels > 0 ? p->opt.deps_levels : 4096;
    uint32_t WW = (uint32_t)((levels + 63) / 64);
    uint32_t need = (D.J + 2u + 63u) / 64u;   // deepest possible level is J + 1
    WW = std::max<uint32_t>(1u, std::min(WW, need));
    D.WW = WW;
    D.Wlevels = WW * 64u;
    D.heuristic = (uint32_t)std::max(0, p->opt.heuristic);
    if (D.heuristic > 5) { delete p; return fail(ASP_E_ARG, "unknown heuristic"); }
    if (p->opt.learning < 0 || p->opt.learning > 1) { delete p; return fail(ASP_E_ARG, "unknown learning"); }
    D.learning = (uint32_t)p->opt.learning;
    if (p->opt.backjump < 0 || p->opt.backjump > 1 || p->opt.restart_conflicts < 0) {
        delete p;
        return fail(ASP_E_ARG, "unknown backjump or negative restart_conflicts");
    }
    D.backjump = (uint32_t)p->opt.backjump;
    D.restart_unit = (uint32_t)p->opt.restart_conflicts;
    if (p->opt.conflicts_per_round < 0 || p->opt.conflicts_per_round > 4) {
        delete p;
        return fail(ASP_E_ARG, "conflicts_per_round must be 0..4");
    }
    D.conf_per_round = (uint32_t)std::max(1, p->opt.conflicts_per_round);
    if (p->opt.frontier < 0 || p->opt.frontier > 3) { delete p; return fail(ASP_E_ARG, "unknown frontier mode"); }
    D.frontier = (uint32_t)p->opt.frontier;
    D.stall_cta = 0xFFFFFFFFu;
    D.barrier_ns = 20000000000ull;
    p->n_nogoods = H.n_nogoods;
    p->n_literals = H.n_literals;
    p->n_units = (int64_t)H.units.size();
    p->n_long = (int64_t)H.long_rel.size();
    p->empty_nogood = H.has_empty_nogood;
    p->store_bytes = (int64_t)D.lits_static * 4;

    rc = ASP_OK;
    D.lits = (uint32_t *)dalloc(p, ((size_t)D.lits_cap + 128) * 4);
    if (!D.lits) rc = fail(ASP_E_OOM, "device allocation failed (nogood store)");
    if (rc == ASP_OK) {
        cudaError_t e = cudaMemcpyAsync(D.lits, lits.data(), lits.size() * 4, cudaMemcpyHostToDevice, p->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "upload store");
        if (rc == ASP_OK) e = cudaMemsetAsync(D.lits + lits.size(), 0xFF, ((size_t)D.lits_cap + 128 - lits.size()) * 4, p->stream);
        if (rc == ASP_OK && e != cudaSuccess) rc = cuda_fail(e, "clear learned region");
    }
    if (rc == ASP_OK) D.long_ids = upload(p, long_ids, rc);
    if (rc == ASP_OK) D.rule_head = upload(p, H.rule_head, rc);
    if (rc == ASP_OK) D.rpos_off = upload(p, H.rpos_off, rc);
    if (rc == ASP_OK) D.rpos = upload(p, H.rpos, rc);
    if (rc == ASP_OK) D.rneg_off = upload(p, H.rneg_off, rc);
    if (rc == ASP_OK) D.rneg = upload(p, H.rneg, rc);
    if (rc == ASP_OK) D.score = upload(p, D.heuristic == 4 ? H.score_jw : H.score, rc);
    if (rc == ASP_OK) D.rfeat = upload(p, H.rfeat, rc);
    if (rc == ASP_OK && (D.heuristic == 2 || D.heuristic == 3)) {
        if (!p->opt.mlp_weights) rc = fail(ASP_E_ARG, "learned heuristic without mlp_weights");
        else {
            // bf16 by round-to-nearest-even of the float bits
            std::vector<uint16_t> w(MLP_PARAMS);
            for (int i = 0; i < MLP_PARAMS; i++) {
                uint32_t u;
                std::memcpy(&u, p->opt.mlp_weights + i, 4);
                w[i] = (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
            }
            D.mlp = upload(p, w, rc);
        }
    }
    if (rc == ASP_OK && D.heuristic == 3) {
        // the search-state features at their values before the first
        // decision: activity 0, every negative body atom unassigned, none
        // false, level 1, no conflicts, empty trail
        std::vector<float> X((size_t)D.J * N_FEATURES, 0.0f);
        for (uint32_t j = 0; j < D.J; j++) {
            float *x = X.data() + (size_t)j * N_FEATURES;
            for (int q = 0; q < RULE_STATIC_FEATURES; q++) x[q] = H.rfeat[(size_t)j * RULE_STATIC_FEATURES + q];
            x[9] = (float)(H.rneg_off[j + 1] - H.rneg_off[j]);
            x[11] = 1.0f / 64.0f;
        }
        float *prior = (float *)dalloc(p, (size_t)D.J * sizeof(float) + 4);
        if (!prior) rc = fail(ASP_E_OOM, "device allocation failed (prior)");
        else rc = mlp_prior(D.mlp, X, (int64_t)D.J, prior, p->stream);
        D.prior = prior;
    }
    if (rc == ASP_OK && p->opt.trace_capacity > 0) {
        D.trace_cap = (uint32_t)std::min<int64_t>(p->opt.trace_capacity, 1 << 24);
        D.trace = (uint32_t *)dalloc(p, (size_t)D.trace_cap * TRACE_WORDS * 4);
        if (!D.trace) rc = fail(ASP_E_OOM, "device allocation failed (trace)");
    }
    auto alloc = [&](size_t bytes) -> void * {
        if (rc != ASP_OK) return nullptr;
        void *q = dalloc(p, bytes);
        if (!q) rc = fail(ASP_E_OOM, "device allocation failed");
        return q;
    };
    D.learned_ids = (uint32_t *)alloc((size_t)D.learned_ng_cap * 4);
    D.nwatch = (uint2 *)alloc(((size_t)D.n_long + D.learned_ng_cap) * sizeof(uint2));
    if (rc == ASP_OK && D.n_long > 0) {
        // long static nogoods (more than BUCKET_MAX literals) watch their first two
        std::vector<uint2> w0(D.n_long, make_uint2(0u, 1u));
        cudaError_t e = cudaMemcpyAsync(D.nwatch, w0.data(), w0.size() * sizeof(uint2), cudaMemcpyHostToDevice, p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "watches");
    }
    D.act = (uint32_t *)alloc((size_t)D.J * 4 + 8);
    if (rc == ASP_OK && D.heuristic == 5) {
        std::vector<uint32_t> hf((size_t)D.na + 1, 0u);
        for (uint32_t j = 0; j < D.J; j++) hf[(size_t)H.rule_head[j] + 1]++;
        for (uint32_t a = 0; a < D.na; a++) hf[a + 1] += hf[a];
        D.head_first = upload(p, hf, rc);
    }
    D.asg = (uint32_t *)alloc((size_t)D.asg_words * 4 + 4);
    D.dl = (int32_t *)alloc((size_t)D.nv * 4 + 4);
    D.reason = (uint32_t *)alloc((size_t)D.nv * 4 + 4);
    D.deps = (unsigned long long *)alloc((size_t)D.nv * WW * 8 + 8);
    D.trail = (uint32_t *)alloc((size_t)D.nv * 4 + 4);
    D.level_start = (uint32_t *)alloc(((size_t)D.J + 4) * 4);
    D.dec_var = (uint32_t *)alloc(((size_t)D.J + 4) * 4);
    D.lm = (uint32_t *)alloc(((size_t)D.na + 31) / 32 * 4 + 4);
    D.ctl = (Ctl *)alloc(sizeof(Ctl) * 2);
    D.acc = (Acc *)alloc(sizeof(Acc) * 4);
    D.stats = (DevStats *)alloc(sizeof(DevStats));
    D.bar = (Barrier *)alloc(sizeof(Barrier));
    p->d_result = (long long *)alloc(sizeof(long long) * 4);
    p->d_sweep_acc = (Acc *)alloc(sizeof(Acc));
    if (D.learning) {
        D.tpos = (uint32_t *)alloc((size_t)D.nv * 4 + 4);
        D.stamp = (uint32_t *)alloc((size_t)D.nv * 4 + 4);
        D.cand = (uint32_t *)alloc(((size_t)D.nv + 31) / 32 * 4 + 8);
        D.epoch = (uint32_t *)alloc(16);
        if (rc == ASP_OK) {
            cudaError_t e = cudaMemsetAsync(D.stamp, 0, (size_t)D.nv * 4 + 4, p->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(D.epoch, 0, 16, p->stream);
            if (e != cudaSuccess) rc = cuda_fail(e, "clear stamps");
        }
    }
    if (rc == ASP_OK && p->opt.frontier == 1) {
        // per variable, the ids of the bucket nogoods it occurs in
        std::vector<uint32_t> off((size_t)D.nv + 1, 0), occ;
        for (int L = 2; L <= BUCKET_MAX; L++) {
            const std::vector<uint32_t> &rows = H.bucket_rows[L];
            for (size_t t = 0; t < rows.size(); t++) off[(rows[t] >> 1) + 1]++;
        }
        for (uint32_t v = 0; v < D.nv; v++) off[v + 1] += off[v];
        occ.resize(off[D.nv]);
        std::vector<uint32_t> fill(off.begin(), off.end() - 1);
        for (int L = 2; L <= BUCKET_MAX; L++) {
            const std::vector<uint32_t> &rows = H.bucket_rows[L];
            for (size_t t = 0; t < rows.size(); t++)
                occ[fill[rows[t] >> 1]++] = bucket_nogood_id((uint32_t)L, (uint32_t)(t / (size_t)L));
        }
        D.frontier = 1;
        D.occ_off = upload(p, off, rc);
        if (rc == ASP_OK) D.occ = upload(p, occ, rc);
    }
    if (rc == ASP_OK) rc = plan_grid(p, H);
    if (rc == ASP_OK) rc = plan_batch(p, H, 0);
    if (rc == ASP_OK) rc = plan_batch(p, H, 1);
    if (rc == ASP_OK) {
        cudaError_t e = p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = cuda_fail(e, "load");
    }
    if (rc != ASP_OK) {
        release_all(p);
        delete p;
        return rc;
    }
    *out = p;
    return ASP_OK;
}

void asp_free(asp_prog *p)
{
    if (!p) return;
    release_all(p);
    delete p;
}

}  // extern "C"

// Reset the search state on the stream and set the first control block.
static int reset_state(asp_prog *p, uint32_t mode, int64_t max_models, int64_t models_cap,
                       unsigned long long *d_models, long long *d_result,
                       uint32_t n_input)
{
    Dev &D = p->D;
    cudaStream_t st = p->stream;
    cudaError_t e = cudaSuccess;
    if (mode == MODE_SOLVE) {
        e = cudaMemsetAsync(D.asg, 0, (size_t)D.asg_words * 4 + 4, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(D.dl, 0, (size_t)D.nv * 4 + 4, st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(D.act, 0, (size_t)D.J * 4 + 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.stats, 0, sizeof(DevStats), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.bar, 0, sizeof(Barrier), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.level_start, 0, ((size_t)D.J + 4) * 4, st);
    if (e == cudaSuccess && D.dirty) e = cudaMemsetAsync(D.dirty, 0, (size_t)D.dirty_words * 2 * 4, st);
    static thread_local Ctl ctl[2];
    static thread_local Acc acc[4];
    std::memset(ctl, 0, sizeof(ctl));
    ctl[0].op = OP_INIT;
    ctl[0].cdl = 1;
    ctl[0].tc = n_input;
    ctl[0].tb = n_input;
    ctl[0].lfill = D.lits_static;
    for (int i = 0; i < 4; i++) {
        acc[i].ckey = NO_KEY; acc[i].cslot[0] = acc[i].cslot[1] = acc[i].cslot[2] = NO_KEY; acc[i].dkey = 0; acc[i].nclaim = 0; acc[i].flag = 0;
        acc[i].minU = 0xFFFFFFFFu; acc[i].nlits = 0; acc[i].checks = 0; acc[i].visits = 0; acc[i].tbusy = 0; acc[i].tsweep = 0; acc[i].tlong = 0; acc[i].tbuck = 0;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(D.ctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(D.acc, acc, sizeof(acc), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "reset");
    D.mode = mode;
    D.max_models = max_models;
    D.models_cap = models_cap;
    D.models = d_models;
    D.result = d_result;
    D.conflict_budget = p->opt.conflict_budget;
    D.time_budget_ns = p->opt.time_budget_ms > 0 ? p->opt.time_budget_ms * 1000000ll : 0;
    return ASP_OK;
}

static void fill_stats(const asp_prog *p, const DevStats &s, asp_stats_t &o)
{
    std::memset(&o, 0, sizeof(o));
    const Dev &D = p->D;
    o.n_vars = D.nv; o.n_atoms = D.na; o.n_rules_with_head = D.J;
    o.n_nogoods = p->n_nogoods; o.n_literals = p->n_literals;
    o.n_unit_nogoods = p->n_units; o.n_long_nogoods = p->n_long; o.store_bytes = p->store_bytes;
    o.rounds = (int64_t)s.rounds; o.literal_checks = (int64_t)s.checks; o.propagations = (int64_t)s.props;
    o.conflicts = (int64_t)s.conflicts; o.decisions = (int64_t)s.decisions; o.completions = (int64_t)s.completions;
    o.learned = (int64_t)s.learned; o.learned_literals = (int64_t)s.learned_lits; o.loop_nogoods = (int64_t)s.loops;
    o.models = (int64_t)s.models; o.max_level = (int64_t)s.max_level;
    o.ns_total = (int64_t)s.ns_total; o.ns_sweep = (int64_t)s.ns_sweep; o.ns_analysis = (int64_t)s.ns_analysis;
    o.ns_decision = (int64_t)s.ns_decision; o.ns_stability = (int64_t)s.ns_stab;
    o.ns_buckets = (int64_t)s.ns_buckets; o.ns_learned = (int64_t)s.ns_learned; o.ns_barrier = (int64_t)s.ns_barrier;
    o.view_mode = D.view_mode; o.batch_view_mode = p->D1[0].view_mode;
    o.ns_slowest_cta = (int64_t)s.ns_slowest; o.ns_slowest_sweep = (int64_t)s.ns_slowest_sweep;
    o.ns_slowest_long = (int64_t)s.ns_slowest_long; o.ns_slowest_buckets = (int64_t)s.ns_slowest_buckets;
    o.restarts = (int64_t)s.restarts; o.conflict_rounds = (int64_t)s.conflict_rounds;
    o.nogood_visits = (int64_t)s.visits;
}

extern "C" {

int asp_solve_async(asp_prog *p, int64_t max_models, uint64_t *d_models, int64_t models_cap, int64_t *d_result)
{
    g_err.clear();
    if (!p || !d_result || max_models < 0 || models_cap < 0 || (models_cap > 0 && !d_models))
        return fail(ASP_E_ARG, "bad argument");
    if (p->empty_nogood) {
        // a constraint with an empty body: no interpretation satisfies it
        long long r[4] = {ASP_STATUS_UNSAT, 0, 0, 1};
        cudaError_t e = cudaMemcpyAsync(d_result, r, sizeof(r), cudaMemcpyHostToDevice, p->stream);
        return e == cudaSuccess ? ASP_OK : cuda_fail(e, "result");
    }
    int rc = reset_state(p, MODE_SOLVE, max_models, models_cap, (unsigned long long *)d_models,
                         (long long *)d_result, 0);
    if (rc != ASP_OK) return rc;
    cudaError_t e = launch_solve(p->D, p->grid, p->block, p->smem, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "launch");
    return ASP_OK;
}

static int finish(asp_prog *p, long long *res)
{
    cudaError_t e = p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "solve");
    e = cudaMemcpy(res, p->d_result, sizeof(long long) * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "result");
    return ASP_OK;
}

int asp_solve(asp_prog *p, int64_t max_models, uint64_t *models, int64_t models_cap,
              int64_t *n_models, int32_t *status)
{
    g_err.clear();
    if (!p || max_models < 0 || models_cap < 0 || (models_cap > 0 && !models))
        return fail(ASP_E_ARG, "bad argument");
    const int64_t words = ((int64_t)p->D.na + 63) / 64;
    int64_t rows = std::max<int64_t>(models_cap, 1);
    if (rows > p->d_models_rows) {
        void *q = dalloc(p, (size_t)(rows * std::max<int64_t>(words, 1)) * 8);
        if (!q) return fail(ASP_E_OOM, "device allocation failed (models)");
        p->d_models = (unsigned long long *)q;
        p->d_models_rows = rows;
    }
    int rc = asp_solve_async(p, max_models, (uint64_t *)p->d_models, models_cap, (int64_t *)p->d_result);
    if (rc != ASP_OK) return rc;
    long long res[4];
    if (p->empty_nogood) {
        cudaError_t e = p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "solve");
        if (n_models) *n_models = 0;
        if (status) *status = ASP_STATUS_UNSAT;
        return ASP_OK;
    }
    rc = finish(p, res);
    if (rc != ASP_OK) return rc;
    int64_t got = res[1];
    int64_t copy = std::min<int64_t>(got, models_cap);
    if (copy > 0 && words > 0) {
        cudaError_t e = cudaMemcpy(models, p->d_models, (size_t)(copy * words) * 8, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "models");
    }
    if (n_models) *n_models = got;
    if (status) *status = (int32_t)res[0];
    if (res[2] != 0) return fail(ASP_E_DEVICE, "device-side error (learned store full or barrier timeout)");
    if (got > models_cap) return fail(ASP_E_CAPACITY, "more answer sets than model buffer rows");
    return ASP_OK;
}

int asp_stats(const asp_prog *p, asp_stats_t *out)
{
    if (!p || !out) return fail(ASP_E_ARG, "bad argument");
    cudaError_t e = p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "stats sync");
    DevStats s;
    e = cudaMemcpy(&s, p->D.stats, sizeof(s), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "stats");
    fill_stats(p, s, *out);
    return ASP_OK;
}

int asp_debug_propagate(asp_prog *p, const int8_t *partial, int8_t *closure, int32_t *conflict)
{
    g_err.clear();
    if (!p || !partial || !closure) return fail(ASP_E_ARG, "bad argument");
    const Dev &D = p->D;
    std::vector<uint32_t> asg(D.asg_words + 1, 0u), trail;
    std::vector<int32_t> dl(D.nv + 1, 0);
    std::vector<uint32_t> reason(D.nv + 1, R_INPUT);
    for (uint32_t v = 0; v < D.nv; v++) {
        if (partial[v] == 0) continue;
        uint32_t code = partial[v] > 0 ? V_T : V_F;
        asg[v >> 3] |= code << ((v & 7u) * 4u);
        trail.push_back(v | (code == V_F ? TRAIL_F : 0u));
        dl[v] = 1;
    }
    cudaStream_t st = p->stream;
    cudaError_t e = cudaMemcpyAsync(p->D.asg, asg.data(), asg.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->D.dl, dl.data(), (size_t)D.nv * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->D.reason, reason.data(), (size_t)D.nv * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !trail.empty())
        e = cudaMemcpyAsync(p->D.trail, trail.data(), trail.size() * 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "upload partial");
    int rc = reset_state(p, MODE_PROPAGATE, 0, 0, nullptr, p->d_result, (uint32_t)trail.size());
    if (rc != ASP_OK) return rc;
    long long res[4] = {0, 0, 0, 0};
    if (p->empty_nogood) {
        res[3] = 1;
    } else {
        e = launch_solve(p->D, p->grid, p->block, p->smem, st);
        if (e != cudaSuccess) return cuda_fail(e, "launch");
        rc = finish(p, res);
        if (rc != ASP_OK) return rc;
    }
    e = cudaMemcpy(asg.data(), p->D.asg, (size_t)D.asg_words * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "download closure");
    for (uint32_t v = 0; v < D.nv; v++) {
        uint32_t c = (asg[v >> 3] >> ((v & 7u) * 4u)) & 3u;
        closure[v] = c == V_T ? 1 : c == V_F ? -1 : c == 3u ? 2 : 0;
    }
    if (conflict) *conflict = (int32_t)res[3];
    if (res[2] != 0) return fail(ASP_E_DEVICE, "device-side error");
    return ASP_OK;
}

int asp_sweep(asp_prog *p, int32_t passes)
{
    if (!p || passes < 1) return fail(ASP_E_ARG, "bad argument");
    Acc a;
    a.ckey = NO_KEY; a.cslot[0] = a.cslot[1] = a.cslot[2] = NO_KEY;
    a.dkey = 0; a.nclaim = 0; a.flag = 0; a.minU = 0xFFFFFFFFu; a.nlits = 0; a.checks = 0; a.visits = 0;
    a.tbusy = 0; a.tsweep = 0; a.tlong = 0; a.tbuck = 0;
    cudaError_t e = cudaMemcpyAsync(p->d_sweep_acc, &a, sizeof(a), cudaMemcpyHostToDevice, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sweep reset");
    e = launch_sweep(p->D, p->d_sweep_acc, p->grid, p->block, p->smem, p->stream, (uint32_t)passes);
    if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
    return ASP_OK;
}

int asp_debug_state(asp_prog *p, int32_t *trail, int64_t *n_trail, int32_t *level,
                    uint32_t *reason, uint64_t *deps, int32_t deps_words)
{
    if (!p) return fail(ASP_E_ARG, "bad argument");
    cudaError_t e = p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "sync");
    const Dev &D = p->D;
    DevStats s;
    e = cudaMemcpy(&s, D.stats, sizeof(s), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "state");
    int64_t nt = std::min<int64_t>((int64_t)s.pad, (int64_t)D.nv);
    if (n_trail) *n_trail = nt;
    if (trail && nt > 0) {
        e = cudaMemcpy(trail, D.trail, (size_t)nt * 4, cudaMemcpyDeviceToHost);
        for (int64_t i = 0; i < nt; i++) trail[i] = (int32_t)((uint32_t)trail[i] & TRAIL_VAR);
    }
    if (e == cudaSuccess && level) e = cudaMemcpy(level, D.dl, (size_t)D.nv * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && reason) e = cudaMemcpy(reason, D.reason, (size_t)D.nv * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && deps && deps_words > 0) {
        int32_t w = std::min<int32_t>(deps_words, (int32_t)D.WW);
        e = cudaMemcpy2D(deps, (size_t)deps_words * 8, D.deps, (size_t)D.WW * 8, (size_t)w * 8, D.nv,
                         cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return cuda_fail(e, "state");
    return ASP_OK;
}

int asp_debug_last_conflict(asp_prog *p, int64_t *info, int32_t *trail, int64_t trail_cap)
{
    if (!p || !info) return fail(ASP_E_ARG, "bad argument");
    cudaError_t e = p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "sync");
    DevStats s;
    e = cudaMemcpy(&s, p->D.stats, sizeof(s), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "state");
    info[0] = (int64_t)s.dbg_conf;
    info[1] = (int64_t)s.dbg_tend;
    info[2] = (int64_t)s.dbg_lfill;
    info[3] = (int64_t)s.dbg_len;
    info[4] = (int64_t)s.dbg_target;
    info[5] = (int64_t)s.dbg_level;
    const int64_t nt = std::min<int64_t>(std::min<int64_t>((int64_t)s.dbg_tend, (int64_t)p->D.nv), trail_cap);
    if (trail && nt > 0) {
        e = cudaMemcpy(trail, p->D.trail, (size_t)nt * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "state");
        for (int64_t i = 0; i < nt; i++) {
            const uint32_t t = (uint32_t)trail[i];
            trail[i] = (int32_t)mk_lit(t & TRAIL_VAR, (t & TRAIL_F) != 0u);
        }
    }
    return ASP_OK;
}

int64_t asp_debug_nogood(asp_prog *p, uint32_t id, int32_t *lits, int64_t cap)
{
    if (!p) return fail(ASP_E_ARG, "bad argument");
    std::vector<uint32_t> buf;
    if (id & BUCKET_ID) {
        const uint32_t L = ((id >> 27) & 15u) + 1u, k = id & 0x7FFFFFFu;
        if (L < 2 || L > (uint32_t)BUCKET_MAX || k >= p->D.bk_n[L]) return fail(ASP_E_ARG, "bad nogood id");
        // literal q sits at bk_base[L] + q * bk_n[L] + k: one strided copy
        uint32_t w[BUCKET_MAX];
        cudaError_t e = cudaMemcpy2D(w, 4, p->D.lits + p->D.bk_base[L] + k, (size_t)p->D.bk_n[L] * 4, 4, L,
                                     cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "nogood");
        for (uint32_t q = 0; q < L && (int64_t)q < cap; q++) lits[q] = (int32_t)w[q];
        return L;
    }
    if (id >= p->D.lits_cap) return fail(ASP_E_ARG, "bad argument");
    const uint32_t step = 256;
    const uint64_t alloc_words = (uint64_t)p->D.lits_cap + 128;
    for (uint64_t off = id; off < alloc_words; off += step) {
        uint32_t tmp[256];
        uint32_t n = (uint32_t)std::min<uint64_t>(step, alloc_words - off);
        cudaError_t e = cudaMemcpy(tmp, p->D.lits + off, (size_t)n * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "nogood");
        bool done = false;
        for (uint32_t i = 0; i < n; i++) {
            buf.push_back(tmp[i] & ~END_BIT);
            if (tmp[i] & END_BIT) { done = true; break; }
        }
        if (done) break;
    }
    for (int64_t i = 0; i < (int64_t)buf.size() && i < cap; i++) lits[i] = (int32_t)buf[i];
    return (int64_t)buf.size();
}

int64_t asp_debug_learned(asp_prog *p, uint32_t *ids, int64_t cap)
{
    if (!p || cap < 0 || (cap > 0 && !ids)) return fail(ASP_E_ARG, "bad argument");
    cudaError_t e = p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "sync");
    Ctl c[2];
    e = cudaMemcpy(c, p->D.ctl, sizeof(c), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "control");
    // the count only grows from phase to phase: the larger of the two
    // control blocks is the last one written
    const int64_t n = std::min<int64_t>(std::max(c[0].n_learned, c[1].n_learned), p->D.learned_ng_cap);
    const int64_t k = std::min(n, cap);
    if (k > 0) {
        e = cudaMemcpy(ids, p->D.learned_ids, (size_t)k * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "learned ids");
    }
    return n;
}

int asp_debug_barrier(asp_prog *p, int32_t stall_cta, int32_t wait_limit_ms)
{
    if (!p) return fail(ASP_E_ARG, "bad argument");
    if (stall_cta >= p->grid) return fail(ASP_E_ARG, "stall_cta is not a CTA of the solver grid");
    p->D.stall_cta = stall_cta < 0 ? 0xFFFFFFFFu : (uint32_t)stall_cta;
    p->D.barrier_ns = wait_limit_ms > 0 ? (unsigned long long)wait_limit_ms * 1000000ull : 20000000000ull;
    return ASP_OK;
}

int asp_debug_fail_alloc(int64_t nth)
{
    if (nth < 0) return fail(ASP_E_ARG, "bad argument");
    g_alloc_fail_in.store(nth);
    return ASP_OK;
}

int asp_build_info(int32_t *binary_version, int32_t *ptx_version)
{
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(ASP_E_NODEVICE, "no CUDA device");
    cudaFuncAttributes a;
    cudaError_t e = solve_attributes(&a);
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
    if (binary_version) *binary_version = a.binaryVersion;
    if (ptx_version) *ptx_version = a.ptxVersion;
    return ASP_OK;
}

int64_t asp_trace(asp_prog *p, float *features, int32_t *labels, int32_t *rules, int64_t cap)
{
    if (!p || cap < 0 || (cap > 0 && (!features || !labels))) return fail(ASP_E_ARG, "bad argument");
    if (!p->D.trace) return 0;
    cudaError_t e = p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "sync");
    DevStats s;
    e = cudaMemcpy(&s, p->D.stats, sizeof(s), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "trace");
    const int64_t n = std::min<int64_t>({(int64_t)s.trace_n, (int64_t)p->D.trace_cap, cap});
    std::vector<uint32_t> rec((size_t)std::max<int64_t>(n, 1) * TRACE_WORDS);
    if (n > 0) {
        e = cudaMemcpy(rec.data(), p->D.trace, (size_t)n * TRACE_WORDS * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "trace");
    }
    for (int64_t i = 0; i < n; i++) {
        std::memcpy(features + i * N_FEATURES, rec.data() + i * TRACE_WORDS, N_FEATURES * 4);
        labels[i] = rec[(size_t)i * TRACE_WORDS + 19] ? (int32_t)rec[(size_t)i * TRACE_WORDS + 18] : -1;
        if (rules) rules[i] = (int32_t)rec[(size_t)i * TRACE_WORDS + 16];
    }
    return n;
}

int asp_solve_batch(int32_t n, asp_prog *const *progs, int64_t max_models_each,
                    int32_t *statuses, int64_t *n_models, uint64_t *const *models,
                    const int64_t *models_cap)
{
    g_err.clear();
    if (n < 0 || max_models_each < 0 || (n > 0 && (!progs || !statuses || !n_models))) return fail(ASP_E_ARG, "bad argument");
    if (n == 0) return ASP_OK;
    asp_batch *b = nullptr;
    int rc = asp_batch_create(n, progs, max_models_each, models_cap, 0, &b);
    if (rc != ASP_OK) return rc;
    rc = asp_batch_run(b, statuses, n_models, models);
    std::string err = g_err;
    asp_batch_free(b);
    g_err = err;
    return rc;
}

int asp_batch_create(int32_t n, asp_prog *const *progs, int64_t max_models_each, const int64_t *models_cap,
                     int32_t config, asp_batch **out)
{
    g_err.clear();
    if (!out) return fail(ASP_E_ARG, "out is NULL");
    *out = nullptr;
    if (n <= 0 || max_models_each < 0 || !progs) return fail(ASP_E_ARG, "bad argument");
    if (config < ASP_BATCH_AUTOTUNE || config > 1) return fail(ASP_E_ARG, "unknown batch configuration");
    for (int32_t i = 0; i < n; i++) {
        if (!progs[i]) return fail(ASP_E_ARG, "null program");
        if (progs[i]->stream != progs[0]->stream) return fail(ASP_E_ARG, "programs loaded on different streams");
        if (progs[i]->device != progs[0]->device) return fail(ASP_E_ARG, "programs loaded on different devices");
        if (models_cap && models_cap[i] < 0) return fail(ASP_E_ARG, "negative model capacity");
    }
    asp_batch *b = new asp_batch;
    b->progs.assign(progs, progs + n);
    b->max_models_each = max_models_each;
    b->caps.resize(n);
    for (int32_t i = 0; i < n; i++) b->caps[i] = models_cap ? models_cap[i] : 0;
    // an explicit configuration keeps the programs' own choice of frontier;
    // the autotuner tries both where the lists exist
    bool lists = false;
    for (int32_t i = 0; i < n; i++) {
        b->units |= progs[i]->D1[0].frontier == 2u;
        lists |= progs[i]->batch_units.built;
    }
    auto bail = [&](int rc) { asp_batch_free(b); return rc; };
    // model buffers of every program
    for (int32_t i = 0; i < n; i++) {
        asp_prog *p = progs[i];
        const int64_t words = std::max<int64_t>(((int64_t)p->D.na + 63) / 64, 1);
        const int64_t rows = std::max<int64_t>(b->caps[i], 1);
        if (rows > p->d_models_rows) {
            void *q = dalloc(p, (size_t)(rows * words) * 8);
            if (!q) return bail(fail(ASP_E_OOM, "device allocation failed (models)"));
            p->d_models = (unsigned long long *)q;
            p->d_models_rows = rows;
        }
    }
    // a stream that can be captured (the legacy default stream cannot)
    b->stream = progs[0]->stream;
    if (!b->stream) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { b->stream = nullptr; return bail(cuda_fail(e, "batch stream")); }
        b->own_stream = true;
    }
    asp_prog *p0 = progs[0];
    b->scratch_bytes = sizeof(Dev) * (size_t)n + 4 * (size_t)n + 64;
    if (p0->opt.dev_alloc) b->scratch = p0->opt.dev_alloc(b->scratch_bytes, p0->opt.alloc_ctx);
    else if (cudaMalloc(&b->scratch, b->scratch_bytes) != cudaSuccess) { cudaGetLastError(); b->scratch = nullptr; }
    if (!b->scratch) return bail(fail(ASP_E_OOM, "device allocation failed (batch descriptors)"));
    // queue order: largest store first
    std::vector<uint32_t> order(n);
    for (int32_t i = 0; i < n; i++) order[i] = (uint32_t)i;
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t c) { return progs[a]->n_literals > progs[c]->n_literals; });
    int chosen = config < 0 ? 0 : config;
    if (config == ASP_BATCH_AUTOTUNE) {
        // each configuration solves the same sample (up to 256 programs spread
        // over the queue order, at most 8 conflicts and 0.5 s each) once; the
        // lower device time per program wins
        const size_t S = std::min<size_t>((size_t)n, 256);
        std::vector<uint32_t> sample(S);
        for (size_t k = 0; k < S; k++) sample[k] = order[k * (size_t)n / S];
        // schedules: the two kernel configurations, each with full sweeps
        // and (where the programs have unit lists) with the unit frontier
        double best = -1.0;
        bool best_units = false;
        for (int u = 0; u < (lists ? 2 : 1); u++) {
            b->units = u == 1;
            for (int c = 0; c < 2; c++) {
                const double t = batch_trial(b, c, sample);
                b->trial_ns[c + 2 * u] = t;
                if (t >= 0.0 && (best < 0.0 || t < best)) { best = t; chosen = c; best_units = u == 1; }
            }
        }
        if (best < 0.0) return bail(fail(ASP_E_CUDA, "no batch configuration can run"));
        b->units = best_units;
    }
    int rc = batch_prepare(b, chosen, order);
    if (rc != ASP_OK) return bail(rc);
    // capture queue reset + launch once; every asp_batch_run replays it
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e2 = batch_enqueue(b);
        e = cudaStreamEndCapture(b->stream, &b->graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) return bail(cuda_fail(e, "batch graph"));
    *out = b;
    return ASP_OK;
}

int asp_batch_run(asp_batch *b, int32_t *statuses, int64_t *n_models, uint64_t *const *models)
{
    g_err.clear();
    if (!b || !statuses || !n_models) return fail(ASP_E_ARG, "bad argument");
    const int32_t n = (int32_t)b->progs.size();
    for (int32_t i = 0; i < n; i++)
        if (b->caps[i] > 0 && (!models || !models[i])) return fail(ASP_E_ARG, "null model buffer");
    cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch solve");
    bool device_error = false, capacity = false;
    for (int32_t i = 0; i < n; i++) {
        asp_prog *p = b->progs[i];
        long long res[4];
        e = cudaMemcpy(res, p->d_result, sizeof(res), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "batch result");
        statuses[i] = (int32_t)res[0];
        n_models[i] = res[1];
        device_error |= res[2] != 0;
        const int64_t cap = b->caps[i];
        const int64_t words = ((int64_t)p->D.na + 63) / 64;
        const int64_t copy = std::min<int64_t>(res[1], cap);
        capacity |= res[1] > cap && cap > 0;
        if (copy > 0 && words > 0) {
            e = cudaMemcpy(models[i], p->d_models, (size_t)(copy * words) * 8, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(e, "batch models");
        }
    }
    if (device_error) return fail(ASP_E_DEVICE, "device-side error in some program (learned store full)");
    if (capacity) return fail(ASP_E_CAPACITY, "more answer sets than model buffer rows for some program");
    return ASP_OK;
}

int asp_batch_info(const asp_batch *b, int32_t *config, int32_t *block_threads, int32_t *grid, int32_t *frontier,
                   double *trial_ns)
{
    if (!b) return fail(ASP_E_ARG, "bad argument");
    if (config) *config = b->config;
    if (block_threads) *block_threads = batch_threads(b->config);
    if (grid) *grid = b->grid;
    if (frontier) *frontier = b->units ? ASP_FRONTIER_UNITS : ASP_FRONTIER_FULL;
    if (trial_ns)
        for (int i = 0; i < 4; i++) trial_ns[i] = b->trial_ns[i];
    return ASP_OK;
}

void asp_batch_free(asp_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->scratch) {
        asp_prog *p0 = b->progs[0];
        if (p0->opt.dev_free) p0->opt.dev_free(b->scratch, b->scratch_bytes, p0->opt.alloc_ctx);
        else cudaFree(b->scratch);
    }
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
