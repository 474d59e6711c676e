// Device-resident conflict-driven answer-set search (sm_103a).
//
// One persistent cooperative kernel runs the whole loop of Algorithm 1:
// InitialPropagation, propagate-and-check sweeps to fixpoint (Section 4.1),
// fwd-learning from decision-level dependency bitmaps (Section 4.2,
// Algorithm 4), Backjump, Decision over applicable rules (Section 2),
// CompleteAssignment, and the stability step.  Phases are separated by a
// grid barrier; the leader (CTA 0, thread 0) writes the control block for the
// next phase into the other half of a double buffer, so all CTAs read a
// stable copy while it is being updated.
//
// Sweep design.  The static nogoods sit in one bucket per exact length
// (Section 4: one kernel per length class), stored structure-of-arrays, and
// are cut into contiguous ranges, one per CTA, along groups of nogoods (an
// atom's rules and the atom's own nogood).  Each CTA keeps a 2-bit view of
// the assignment in shared memory: all atoms, plus the auxiliary variables
// of the rules its ranges refer to.  One lane classifies one nogood against
// that view.  A claim (atomicOr on the global 4-bit codes) computes the
// claimed variable's dependency bitmap at once, from its reason, and is then
// published in the CTA's own view, so chains of implications inside a CTA
// can resolve within one sweep; other CTAs see the claim after the next
// barrier.  Long and learned nogoods are classified by one warp each (ballot
// and popc over lanes), against the global codes.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "device.cuh"
#include "mlp.cuh"
#include "store.h"

namespace aspgpu {

#define FULL_MASK 0xFFFFFFFFu

// CTA barrier that counts every thread on its own (PTX barrier.sync
// without .aligned).  The aligned form counts a warp as arrived when its
// first threads get there, which let warps pass while lane 0 of another
// warp was still finishing a section it runs alone (an atomic reservation,
// a control-block copy) and read shared values before they were written.
__device__ __forceinline__ void cta_sync()
{
    asm volatile("barrier.sync 0;" ::: "memory");
}

// ------------------------------------------------------------ primitives

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const unsigned int *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier number gen (0, 1, ... in every CTA) of a launch, with a
// bounded wait: returns false (and sets the sticky error flag) if the other
// CTAs do not arrive within limit_ns (20 s unless a test shortens it), or
// if another CTA gave up.  The host zeroes the counter before each launch,
// so barrier gen is complete once it reaches (gen + 1) x CTAs; a CTA
// arrives with a release add that returns nothing (the CTA's writes,
// ordered before it by the CTA barrier, become visible with it) and waits
// with acquire loads.
__device__ __forceinline__ bool grid_sync(Barrier *b, unsigned nblocks, unsigned long long limit_ns, uint32_t gen)
{
    __shared__ int s_ok;
    cta_sync();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (nblocks > 1) {
            const unsigned long long target = ((unsigned long long)gen + 1ull) * nblocks;
            asm volatile("red.release.gpu.global.add.u64 [%0], %1;" :: "l"(&b->count), "l"(1ull) : "memory");
            unsigned long long t0 = 0;
            for (unsigned spins = 1; ld_acquire_u64(&b->count) < target; spins++) {
                if ((spins & 255u) == 0u) {
                    if (ld_acquire_u32(&b->err)) { ok = 0; break; }
                    const unsigned long long now = globaltimer_ns();
                    if (t0 == 0) t0 = now;
                    else if (now - t0 > limit_ns) {
                        atomicExch(&b->err, 1u);
                        ok = 0;
                        break;
                    }
                }
            }
            __threadfence();
        }
        s_ok = ok;
    }
    cta_sync();
    return s_ok != 0;
}

__device__ __forceinline__ uint32_t nib(uint32_t word, uint32_t v) { return (word >> ((v & 7u) * 4u)) & 0xFu; }

// effective value during a round: fresh variables (claimed this round) read
// as unassigned
__device__ __forceinline__ uint32_t eff_val(uint32_t code, uint32_t fresh_cur)
{
    return (code & fresh_cur) ? 0u : (code & 3u);
}

__device__ __forceinline__ uint32_t global_val(const Dev &D, uint32_t v, uint32_t fresh_cur)
{
    return eff_val(nib(__ldcg(D.asg + (v >> 3)), v), fresh_cur);
}

// words of a dependency bitmap that can be non-zero for a variable at level L
__device__ __forceinline__ uint32_t deps_words(const Dev &D, uint32_t L)
{
    uint32_t w = (L + 63u) >> 6;
    return w < D.WW ? w : D.WW;
}

// bit of level L (levels >= Wlevels share the overflow bit Wlevels-1)
__device__ __forceinline__ uint32_t level_bit(const Dev &D, uint32_t L)
{
    return L < D.Wlevels ? L - 1u : D.Wlevels - 1u;
}

__device__ __forceinline__ uint32_t lit_at(const Dev &D, uint32_t idx)
{
    return idx < D.lits_static ? __ldg(D.lits + idx) : __ldcg(D.lits + idx);
}

// literal q (without end flag) and length of nogood `id`
__device__ __forceinline__ uint32_t ng_lit(const Dev &D, uint32_t id, uint32_t q)
{
    if (id & BUCKET_ID) {
        const uint32_t L = ((id >> 27) & 15u) + 1u, k = id & 0x7FFFFFFu;
        return __ldg(D.lits + D.bk_base[L] + (size_t)q * D.bk_n[L] + k);
    }
    return lit_at(D, id + q) & ~END_BIT;
}

__device__ __forceinline__ uint32_t ng_len(const Dev &D, uint32_t id)
{
    if (id & BUCKET_ID) return ((id >> 27) & 15u) + 1u;
    uint32_t n = 1;
    while (!(lit_at(D, id + n - 1u) & END_BIT)) n++;
    return n;
}

// ---------------------------------------------------------------- views

// The CTA's view (0 unassigned, 1 true, 2 false; 2 bits or one byte per
// entry) of the atoms [0, na_v) and of the auxiliary variables
// [auxlo, auxlo + auxn), which follow the atoms at entry aux_base (a
// multiple of 16).
struct View {
    volatile uint32_t *w;
    uint32_t na_v, aux_base, auxlo, auxn;
    bool bytes;

    // entry of v in the view, or 0xFFFFFFFF if v is not in it
    __device__ __forceinline__ uint32_t index(uint32_t v) const
    {
        if (v < na_v) return v;
        uint32_t k = v - auxlo;
        return k < auxn ? aux_base + k : 0xFFFFFFFFu;
    }
    // variable of entry i
    __device__ __forceinline__ uint32_t var(uint32_t i) const { return i < aux_base ? i : i - aux_base + auxlo; }
    __device__ __forceinline__ uint32_t get(uint32_t i) const
    {
        if (bytes) return reinterpret_cast<volatile const uint8_t *>(w)[i];
        return (w[i >> 4] >> (2u * (i & 15u))) & 3u;
    }
    // set entry i to val; true if it was unassigned
    __device__ __forceinline__ bool put(uint32_t i, uint32_t val) const
    {
        if (bytes) {
            volatile uint8_t *b = reinterpret_cast<volatile uint8_t *>(w);
            const uint32_t old = b[i];
            b[i] = (uint8_t)val;
            return old == 0u;
        }
        uint32_t sh = 2u * (i & 15u);
        uint32_t old = atomicOr((uint32_t *)(w + (i >> 4)), val << sh);
        return ((old >> sh) & 3u) == 0u;
    }
    __device__ __forceinline__ void clear(uint32_t i) const
    {
        if (bytes) reinterpret_cast<volatile uint8_t *>(w)[i] = 0;
        else atomicAnd((uint32_t *)(w + (i >> 4)), ~(3u << (2u * (i & 15u))));
    }
};

__device__ __forceinline__ uint32_t view_val(const Dev &D, const View &V, uint32_t v, uint32_t fresh_cur)
{
    uint32_t i = V.index(v);
    if (i != 0xFFFFFFFFu) return V.get(i);
    return global_val(D, v, fresh_cur);
}

__device__ __forceinline__ bool view_set(const View &V, uint32_t v, uint32_t val)
{
    uint32_t i = V.index(v);
    return i != 0xFFFFFFFFu && V.put(i, val);
}

__device__ __forceinline__ void view_clear(const View &V, uint32_t v)
{
    uint32_t i = V.index(v);
    if (i != 0xFFFFFFFFu) V.clear(i);
}

// 2-bit effective values of the 8 variables of one global code word
__device__ __forceinline__ uint32_t pack8(uint32_t word, uint32_t fresh_cur)
{
    uint32_t m = 0;
#pragma unroll
    for (uint32_t q = 0; q < 8u; q++) m |= eff_val((word >> (4u * q)) & 0xFu, fresh_cur) << (2u * q);
    return m;
}

// effective values of the 4 variables at nibbles sh..sh+3 of code words
// (a, b), one per byte
__device__ __forceinline__ uint32_t bytes4(uint32_t a, uint32_t b, uint32_t sh, uint32_t fresh_cur)
{
    const uint32_t x = (uint32_t)((((unsigned long long)b << 32) | a) >> (4u * sh));
    uint32_t m = 0;
#pragma unroll
    for (uint32_t q = 0; q < 4u; q++) m |= eff_val((x >> (4u * q)) & 0xFu, fresh_cur) << (8u * q);
    return m;
}

// Byte view: one view word holds 4 variables (half a global code word).
__device__ __forceinline__ void view_reload_bytes(const Dev &D, const View &V, uint32_t fresh_cur)
{
    const uint32_t wa = (V.na_v + 3u) >> 2, wx = (V.auxn + 3u) >> 2;
    for (uint32_t k = threadIdx.x; k < wa; k += blockDim.x) {
        const uint32_t v0 = 4u * k;
        uint32_t m = bytes4(__ldcg(D.asg + (v0 >> 3)), 0u, v0 & 7u, fresh_cur);
        const uint32_t valid = V.na_v - v0;
        if (valid < 4u) m &= (1u << (8u * valid)) - 1u;
        V.w[k] = m;
    }
    for (uint32_t k = wa + threadIdx.x; k < V.aux_base / 4u; k += blockDim.x) V.w[k] = 0u;
    for (uint32_t k = threadIdx.x; k < wx; k += blockDim.x) {
        const uint32_t v0 = V.auxlo + 4u * k, w0 = v0 >> 3;
        const uint32_t a = __ldcg(D.asg + w0);
        const uint32_t b = w0 + 1u < D.asg_words ? __ldcg(D.asg + w0 + 1u) : 0u;
        uint32_t m = bytes4(a, b, v0 & 7u, fresh_cur);
        const uint32_t valid = V.auxn - 4u * k;
        if (valid < 4u) m &= (1u << (8u * valid)) - 1u;
        V.w[V.aux_base / 4u + k] = m;
    }
}

// Rebuild the whole view from the global codes (fresh claims read as
// unassigned); one 2-bit view word holds 16 variables = two global code
// words.
__device__ __forceinline__ void view_reload(const Dev &D, const View &V, uint32_t fresh_cur)
{
    if (V.bytes) {
        view_reload_bytes(D, V, fresh_cur);
        return;
    }
    const uint32_t wa = (V.na_v + 15u) >> 4, wx = (V.auxn + 15u) >> 4;
    for (uint32_t k = threadIdx.x; k < wa; k += blockDim.x) {
        uint32_t lo = __ldcg(D.asg + 2u * k), hi = 2u * k + 1u < D.asg_words ? __ldcg(D.asg + 2u * k + 1u) : 0u;
        uint32_t m = pack8(lo, fresh_cur) | (pack8(hi, fresh_cur) << 16);
        uint32_t valid = V.na_v - 16u * k;    // entries of this word that are atoms
        if (valid < 16u) m &= (1u << (2u * valid)) - 1u;
        V.w[k] = m;
    }
    for (uint32_t k = threadIdx.x; k < wx; k += blockDim.x) {
        // variables auxlo + 16k .. +15: spread over up to three code words
        const uint32_t v0 = V.auxlo + 16u * k;
        const uint32_t w0 = v0 >> 3, sh = v0 & 7u;
        uint32_t a = __ldcg(D.asg + w0);
        uint32_t b = w0 + 1u < D.asg_words ? __ldcg(D.asg + w0 + 1u) : 0u;
        uint32_t c = w0 + 2u < D.asg_words ? __ldcg(D.asg + w0 + 2u) : 0u;
        // 24 nibbles starting at a; take 16 from nibble sh
        unsigned long long lo64 = ((unsigned long long)b << 32) | a;
        uint32_t first8 = (uint32_t)(lo64 >> (4u * sh));
        unsigned long long hi64 = ((unsigned long long)c << 32) | b;
        uint32_t next8 = (uint32_t)(hi64 >> (4u * sh));
        uint32_t m = pack8(first8, fresh_cur) | (pack8(next8, fresh_cur) << 16);
        uint32_t valid = V.auxn - 16u * k;
        if (valid < 16u) m &= (1u << (2u * valid)) - 1u;
        V.w[V.aux_base / 16u + k] = m;
    }
}

// ---------------------------------------------------------------- claims

// Claim the complement of an unassigned literal: 0 won, 1 agreed, 2 clash.
__device__ __forceinline__ int claim_var(uint32_t *asg, uint32_t v, uint32_t valbit, uint32_t fresh_cur)
{
    uint32_t sh = (v & 7u) * 4u;
    uint32_t old = atomicOr(asg + (v >> 3), (valbit | fresh_cur) << sh);
    uint32_t ov = (old >> sh) & 3u;
    if (ov == 0u) return 0;
    if (ov & valbit) return 1;
    return 2;
}

struct SweepCtx {
    const Dev *D;
    View V;
    uint32_t fresh;        // fresh bit of the current round
    uint32_t cdl;          // level of new claims
    uint32_t tbase;        // trail index of this phase's first claim
    Acc *acc;              // this phase's accumulators
    bool do_claim;
    bool use_view;
    uint32_t dec_v;        // decision variable set in this phase (its level
                           // and bitmap are known here before they reach memory)
    uint32_t cta;          // this CTA's part of the static partition
    uint32_t gw, nw;       // warp index and warp count of the solving group
    // inside a sweep: claims are listed in shared memory and copied to the
    // trail once at the end of the sweep (one global atomic per CTA)
    bool listed = false;
    // frontier by units: the next round's dirty bitmap (null otherwise)
    uint32_t *dmark = nullptr;
    // frontier by units with chaining in the round (frontier = 3): a claim
    // queues the CTA's own units that hold its variable for a later wave of
    // the same sweep
    bool chain = false;
};

constexpr uint32_t CLAIM_BUF = 256;
// first unit of each bucket in this CTA's part of the partition (units of
// unit_groups(L) groups of 32 nogoods); entry BUCKET_MAX + 1 = all units
__shared__ uint32_t s_ubase[BUCKET_MAX + 2];
// this CTA's range [s_krange[L][0], s_krange[L][1]) of bucket L
__shared__ uint32_t s_krange[BUCKET_MAX + 1][2];
__shared__ uint32_t s_claims[CLAIM_BUF];
__shared__ unsigned int s_ncl, s_cbase;
// next bucket unit of the CTA's queue in the current sweep (solver sweeps;
// sweeps that do not claim alternate between s_unit2[0] and s_unit2[1])
__shared__ unsigned int s_unit, s_unit2[2];
// CTA 0, thread 0: time in the sweeps on long and learned nogoods and on
// the buckets
__shared__ unsigned long long s_tlearned, s_tbuckets;
// the same two parts, max over the CTA's warps in the current sweep
__shared__ unsigned long long s_wmax[2];
// frontier by units (single-program solver only): this round's queue of the
// CTA's bucket units (local unit indices) and its length
constexpr uint32_t DQ_CAP = 1024;
__shared__ uint32_t s_dq[DQ_CAP];
__shared__ unsigned int s_nq;
// frontier = 3: units already in this round's queue (local units below
// DQ_BITS), the per-wave pop counters, and the CTA's global unit range
constexpr uint32_t DQ_BITS = 4096, DQ_WAVES = 4;
__shared__ uint32_t s_dqbits[DQ_BITS / 32];
__shared__ unsigned int s_wave[DQ_WAVES];
__shared__ uint32_t s_ub[3];

// Queue local unit `local` once per round (frontier = 3); the caller keeps
// it below DQ_BITS.
__device__ __forceinline__ void dq_push_once(uint32_t local)
{
    const uint32_t bit = 1u << (local & 31u);
    if (atomicOr(&s_dqbits[local >> 5], bit) & bit) return;
    const uint32_t pos = atomicAdd(&s_nq, 1u);
    if (pos < DQ_CAP) s_dq[pos] = local;
}

// frontier = 3: after a claim of x is published in the CTA's view, queue
// the CTA's own units that hold x for the next wave of this sweep (units of
// other CTAs, and any that do not fit, are checked next round through the
// dirty bitmap).  All 32 lanes call it with the same x.
__device__ __forceinline__ void warp_push_units(const SweepCtx &X, uint32_t x)
{
    const Dev &D = *X.D;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t ub0 = s_ub[0], ub1 = s_ub[1];
    const uint32_t o0 = __ldg(D.occ_uoff + x), o1 = __ldg(D.occ_uoff + x + 1u);
    for (uint32_t o = o0 + lane; o < o1; o += 32u) {
        const uint32_t u = __ldg(D.occ_unit + o);
        if (u >= ub0 && u < ub1 && u - ub0 < DQ_BITS) dq_push_once(u - ub0);
    }
}

// The same from one lane.
__device__ __forceinline__ void lane_push_units(const SweepCtx &X, uint32_t x)
{
    const Dev &D = *X.D;
    const uint32_t ub0 = s_ub[0], ub1 = s_ub[1];
    const uint32_t o0 = __ldg(D.occ_uoff + x), o1 = __ldg(D.occ_uoff + x + 1u);
    for (uint32_t o = o0; o < o1; o++) {
        const uint32_t u = __ldg(D.occ_unit + o);
        if (u >= ub0 && u < ub1 && u - ub0 < DQ_BITS) dq_push_once(u - ub0);
    }
}

// Frontier by units: this CTA's bucket units to check in the round -- those
// whose bit is set in the round's dirty bitmap `buf` (set by the claims of
// the previous claiming phase; the bits read are cleared) and, in a decision
// phase, those holding the decision variable dec_v.  Warp 0 writes the queue
// (s_nq > DQ_CAP: it overflowed, and the CTA sweeps all its units); the
// caller synchronises the CTA before the sweep.
__device__ __forceinline__ void build_unit_queue(const Dev &D, uint32_t cta, uint32_t *buf, uint32_t dec_v)
{
    if (threadIdx.x >= 32u) return;
    const uint32_t lane = threadIdx.x;
    const uint32_t ub0 = __ldg(D.cta_ubase + cta), ub1 = __ldg(D.cta_ubase + cta + 1u);
    if (ub1 > ub0) {
        const uint32_t w_first = ub0 >> 5, w_last = (ub1 - 1u) >> 5;
        for (uint32_t w0 = w_first; w0 <= w_last; w0 += 32u) {
            const uint32_t w = w0 + lane;
            uint32_t bits = 0u;
            if (w <= w_last) {
                uint32_t own = ~0u;
                if (w == w_first) own &= ~0u << (ub0 & 31u);
                if (w == w_last && (ub1 & 31u)) own &= (1u << (ub1 & 31u)) - 1u;
                bits = __ldcg(buf + w) & own;
                if (bits) atomicAnd(buf + w, ~bits);
            }
            while (bits) {
                const uint32_t b = (uint32_t)__ffs(bits) - 1u;
                bits &= bits - 1u;
                const uint32_t local = w * 32u + b - ub0;
                if (D.frontier == 3u && local < DQ_BITS) {
                    dq_push_once(local);
                } else {
                    const uint32_t pos = atomicAdd(&s_nq, 1u);
                    if (pos < DQ_CAP) s_dq[pos] = local;
                }
            }
        }
    }
    if (dec_v != 0xFFFFFFFFu) {
        const uint32_t o0 = __ldg(D.occ_uoff + dec_v), o1 = __ldg(D.occ_uoff + dec_v + 1u);
        for (uint32_t o = o0 + lane; o < o1; o += 32u) {
            const uint32_t u = __ldg(D.occ_unit + o);
            if (u >= ub0 && u < ub1) {
                if (D.frontier == 3u && u - ub0 < DQ_BITS) {
                    dq_push_once(u - ub0);
                } else {
                    const uint32_t pos = atomicAdd(&s_nq, 1u);
                    if (pos < DQ_CAP) s_dq[pos] = u - ub0;
                }
            }
        }
    }
}

__device__ __forceinline__ void report_conflict(const SweepCtx &X, uint32_t id, uint32_t len)
{
    const unsigned long long key = ((unsigned long long)len << 32) | id;
    atomicMin(&X.acc->ckey, key);
    atomicMin(&X.acc->cslot[id % 3u], key);    // read only with several conflicts per round
}

// Record a won claim: trail slot, level, reason.
__device__ __forceinline__ void record_claim(const SweepCtx &X, uint32_t v, uint32_t valbit, uint32_t id)
{
    const Dev &D = *X.D;
    D.dl[v] = (int32_t)X.cdl;
    D.reason[v] = id;
    const uint32_t entry = v | (valbit == V_F ? TRAIL_F : 0u);
    if (X.listed) {
        const uint32_t i = atomicAdd(&s_ncl, 1u);
        if (i < CLAIM_BUF) { s_claims[i] = entry; return; }
    }
    uint32_t pos = X.tbase + atomicAdd(&X.acc->nclaim, 1u);
    if (pos < D.nv) {
        D.trail[pos] = entry;
        if (D.tpos) D.tpos[v] = pos;
    }
}

// Frontier by units: the bucket units holding variable x are checked in the
// next round; set their bits in that round's dirty bitmap.  All 32 lanes call
// it with the same x.
__device__ __forceinline__ void warp_mark_units(const SweepCtx &X, uint32_t x)
{
    if (!X.dmark) return;
    const Dev &D = *X.D;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t o0 = __ldg(D.occ_uoff + x), o1 = __ldg(D.occ_uoff + x + 1u);
    for (uint32_t o = o0 + lane; o < o1; o += 32u) {
        const uint32_t u = __ldg(D.occ_unit + o);
        atomicOr(X.dmark + (u >> 5), 1u << (u & 31u));
    }
}

// The same from one lane.
__device__ __forceinline__ void lane_mark_units(const SweepCtx &X, uint32_t x)
{
    if (!X.dmark) return;
    const Dev &D = *X.D;
    const uint32_t o0 = __ldg(D.occ_uoff + x), o1 = __ldg(D.occ_uoff + x + 1u);
    for (uint32_t o = o0; o < o1; o++) {
        const uint32_t u = __ldg(D.occ_unit + o);
        atomicOr(X.dmark + (u >> 5), 1u << (u & 31u));
    }
}

// One lane per literal u of a reason (has = false on lanes holding none):
// the warp ORs Deps[u] over lanes with level > 1 and writes Deps[x]
// (Section 4.2, mk_dl_bitmap).  All 32 lanes call it.
__device__ __forceinline__ void warp_or_deps(const SweepCtx &X, bool has, uint32_t u, uint32_t x,
                                             int writer, bool accumulate)
{
    const Dev &D = *X.D;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t L = X.cdl;
    const uint32_t nw = deps_words(D, L);
    const bool is_dec = has && u == X.dec_v;
    // a decision's bitmap is the bit of its own level: with the level, the
    // reason tells whether the bitmap words need loading at all (a learned
    // nogood of fwd-learning holds decisions only)
    int32_t Lu = !has ? 0 : is_dec ? (int32_t)L : __ldcg(D.dl + u);
    const uint32_t ru = (has && !is_dec) ? __ldcg(D.reason + u) : 0u;
    uint32_t nwu = (has && Lu > 1) ? deps_words(D, (uint32_t)Lu) : 0u;
    const bool dec = is_dec || (has && Lu > 1 && ru == R_DECISION);
    const uint32_t dbit = level_bit(D, dec ? (uint32_t)Lu : L);
    for (uint32_t w = 0; w < nw; w++) {
        unsigned long long c = w >= nwu ? 0ull
                             : dec ? (w == (dbit >> 6) ? (1ull << (dbit & 63u)) : 0ull)
                             : __ldcg(D.deps + (size_t)u * D.WW + w);
        unsigned lo = __reduce_or_sync(FULL_MASK, (unsigned)c);
        unsigned hi = __reduce_or_sync(FULL_MASK, (unsigned)(c >> 32));
        if ((int)lane == writer) {
            unsigned long long m = ((unsigned long long)hi << 32) | lo;
            unsigned long long *dst = D.deps + (size_t)x * D.WW + w;
            *dst = accumulate ? (__ldcg(dst) | m) : m;
        }
    }
}

// value of a literal's variable during the sweep (view, else global codes)
__device__ __forceinline__ uint32_t lit_val(const SweepCtx &X, uint32_t l)
{
    return X.use_view ? view_val(*X.D, X.V, l >> 1, X.fresh) : global_val(*X.D, l >> 1, X.fresh);
}

// Dependency bitmap of x from the other variables of one lane's nogood
// (var), OR over those with level > 1 (Section 4.2, mk_dl_bitmap).
template <int L>
__device__ __forceinline__ void lane_deps(const SweepCtx &X, const uint32_t (&var)[L], uint32_t x)
{
    const Dev &D = *X.D;
    const uint32_t nw = deps_words(D, X.cdl);
    const uint32_t dbit = level_bit(D, X.cdl);
    int32_t Lu[L];
#pragma unroll
    for (int q = 0; q < L; q++) {
        uint32_t u = var[q];
        Lu[q] = (u == x) ? 0 : (u == X.dec_v) ? (int32_t)X.cdl : __ldcg(D.dl + u);
    }
    for (uint32_t w = 0; w < nw; w++) {
        unsigned long long acc = 0;
#pragma unroll
        for (int q = 0; q < L; q++) {
            uint32_t u = var[q];
            if (Lu[q] > 1 && w < deps_words(D, (uint32_t)Lu[q]))
                acc |= (u == X.dec_v) ? (w == (dbit >> 6) ? (1ull << (dbit & 63u)) : 0ull)
                                      : __ldcg(D.deps + (size_t)u * D.WW + w);
        }
        D.deps[(size_t)x * D.WW + w] = acc;
    }
}

// Dependency bitmaps (Section 4.2, mk_dl_bitmap) -- and, with the frontier
// by units, the unit marks -- of every claim of a group of 32 nogoods at
// once: the claims take equal shares of the warp's lanes (32 / p2 lanes
// each, p2 the claim count rounded up to a power of two), and the lanes of a
// claim split its bitmap words and its occurrence list, so the group costs
// the two dependent loads of one claim whatever the number of claims.  All 32
// lanes call it; won: this lane's nogood claimed x; tl: its literals as view
// entries.  Returns whether the group made a claim.
template <int L, bool MARK>
__device__ __forceinline__ bool group_claims(const SweepCtx &X, bool won, const uint32_t (&tl)[L], uint32_t x)
{
    const Dev &D = *X.D;
    const unsigned m = __ballot_sync(FULL_MASK, won);
    if (!m) return false;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nc = (uint32_t)__popc(m);
    uint32_t p2 = 1u;
    while (p2 < nc) p2 <<= 1;
    const uint32_t gs = 32u / p2, c = lane / gs, sub = lane % gs;
    // the lane of the c-th claim
    unsigned mm = m;
    for (uint32_t i = 0; i < c && mm; i++) mm &= mm - 1u;
    const int src = mm ? __ffs(mm) - 1 : 0;
    uint32_t var[L];
#pragma unroll
    for (int q = 0; q < L; q++) var[q] = X.V.var(__shfl_sync(FULL_MASK, tl[q], src) >> 2);
    const uint32_t xs = __shfl_sync(FULL_MASK, x, src);
    if (c >= nc) return true;
    // unit marks: the bounds of the claim's unit list load with the levels,
    // and its first entry for this lane with the bitmap words, so the marks
    // add no dependent load to the claim
    uint32_t o0 = 0u, o1 = 0u;
    if constexpr (MARK) {
        if (X.dmark) {
            o0 = __ldg(D.occ_uoff + xs);
            o1 = __ldg(D.occ_uoff + xs + 1u);
        }
    }
    if (X.cdl > 1u) {
        const uint32_t nw = deps_words(D, X.cdl);
        const uint32_t dbit = level_bit(D, X.cdl);
        int32_t Lu[L];
        bool has_dec = false;
#pragma unroll
        for (int q = 0; q < L; q++) {
            const uint32_t u = var[q];
            has_dec |= u != xs && u == X.dec_v;
            Lu[q] = (u != xs && u != X.dec_v) ? __ldcg(D.dl + u) : 0;
        }
        uint32_t first = 0xFFFFFFFFu;
        if constexpr (MARK) {
            if (o0 + sub < o1) first = __ldg(D.occ_unit + o0 + sub);
        }
        for (uint32_t w = sub; w < nw; w += gs) {
            unsigned long long acc = (has_dec && w == (dbit >> 6)) ? (1ull << (dbit & 63u)) : 0ull;
#pragma unroll
            for (int q = 0; q < L; q++)
                if (Lu[q] > 1 && 64u * w < (uint32_t)Lu[q]) acc |= __ldcg(D.deps + (size_t)var[q] * D.WW + w);
            D.deps[(size_t)xs * D.WW + w] = acc;
        }
        if constexpr (MARK) {
            if (first != 0xFFFFFFFFu) atomicOr(X.dmark + (first >> 5), 1u << (first & 31u));
            for (uint32_t o = o0 + sub + gs; o < o1; o += gs) {
                const uint32_t u = __ldg(D.occ_unit + o);
                atomicOr(X.dmark + (u >> 5), 1u << (u & 31u));
            }
        }
        return true;
    }
    if constexpr (MARK) {
        for (uint32_t o = o0 + sub; o < o1; o += gs) {
            const uint32_t u = __ldg(D.occ_unit + o);
            atomicOr(X.dmark + (u >> 5), 1u << (u & 31u));
        }
    }
    return true;
}

// Dependency bitmap of x (claimed by one lane) computed by the whole warp,
// for a nogood of L <= BUCKET_MAX literals known at run time (var[q] for
// q < L): every lane loads the levels of the nogood's other variables and
// ORs the bitmap words w = lane, lane + 32, ... over those with level > 1
// (Section 4.2, mk_dl_bitmap).  All 32 lanes call it with the same arguments.
__device__ __forceinline__ void warp_deps_dyn(const SweepCtx &X, const uint32_t (&var)[BUCKET_MAX], uint32_t L,
                                              uint32_t x)
{
    const Dev &D = *X.D;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nw = deps_words(D, X.cdl);
    const uint32_t dbit = level_bit(D, X.cdl);
    int32_t Lu[BUCKET_MAX];
    bool has_dec = false;
#pragma unroll
    for (int q = 0; q < BUCKET_MAX; q++) {
        const uint32_t u = var[q];
        const bool in = (uint32_t)q < L;
        has_dec |= in && u != x && u == X.dec_v;
        Lu[q] = (in && u != x && u != X.dec_v) ? __ldcg(D.dl + u) : 0;
    }
    for (uint32_t w = lane; w < nw; w += 32u) {
        unsigned long long acc = (has_dec && w == (dbit >> 6)) ? (1ull << (dbit & 63u)) : 0ull;
#pragma unroll
        for (int q = 0; q < BUCKET_MAX; q++)
            if (Lu[q] > 1 && 64u * w < (uint32_t)Lu[q]) acc |= __ldcg(D.deps + (size_t)var[q] * D.WW + w);
        D.deps[(size_t)x * D.WW + w] = acc;
    }
}

// U groups of 32 nogoods of bucket L, lane = nogood k0 + t*stride + lane.
// All literals are loaded (coalesced, one row per literal position) and
// their values gathered before any is classified: a nogood is satisfied if
// some literal's complement holds, violated if all hold, unit if exactly one
// is unassigned and the rest hold (Section 2).  Repeats while a claim of
// this warp changed the view.
template <int L, int U, bool MARK>
__device__ __forceinline__ void bucket_tasks(const SweepCtx &X, uint32_t k0, uint32_t k1, uint32_t stride)
{
    const Dev &D = *X.D;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t *base = D.lits + D.bk_base[L];
    const uint32_t n = D.bk_n[L];
    uint32_t lit[U][L];
#pragma unroll
    for (int t = 0; t < U; t++) {
        const uint32_t k = k0 + (uint32_t)t * stride + lane;
#pragma unroll
        for (int q = 0; q < L; q++) lit[t][q] = k < k1 ? __ldg(base + (size_t)q * n + k) : PAD_LIT;
    }
    for (int pass = 0; pass < 2; pass++) {
        uint32_t val[U][L];
#pragma unroll
        for (int t = 0; t < U; t++)
#pragma unroll
            for (int q = 0; q < L; q++) val[t][q] = lit[t][q] == PAD_LIT ? 0u : lit_val(X, lit[t][q]);
        bool pub = false;
#pragma unroll
        for (int t = 0; t < U; t++) {
            const uint32_t k = k0 + (uint32_t)t * stride + lane;
            if (k >= k1) continue;
            bool sat = false;
            uint32_t n_un = 0, ul = 0;
#pragma unroll
            for (int q = 0; q < L; q++) {
                uint32_t v = val[t][q];
                sat |= v == ((lit[t][q] & 1u) ? V_T : V_F);
                if (v == 0u) { n_un++; ul = lit[t][q]; }
            }
            if (sat || n_un > 1u) continue;
            const uint32_t id = bucket_nogood_id((uint32_t)L, k);
            if (n_un == 0u) { report_conflict(X, id, (uint32_t)L); continue; }
            if (!X.do_claim) { atomicAdd(&X.acc->flag, 1u); continue; }
            const uint32_t x = ul >> 1, valbit = (ul & 1u) ? V_T : V_F;
            const int r = claim_var(D.asg, x, valbit, X.fresh);
            if (r == 2) { report_conflict(X, id, (uint32_t)L); continue; }
            if (r != 0) continue;
            record_claim(X, x, valbit, id);
            if constexpr (MARK) lane_mark_units(X, x);
            if (X.cdl > 1u) {
                uint32_t var[L];
#pragma unroll
                for (int q = 0; q < L; q++) var[q] = lit[t][q] >> 1;
                lane_deps<L>(X, var, x);
            }
            if (X.use_view) {
                __threadfence_block();
                pub |= view_set(X.V, x, valbit);
            }
        }
        if (!X.use_view || !X.do_claim || !__any_sync(FULL_MASK, pub)) break;
    }
}

// Contribution of one translated literal (entry << 2 | xmask) to its
// nogood's count: t = value ^ xmask is 1 if the literal holds, 2 if its
// complement holds, 0 or 3 if unassigned; the byte of 0x01100001 at t is
// 0, 16 or 1.  Over at most 15 literals the low byte of the sum is
// >= 16: satisfied; 0: violated; 1: unit; 2..15: two or more unassigned.
template <bool BYTES>
__device__ __forceinline__ uint32_t tlit_val(const View &V, uint32_t tl)
{
    const uint32_t i = tl >> 2;
    if (BYTES) return reinterpret_cast<volatile const uint8_t *>(V.w)[i];
    return V.w[i >> 4] >> (2u * (i & 15u));
}
template <bool BYTES>
__device__ __forceinline__ uint32_t tlit_count(const View &V, uint32_t tl)
{
    return __byte_perm(0x01100001u, 0u, (tlit_val<BYTES>(V, tl) ^ tl) & 3u);
}

// a if p, else b, as a predicated select (the group loop below picks a
// row of its register arrays with these, which keeps the arrays in
// registers)
__device__ __forceinline__ uint32_t sel_if(bool p, uint32_t a, uint32_t b)
{
    uint32_t r;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\tselp.b32 %0, %1, %2, q;\n\t}"
        : "=r"(r) : "r"(a), "r"(b), "r"((uint32_t)p));
    return r;
}

// The literals of one lane's nogood of a length-L bucket, as view entries.
template <int L>
struct Row { uint32_t q[L]; };

// The claim path of one group of 32 nogoods of bucket L, taken when the
// count found some lane's nogood unit or violated (cand): that lane
// classifies it again from the current view (a claim of this CTA may have
// changed it since the count), reports a violation, or claims the variable
// of its one unassigned literal; then the group's claims get their
// dependency bitmaps (and, with the frontier by units, their unit marks),
// and are published in the view.  All 32 lanes call it.  Returns whether
// this lane claimed.
template <int L, bool BYTES, bool MARK>
__device__ __forceinline__ bool group_claim_path(const SweepCtx &X, const Row<L> &r, uint32_t k, bool cand)
{
    const Dev &D = *X.D;
    bool won = false;
    uint32_t e = 0, x = 0, valbit = 0;
    if (cand) {
        const uint32_t id = bucket_nogood_id((uint32_t)L, k);
        bool sat = false;
        uint32_t n_un = 0, ul = 0;
#pragma unroll
        for (int q = 0; q < L; q++) {
            const uint32_t tv = (tlit_val<BYTES>(X.V, r.q[q]) ^ r.q[q]) & 3u;
            sat |= tv == 2u;
            if (tv == 0u || tv == 3u) { n_un++; ul = r.q[q]; }
        }
        if (!sat && n_un == 0u) {
            report_conflict(X, id, (uint32_t)L);
        } else if (!sat && n_un == 1u) {
            if (!X.do_claim) {
                atomicAdd(&X.acc->flag, 1u);
            } else {
                e = ul >> 2;
                x = X.V.var(e);
                valbit = (ul & 1u) ? V_T : V_F;
                const int rc = claim_var(D.asg, x, valbit, X.fresh);
                if (rc == 2) report_conflict(X, id, (uint32_t)L);
                else if (rc == 0) { record_claim(X, x, valbit, id); won = true; }
            }
        }
    }
    if (L > 8 && won && (MARK || X.cdl > 1u)) {
        // long buckets (few claims): the claiming lane alone
        if constexpr (MARK) lane_mark_units(X, x);
        if (X.cdl > 1u) {
            uint32_t var[L];
#pragma unroll
            for (int q = 0; q < L; q++) var[q] = X.V.var(r.q[q] >> 2);
            lane_deps<L>(X, var, x);
        }
    }
    if (L <= 8 && (X.cdl > 1u || (MARK && X.dmark))) {
        // bitmaps (and unit marks) of this group's claims, all at once
        if (group_claims<L, MARK>(X, won, r.q, x)) {
            __threadfence_block();
            __syncwarp();
        }
    }
    if (won) {
        __threadfence_block();
        X.V.put(e, valbit);
    }
    if constexpr (MARK) {
        if (X.chain) {
            // frontier = 3: the CTA's units that hold the claims, for the
            // next wave (after the claims are in the view)
            if (L > 8) {
                if (won) lane_push_units(X, x);
            } else {
                unsigned m = __ballot_sync(FULL_MASK, won);
                while (m) {
                    const int src = __ffs(m) - 1;
                    m &= m - 1u;
                    warp_push_units(X, __shfl_sync(FULL_MASK, x, src));
                }
            }
        }
    }
    return won;
}

// bucket_tasks over the translated copy of the store (view modes PACKED
// and BYTES): every literal is in the view, one shared-memory load and
// three integer operations classify it.  Lanes past the end of the range
// load the range's last nogood and drop the result.
template <int L, int U, bool BYTES, bool MARK>
__device__ __forceinline__ void bucket_tasks_view(const SweepCtx &X, uint32_t k0, uint32_t k1)
{
    const Dev &D = *X.D;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t *base = D.vlits + D.bk_base[L];
    const uint32_t n = D.bk_n[L];
    uint32_t lit[U][L];
#pragma unroll
    for (int t = 0; t < U; t++) {
        const uint32_t k = min(k0 + (uint32_t)t * 32u + lane, k1 - 1u);
#pragma unroll
        for (int q = 0; q < L; q++) lit[t][q] = __ldg(base + (size_t)q * n + k);
    }
    for (int pass = 0; pass < 2; pass++) {
        uint32_t cnt[U];
#pragma unroll
        for (int t = 0; t < U; t++) {
            cnt[t] = 0u;
#pragma unroll
            for (int q = 0; q < L; q++) cnt[t] += tlit_count<BYTES>(X.V, lit[t][q]);
        }
        // the groups with a nogood that is violated or unit by the count go
        // through the claim path, one at a time; the path is written out
        // once (the group's row is selected into registers), not once per
        // group, so the loops above stay small enough to stay in the
        // instruction cache from one round to the next
        unsigned cm = 0u;
#pragma unroll
        for (int t = 0; t < U; t++) {
            const uint32_t k = k0 + (uint32_t)t * 32u + lane;
            if (__any_sync(FULL_MASK, k < k1 && (cnt[t] & 0xFFu) <= 1u)) cm |= 1u << t;
        }
        bool pub = false;
        while (cm) {
            const int t = __ffs(cm) - 1;
            cm &= cm - 1u;
            Row<L> r;
            uint32_t c = cnt[0];
#pragma unroll
            for (int q = 0; q < L; q++) r.q[q] = lit[0][q];
#pragma unroll
            for (int tt = 1; tt < U; tt++) {
                c = sel_if(t == tt, cnt[tt], c);
#pragma unroll
                for (int q = 0; q < L; q++) r.q[q] = sel_if(t == tt, lit[tt][q], r.q[q]);
            }
            const uint32_t k = k0 + (uint32_t)t * 32u + lane;
            pub |= group_claim_path<L, BYTES, MARK>(X, r, k, k < k1 && (c & 0xFFu) <= 1u);
        }
        if (!X.do_claim || !__any_sync(FULL_MASK, pub)) break;
    }
}


template <bool BYTES, bool MARK>
__device__ __forceinline__ void run_unit_view(const SweepCtx &X, uint32_t L, uint32_t k0, uint32_t k1)
{
    switch (L) {
    case 2: bucket_tasks_view<2, unit_groups(2), BYTES, MARK>(X, k0, k1); break;
    case 3: bucket_tasks_view<3, unit_groups(3), BYTES, MARK>(X, k0, k1); break;
    case 4: bucket_tasks_view<4, unit_groups(4), BYTES, MARK>(X, k0, k1); break;
    case 5: bucket_tasks_view<5, unit_groups(5), BYTES, MARK>(X, k0, k1); break;
    case 6: bucket_tasks_view<6, unit_groups(6), BYTES, MARK>(X, k0, k1); break;
    case 7: bucket_tasks_view<7, unit_groups(7), BYTES, MARK>(X, k0, k1); break;
    case 8: bucket_tasks_view<8, unit_groups(8), BYTES, MARK>(X, k0, k1); break;
    case 9: bucket_tasks_view<9, unit_groups(9), BYTES, MARK>(X, k0, k1); break;
    case 10: bucket_tasks_view<10, unit_groups(10), BYTES, MARK>(X, k0, k1); break;
    case 11: bucket_tasks_view<11, unit_groups(11), BYTES, MARK>(X, k0, k1); break;
    case 12: bucket_tasks_view<12, unit_groups(12), BYTES, MARK>(X, k0, k1); break;
    case 13: bucket_tasks_view<13, unit_groups(13), BYTES, MARK>(X, k0, k1); break;
    case 14: bucket_tasks_view<14, unit_groups(14), BYTES, MARK>(X, k0, k1); break;
    default: bucket_tasks_view<15, unit_groups(15), BYTES, MARK>(X, k0, k1); break;
    }
}

template <bool MARK>
__device__ __forceinline__ void run_unit(const SweepCtx &X, uint32_t L, uint32_t k0, uint32_t k1)
{
    switch (L) {
    case 2: bucket_tasks<2, unit_groups(2), MARK>(X, k0, k1, 32u); break;
    case 3: bucket_tasks<3, unit_groups(3), MARK>(X, k0, k1, 32u); break;
    case 4: bucket_tasks<4, unit_groups(4), MARK>(X, k0, k1, 32u); break;
    case 5: bucket_tasks<5, unit_groups(5), MARK>(X, k0, k1, 32u); break;
    case 6: bucket_tasks<6, unit_groups(6), MARK>(X, k0, k1, 32u); break;
    case 7: bucket_tasks<7, unit_groups(7), MARK>(X, k0, k1, 32u); break;
    case 8: bucket_tasks<8, unit_groups(8), MARK>(X, k0, k1, 32u); break;
    case 9: bucket_tasks<9, unit_groups(9), MARK>(X, k0, k1, 32u); break;
    case 10: bucket_tasks<10, unit_groups(10), MARK>(X, k0, k1, 32u); break;
    case 11: bucket_tasks<11, unit_groups(11), MARK>(X, k0, k1, 32u); break;
    case 12: bucket_tasks<12, unit_groups(12), MARK>(X, k0, k1, 32u); break;
    case 13: bucket_tasks<13, unit_groups(13), MARK>(X, k0, k1, 32u); break;
    case 14: bucket_tasks<14, unit_groups(14), MARK>(X, k0, k1, 32u); break;
    default: bucket_tasks<15, unit_groups(15), MARK>(X, k0, k1, 32u); break;
    }
}

// A nogood of any length, one warp, lanes over literals (ballot/popc),
// stopping once it is satisfied or has two unassigned literals; literals are
// checked against the global codes, 128 at a time (four loads and their
// gathers in flight before the first ballot).
// Watched literals (Algorithm 2, which uses them for long learned nogoods
// as well): *wslot holds two positions of the nogood.  If neither watched
// literal holds -- one's complement is assigned, or both are unassigned --
// the nogood is neither unit nor violated, and two checks settle it;
// otherwise the scan runs and moves the watches to literals that do not
// hold (the complement found, or the first unassigned ones).  Every such
// nogood is checked every round by one warp, so the watches need no
// per-variable lists and stay valid across backjumps.  Equal positions
// (a nogood of one literal) always scan.
template <bool MARK>
__device__ __forceinline__ void classify_long(const SweepCtx &X, uint32_t id, unsigned long long &checks,
                                              uint2 *wslot)
{
    const Dev &D = *X.D;
    const uint32_t lane = threadIdx.x & 31u;
    uint2 wp = make_uint2(0u, 0u);
    if (wslot) {
        wp = __ldcg(wslot);
        if (wp.x != wp.y) {
            // lanes 0 and 1: the two watched literals
            uint32_t val = 0u, l = 0u;
            if (lane < 2u) {
                l = lit_at(D, id + (lane ? wp.y : wp.x)) & ~END_BIT;
                val = (l >> 1) < D.nv ? global_val(D, l >> 1, X.fresh) : 0u;
            }
            const bool opp = lane < 2u && val == ((l & 1u) ? V_T : V_F);
            const bool un = lane < 2u && val == 0u;
            const unsigned Bopp = __ballot_sync(FULL_MASK, opp), Bun = __ballot_sync(FULL_MASK, un);
            checks += 2u;
            if (Bopp || Bun == 3u) return;
        }
    }
    bool any_opp = false, done = false;
    uint32_t n_un = 0, ulit = 0, len = 0;
    uint32_t opos = 0, upos0 = 0, upos1 = 0;   // positions: a complement found, the first unassigned ones
    for (uint32_t off = id; !done && off < D.lits_cap; off += 128u) {
        uint32_t w[4], code[4];
#pragma unroll
        for (int q = 0; q < 4; q++) w[q] = lit_at(D, off + 32u * q + lane);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            uint32_t v = (w[q] & ~END_BIT) >> 1;
            code[q] = v < D.nv ? nib(__ldcg(D.asg + (v >> 3)), v) : 0u;
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (done) break;
            const uint32_t pos0 = off - id + 32u * (uint32_t)q;
            unsigned Bend = __ballot_sync(FULL_MASK, (w[q] & END_BIT) != 0u);
            unsigned valid = Bend ? ((2u << (__ffs(Bend) - 1)) - 1u) : FULL_MASK;
            uint32_t l = w[q] & ~END_BIT;
            bool mine = ((valid >> lane) & 1u) && (l >> 1) < D.nv;
            uint32_t val = mine ? eff_val(code[q], X.fresh) : 0u;
            bool opp = mine && val == ((l & 1u) ? V_T : V_F);
            bool un = mine && val == 0u;
            unsigned Bopp = __ballot_sync(FULL_MASK, opp);
            unsigned Bun = __ballot_sync(FULL_MASK, un);
            uint32_t first_un = __shfl_sync(FULL_MASK, l, Bun ? __ffs(Bun) - 1 : 0);
            if (Bun && n_un == 0) ulit = first_un;
            if (Bun) {
                const uint32_t b0 = (uint32_t)__ffs(Bun) - 1u;
                const unsigned rest = Bun & (Bun - 1u);
                if (n_un == 0) {
                    upos0 = pos0 + b0;
                    if (rest) upos1 = pos0 + (uint32_t)__ffs(rest) - 1u;
                } else if (n_un == 1) {
                    upos1 = pos0 + b0;
                }
            }
            if (Bopp) opos = pos0 + (uint32_t)__ffs(Bopp) - 1u;
            n_un += (uint32_t)__popc(Bun);
            len += (uint32_t)__popc(valid);
            checks += (uint32_t)__popc(valid);
            if (Bopp) { any_opp = true; done = true; }
            else if (Bend || n_un > 1) done = true;
        }
    }
    if (wslot && lane == 0 && (any_opp || n_un > 0)) {
        // the watches move to literals that do not hold
        uint2 nw;
        if (any_opp) nw = make_uint2(opos, n_un ? upos0 : (wp.x != opos ? wp.x : wp.y));
        else if (n_un > 1) nw = make_uint2(upos0, upos1);
        else nw = make_uint2(upos0, wp.x != upos0 ? wp.x : wp.y);
        if (nw.x != nw.y) *wslot = nw;
    }
    if (any_opp) return;
    int won = 0;
    if (lane == 0) {
        if (n_un == 0) {
            report_conflict(X, id, len);
        } else if (n_un == 1) {
            if (!X.do_claim) {
                atomicAdd(&X.acc->flag, 1u);
            } else {
                uint32_t v = ulit >> 1, valbit = (ulit & 1u) ? V_T : V_F;
                int r = claim_var(D.asg, v, valbit, X.fresh);
                if (r == 0) { record_claim(X, v, valbit, id); won = 1; }
                else if (r == 2) report_conflict(X, id, len);
            }
        }
    }
    won = __shfl_sync(FULL_MASK, won, 0);
    if (!won) return;
    const uint32_t x = ulit >> 1;
    if constexpr (MARK) warp_mark_units(X, x);
    if (X.cdl > 1u) {
        __threadfence_block();
        bool first = true;
        for (uint32_t off = id; off < D.lits_cap; off += 32u) {
            uint32_t w2 = lit_at(D, off + lane);
            unsigned Bend = __ballot_sync(FULL_MASK, (w2 & END_BIT) != 0u);
            unsigned valid = Bend ? ((2u << (__ffs(Bend) - 1)) - 1u) : FULL_MASK;
            uint32_t u2 = (w2 & ~END_BIT) >> 1;
            bool has = ((valid >> lane) & 1u) && u2 != x && u2 < D.nv;
            warp_or_deps(X, has, u2, x, 0, !first);
            first = false;
            if (Bend) break;
        }
    }
    if (lane == 0 && X.use_view) {
        __threadfence_block();
        view_set(X.V, x, (ulit & 1u) ? V_T : V_F);
    }
    if constexpr (MARK) {
        if (X.chain) {
            __syncwarp();
            warp_push_units(X, x);
        }
    }
}

// Frontier round: only the bucket nogoods that contain a variable of the
// trail entries [fr0, fr1) (the previous round's assignments), or this
// phase's decision variable X.dec_v when there is one, can have become unit
// or violated since the last round; every other bucket nogood is as the
// last sweep left it.  One warp per variable (round-robin over CTAs first),
// one lane per nogood of its occurrence list, classified against the global
// codes (this round's claims read as unassigned; the decision variable,
// whose code the leader may still be writing, as true).
__device__ __forceinline__ void frontier_round(const SweepCtx &X, uint32_t fr0, uint32_t fr1, unsigned long long &checks)
{
    const Dev &D = *X.D;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t wpc = blockDim.x >> 5, slot = (X.gw % wpc) * (X.nw / wpc) + X.gw / wpc;
    const bool dec = X.dec_v != 0xFFFFFFFFu;
    const uint32_t count = dec ? 1u : fr1 - fr0;
    for (uint32_t i = slot; i < count; i += X.nw) {
        const uint32_t v = dec ? X.dec_v : __ldcg(D.trail + fr0 + i) & TRAIL_VAR;
        if (v >= D.nv) continue;
        const uint32_t o0 = __ldg(D.occ_off + v), o1 = __ldg(D.occ_off + v + 1u);
        for (uint32_t ob = o0; ob < o1; ob += 32u) {
            const uint32_t o = ob + lane;
            const bool has = o < o1;
            const uint32_t id = has ? __ldg(D.occ + o) : 0u;
            const uint32_t L = has ? ((id >> 27) & 15u) + 1u : 0u, k = id & 0x7FFFFFFu;
            const uint32_t *base = has ? D.lits + D.bk_base[L] + k : D.lits;
            const uint32_t n = has ? D.bk_n[L] : 0u;
            uint32_t lit[BUCKET_MAX];
#pragma unroll
            for (int q = 0; q < BUCKET_MAX; q++) lit[q] = (uint32_t)q < L ? __ldg(base + (size_t)q * n) : 0u;
            bool sat = false;
            uint32_t n_un = 0, ul = 0;
#pragma unroll
            for (int q = 0; q < BUCKET_MAX; q++) {
                if ((uint32_t)q >= L) continue;
                const uint32_t u = lit[q] >> 1;
                const uint32_t val = u == X.dec_v ? V_T : global_val(D, u, X.fresh);
                sat |= val == ((lit[q] & 1u) ? V_T : V_F);
                if (val == 0u) { n_un++; ul = lit[q]; }
            }
            checks += L;
            bool won = false;
            uint32_t x = 0, valbit = 0;
            if (has && !sat && n_un == 0u) {
                report_conflict(X, id, L);
            } else if (has && !sat && n_un == 1u) {
                if (!X.do_claim) {
                    atomicAdd(&X.acc->flag, 1u);
                } else {
                    x = ul >> 1;
                    valbit = (ul & 1u) ? V_T : V_F;
                    const int r = claim_var(D.asg, x, valbit, X.fresh);
                    if (r == 2) report_conflict(X, id, L);
                    else if (r == 0) { record_claim(X, x, valbit, id); won = true; }
                }
            }
            if (X.cdl > 1u) {
                unsigned m = __ballot_sync(FULL_MASK, won);
                if (m) {
                    while (m) {
                        const int src = __ffs(m) - 1;
                        m &= m - 1u;
                        uint32_t var[BUCKET_MAX];
#pragma unroll
                        for (int q = 0; q < BUCKET_MAX; q++) var[q] = __shfl_sync(FULL_MASK, lit[q], src) >> 1;
                        warp_deps_dyn(X, var, __shfl_sync(FULL_MASK, L, src), __shfl_sync(FULL_MASK, x, src));
                    }
                    __threadfence_block();
                    __syncwarp();
                }
            }
            if (won && X.use_view) {
                __threadfence_block();
                view_set(X.V, x, valbit);
            }
        }
    }
}

// The CTA's unit table (s_ubase) from the static partition, once per
// launch; callers synchronise the CTA before the first sweep.
__device__ __forceinline__ void unit_table(const Dev &D, uint32_t cta)
{
    if (threadIdx.x != 0) return;
    s_unit = 0u;
    s_ncl = 0u;
    s_nq = 0u;
    s_unit2[0] = 0u;
    s_unit2[1] = 0u;
    const uint32_t G1 = D.G + 1u;
    uint32_t acc = 0;
    for (uint32_t L = 2; L <= (uint32_t)BUCKET_MAX; L++) {
        s_ubase[L] = acc;
        s_krange[L][0] = __ldg(D.cta_boff + L * G1 + cta);
        s_krange[L][1] = __ldg(D.cta_boff + L * G1 + cta + 1u);
        const uint32_t n = s_krange[L][1] - s_krange[L][0];
        const uint32_t groups = (n + 31u) >> 5, per = unit_groups(L);
        acc += (groups + per - 1u) / per;
    }
    s_ubase[BUCKET_MAX + 1] = acc;
}

// Propagate-and-check over this CTA's ranges of every bucket (full), or
// over the frontier -- the nogoods of the previous round's assignments
// (frontier = 1) or the dirty bucket units (frontier = 2), taken from the
// CTA's queue (DQ = 1, the single-program solver) or straight from the
// round's dirty bitmap, one 32-unit word per warp (DQ = 2, one program per
// CTA: every word belongs to the CTA) -- then (grid-wide) the static long
// nogoods and the learned nogoods.  dbuf: the round's dirty bitmap (DQ = 2).
template <int DQ>
__device__ __forceinline__ void sweep(const SweepCtx &X0, uint32_t n_learned, bool full = true,
                                      uint32_t fr0 = 0u, uint32_t fr1 = 0u, uint32_t pass = 0u,
                                      uint32_t *dbuf = nullptr)
{
    SweepCtx X = X0;
    // Listed claims take their trail slots at the end of the sweep, after
    // any claim that overflowed the list; a claim can rest on an earlier
    // claim of its own CTA (published in the view), so listing breaks the
    // trail's dependency order once the list overflows.  Resolution
    // learning walks the trail backwards and needs that order: there every
    // claim takes its slot when it is made.
    X.listed = X0.do_claim && !X0.D->learning;
    const Dev &D = *X.D;
    const uint32_t lane = threadIdx.x & 31u;
    const bool timer = X.cta == 0 && threadIdx.x == 0 && X.do_claim;
    const bool wtimer = lane == 0 && X.do_claim;
    const unsigned long long t0 = wtimer ? globaltimer_ns() : 0ull;
    // Units of work (one bucket, unit_groups(L) consecutive groups of 32
    // nogoods) are taken from a per-CTA counter, bucket after bucket, so
    // every warp runs about the same number of load-gather-classify chains
    // whatever the mix of lengths.
    // The counters start at 0: reset at launch (unit_table) and, in the
    // solver, at the end of every sweep once no warp reads them any more.
    // Sweeps that do not claim (the sweep timed alone, `pass` = its index
    // in the launch) use two counters: after one barrier no warp is in the
    // previous sweep, so its counter can be cleared for the next one.
    unsigned int *uctr = &s_unit;
    if (!X.do_claim) {
        cta_sync();
        if (threadIdx.x == 0) s_unit2[(pass + 1u) & 1u] = 0u;
        uctr = &s_unit2[pass & 1u];
    }
    const uint32_t *const ubase = s_ubase;     // set up once per launch (unit_table)
    uint32_t units = full ? ubase[BUCKET_MAX + 1] : 0u;
    // frontier by units: the queue (or, if it overflowed, every unit of the
    // CTA); the literals and nogoods of the units checked are counted here
    bool queued = false, count_units = false, words = false;
    if constexpr (DQ == 1) {
        if (!full && D.frontier >= 2u) {
            const uint32_t nq = s_nq;
            queued = nq <= DQ_CAP;
            units = queued ? nq : ubase[BUCKET_MAX + 1];
            count_units = true;
            X.chain = queued && D.frontier == 3u;
        }
    }
    if constexpr (DQ == 2) {
        if (!full && D.frontier >= 2u) {
            words = true;
            units = D.dirty_words;
            count_units = true;
        }
    }
    uint32_t pending = 0u, wbase = 0u;        // DQ = 2: units of the warp's word not yet run
    // frontier = 3: waves of the queue; wave w pops positions [lo, units)
    // with its own counter, and the units claims of wave w queued form wave
    // w + 1 (up to DQ_WAVES waves)
    uint32_t wave = 0u, lo = 0u;
    unsigned long long uvisits = 0;
    // Long and learned nogoods first (one warp each, round-robin over CTAs
    // first, then over the warps of a CTA); the warps that take one then
    // take fewer bucket units from the queue.
    unsigned long long checks = 0;
    const uint32_t nl = D.n_long + n_learned;
    const uint32_t wpc = blockDim.x >> 5, slot = (X.gw % wpc) * (X.nw / wpc) + X.gw / wpc;
    for (uint32_t i = slot; i < nl; i += X.nw) {
        uint32_t id = i < D.n_long ? __ldg(D.long_ids + i) : __ldcg(D.learned_ids + (i - D.n_long));
        classify_long<(DQ != 0)>(X, id, checks, D.nwatch ? D.nwatch + i : nullptr);
    }
    const unsigned long long t1 = wtimer ? globaltimer_ns() : 0ull;
    for (;;) {
        uint32_t u = 0;
        if (words && pending) {
            u = wbase + (uint32_t)__ffs(pending) - 1u;
            pending &= pending - 1u;
        } else {
            if (lane == 0) {
                if constexpr (DQ == 1) u = X.chain ? lo + atomicAdd(&s_wave[wave], 1u) : atomicAdd(uctr, 1u);
                else u = atomicAdd(uctr, 1u);
            }
            u = __shfl_sync(FULL_MASK, u, 0);
            if (u >= units) {
                if constexpr (DQ == 1) {
                    if (X.chain && wave + 1u < DQ_WAVES) {
                        // every warp of the CTA arrives here once per wave;
                        // the queue's length is read between two barriers, so
                        // no warp pushes while it is read
                        cta_sync();
                        if (threadIdx.x == 0) s_ub[2] = min(s_nq, DQ_CAP);
                        cta_sync();
                        const uint32_t nq = s_ub[2];
                        if (nq > units) {
                            lo = units;
                            units = nq;
                            wave++;
                            continue;
                        }
                    }
                }
                break;
            }
            if constexpr (DQ == 1) {
                if (queued) u = s_dq[u];
            }
            if constexpr (DQ == 2) {
                if (words) {
                    // take the word's bits and clear them in one atomic
                    uint32_t b = 0u;
                    if (lane == 0) b = atomicExch(dbuf + u, 0u);
                    pending = __shfl_sync(FULL_MASK, b, 0);
                    wbase = u * 32u;
                    continue;
                }
            }
        }
        uint32_t L = 2;
#pragma unroll
        for (uint32_t q = 3; q <= (uint32_t)BUCKET_MAX; q++)
            if (u >= ubase[q]) L = q;
        const uint32_t first = ubase[L];
        const uint32_t b0 = s_krange[L][0], b1 = s_krange[L][1];
        const uint32_t k0 = b0 + (u - first) * unit_groups(L) * 32u;
        if (D.view_mode == VIEW_BYTES) run_unit_view<true, (DQ != 0)>(X, L, k0, b1);
        else if (D.view_mode == VIEW_PACKED) run_unit_view<false, (DQ != 0)>(X, L, k0, b1);
        else run_unit<(DQ != 0)>(X, L, k0, b1);
        if (count_units && lane == 0) {
            const uint32_t n = min(b1 - k0, unit_groups(L) * 32u);
            checks += (unsigned long long)L * n;
            uvisits += n;
        }
    }
    if (!full && D.frontier == 1u) {
        unsigned long long fchecks = 0;           // per lane (classify_long's are per warp)
        frontier_round(X, fr0, fr1, fchecks);
        checks += __reduce_add_sync(FULL_MASK, (unsigned)fchecks);
    }
    if (lane == 0 && checks) atomicAdd(&X.acc->checks, checks);
    if (lane == 0 && uvisits) atomicAdd(&X.acc->visits, uvisits);
    if (wtimer) {
        const unsigned long long t2 = globaltimer_ns();
        if (timer) {
            s_tlearned += t1 - t0;
            s_tbuckets += t2 - t1;
        }
        atomicMax(&s_wmax[0], t1 - t0);
        atomicMax(&s_wmax[1], t2 - t1);
    }
    if (X.do_claim) {
        // copy the listed claims to the trail: warp 0 reserves the slots,
        // then every thread copies (no barrier under a data-dependent branch)
        cta_sync();
        const uint32_t n = min(s_ncl, CLAIM_BUF);
        if (threadIdx.x == 0) {
            s_unit = 0u; s_nq = 0u;                  // every warp has left the unit queue
            atomicMax(&X.acc->tlong, s_wmax[0]);
            atomicMax(&X.acc->tbuck, s_wmax[1]);
            s_wmax[0] = s_wmax[1] = 0ull;
        }
        if constexpr (DQ == 1) {
            if (X.chain) {
                for (uint32_t w = threadIdx.x; w < DQ_BITS / 32u; w += blockDim.x) s_dqbits[w] = 0u;
                if (threadIdx.x < DQ_WAVES) s_wave[threadIdx.x] = 0u;
            }
        }
        if (threadIdx.x < 32u) {
            uint32_t base = 0;
            if (threadIdx.x == 0 && n) base = atomicAdd(&X.acc->nclaim, n);
            base = __shfl_sync(FULL_MASK, base, 0);
            if (threadIdx.x == 0) s_cbase = X.tbase + base;
        }
        cta_sync();
        const uint32_t b = s_cbase;
        if (threadIdx.x == 0) s_ncl = 0u;           // every thread has read n
        for (uint32_t k = threadIdx.x; k < n; k += blockDim.x)
            if (b + k < D.nv) {
                const uint32_t e = s_claims[k];
                D.trail[b + k] = e;
                if (D.tpos) D.tpos[e & TRAIL_VAR] = b + k;
            }
    }
}

// bitmap word w of "every decision level 2..L" (CompleteAssignment reading)
__device__ __forceinline__ unsigned long long all_levels_word(const Dev &D, uint32_t L, uint32_t w)
{
    // exact bits 1 .. min(L, Wlevels-1)-1, plus overflow if L >= Wlevels
    uint32_t hi = (L < D.Wlevels ? L : D.Wlevels - 1u);   // exclusive upper bit
    unsigned long long m = 0;
    uint32_t lo_bit = w * 64u, hi_bit = lo_bit + 64u;
    uint32_t a = lo_bit > 1u ? lo_bit : 1u, b = hi_bit < hi ? hi_bit : hi;
    if (a < b) {
        uint32_t n = b - a;
        unsigned long long ones = n >= 64u ? ~0ull : ((1ull << n) - 1ull);
        m = ones << (a - lo_bit);
    }
    if (L >= D.Wlevels && w == D.WW - 1u) m |= 1ull << 63;
    return m;
}

// OR of the dependency bitmaps of the literals of nogood `id` other than
// variable `skip` with level > 1, word w.
__device__ __forceinline__ unsigned long long or_deps_word(const Dev &D, uint32_t id, uint32_t skip, uint32_t w)
{
    unsigned long long acc = 0;
    const uint32_t len = ng_len(D, id);
    for (uint32_t q = 0; q < len; q++) {
        uint32_t u = ng_lit(D, id, q) >> 1;
        if (u == skip) continue;
        int32_t L = __ldcg(D.dl + u);
        if (L > 1 && w < deps_words(D, (uint32_t)L)) acc |= __ldcg(D.deps + (size_t)u * D.WW + w);
    }
    return acc;
}

__device__ __forceinline__ unsigned long long shfl_max_u64(unsigned long long x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_down_sync(FULL_MASK, x, o);
        x = y > x ? y : x;
    }
    return x;
}

struct Smem {
    unsigned long long *bm;     // [WW] conflict bitmap
    unsigned long long *red;    // [32]
    uint32_t *misc;             // [16]
    const __nv_bfloat16 *mlp;   // [MLP_PARAMS] after the view (heuristic 2)
};

// The 16 features of candidate rule j (inputs of the learned heuristic):
// its 8 static features, then log1p activity, B- atoms still unassigned and
// already false, decision level / 64, log1p conflicts so far, fraction of
// variables assigned, two zeros.
__device__ __forceinline__ void cand_features(const Dev &D, uint32_t j, uint32_t cdl, uint32_t tend, float *x)
{
    const float *sf = D.rfeat + (size_t)j * 8u;
#pragma unroll
    for (int q = 0; q < 8; q++) x[q] = __ldg(sf + q);
    x[8] = log1pf((float)__ldcg(D.act + j));
    uint32_t un = 0, fa = 0;
    for (uint32_t q = __ldg(D.rneg_off + j); q < __ldg(D.rneg_off + j + 1); q++) {
        const uint32_t a = __ldg(D.rneg + q);
        const uint32_t v = (__ldcg(D.asg + (a >> 3)) >> ((a & 7u) * 4u)) & 3u;
        un += v == 0u;
        fa += v == V_F;
    }
    x[9] = (float)un;
    x[10] = (float)fa;
    x[11] = (float)cdl * (1.0f / 64.0f);
    x[12] = log1pf((float)__ldcg(&D.stats->conflicts));
    x[13] = (float)tend / (float)(D.nv ? D.nv : 1u);
    x[14] = 0.0f;
    x[15] = 0.0f;
}

// order-preserving map of a float to a positive 32-bit key
__device__ __forceinline__ uint32_t float_key(float f)
{
    uint32_t u = __float_as_uint(f);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return u ? u : 1u;
}

// Decision (Section 2 / Section 4): among rules whose head is unassigned,
// with t_r true, n_r not false and b_r unassigned (applicable), pick the
// highest score, ties to the lowest rule index.  Every key is
// (score << 32) | (0xFFFFFFFF - j): the decision phase recovers the rule j
// from the low word.
__device__ __forceinline__ void decide(const Dev &D, const Smem &S, Acc *acc, uint32_t gtid, uint32_t nthreads,
                                       uint32_t cdl, uint32_t tend)
{
    unsigned long long best = 0;
    for (uint32_t j = gtid; j < D.J; j += nthreads) {
        uint32_t h = (uint32_t)__ldg(D.rule_head + j);
        uint32_t b = D.na + 3u * j, t = b + 1u, n = b + 2u;
        uint32_t ch = nib(__ldcg(D.asg + (h >> 3)), h) & 3u;
        uint32_t cb = nib(__ldcg(D.asg + (b >> 3)), b) & 3u;
        uint32_t ct = nib(__ldcg(D.asg + (t >> 3)), t) & 3u;
        uint32_t cn = nib(__ldcg(D.asg + (n >> 3)), n) & 3u;
        if (ch == 0u && cb == 0u && ct == V_T && cn != V_F) {
            unsigned long long key;
            if (D.trace) {
                // sample about one candidate in eight per decision point
                uint32_t hsh = (j * 0x9E3779B1u) ^ (cdl * 0x85EBCA77u) ^ (tend * 0xC2B2AE3Du);
                hsh ^= hsh >> 15;
                hsh *= 0x2C1B3C6Du;
                hsh ^= hsh >> 12;
                if ((hsh & TRACE_SAMPLE_MASK) == 0u) {
                    const uint32_t r = atomicAdd(&D.stats->trace_n, 1u);
                    if (r < D.trace_cap) {
                        float x[N_FEATURES];
                        cand_features(D, j, cdl, tend, x);
                        uint32_t *rec = D.trace + (size_t)r * TRACE_WORDS;
                        for (int q = 0; q < N_FEATURES; q++) rec[q] = __float_as_uint(x[q]);
                        rec[16] = j;
                        rec[17] = cdl;
                        rec[18] = 0u;
                        rec[19] = 0u;
                    }
                }
            }
            if (D.heuristic == 3) {
                key = ((unsigned long long)float_key(__ldg(D.prior + j)) << 32) | (0xFFFFFFFFull - j);
            } else if (D.heuristic == 2) {
                // plain score (log1p occurrences of the head, feature 0) plus
                // the log of the learned probability that the rule's body
                // holds in an answer set
                float x[N_FEATURES];
                cand_features(D, j, cdl, tend, x);
                const float z = mlp_score(S.mlp, x);
                const float log_p = z >= 0.0f ? -log1pf(__expf(-z)) : z - log1pf(__expf(z));
                key = ((unsigned long long)float_key(x[0] + log_p) << 32) | (0xFFFFFFFFull - j);
            } else if (D.heuristic == 5) {
                // activity, plus the head's occurrences times a millionth of
                // the current increment (at most 4095 of them: less than one
                // bump) to order rules of equal activity; ties to the lowest
                // rule.  The low word stays ~j, which the decision phase decodes.
                const float *vact = reinterpret_cast<const float *>(D.act);
                const float a = __ldcg(vact + j);
                const float occ = (float)min(__ldg(D.score + j), 4095u);
                const float sc = a + occ * (__ldcg(vact + D.J) * 1e-6f);
                key = ((unsigned long long)float_key(sc) << 32) | (0xFFFFFFFFull - j);
            } else {
                unsigned long long sc = __ldg(D.score + j);
                if (D.heuristic == 1) sc += (unsigned long long)__ldcg(D.act + j) * 8ull;
                if (sc > 0x7FFFFFFFull) sc = 0x7FFFFFFFull;
                key = ((sc + 1ull) << 32) | (0xFFFFFFFFull - j);
            }
            best = key > best ? key : best;
        }
    }
    best = shfl_max_u64(best);
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    if (lane == 0) S.red[wid] = best;
    cta_sync();
    if (wid == 0) {
        unsigned long long x = lane < (blockDim.x >> 5) ? S.red[lane] : 0ull;
        x = shfl_max_u64(x);
        if (lane == 0 && x) atomicMax(&acc->dkey, x);
    }
}

// VSIDS-style activity (heuristic 5, not in the paper; the paper's
// Decision kernel names activity among its heuristics): every variable of a
// learned nogood bumps the rules it stands for -- b_j, t_j or n_j rule j, an
// atom the rules with it as head -- by the current increment, stored as a
// float after the J activities.  The increment grows by 1/0.95 per learned
// nogood (vsids_decay), so earlier bumps count less and less.
__device__ __forceinline__ void vsids_bump(const Dev &D, uint32_t var, float inc)
{
    float *vact = reinterpret_cast<float *>(D.act);
    if (var >= D.nv) return;
    if (var >= D.na) {
        atomicAdd(vact + (var - D.na) / 3u, inc);
        return;
    }
    for (uint32_t j = __ldg(D.head_first + var); j < __ldg(D.head_first + var + 1u); j++) atomicAdd(vact + j, inc);
}

// After each analysis (all threads of the analysing CTA): the increment
// grows by 1/0.95; above 1e20 every activity and the increment are scaled
// by 1e-20, which keeps their order.
__device__ __forceinline__ void vsids_decay(const Dev &D)
{
    __shared__ int s_rescale;
    float *vact = reinterpret_cast<float *>(D.act);
    cta_sync();
    if (threadIdx.x == 0) {
        float inc = __ldcg(vact + D.J) * (1.0f / 0.95f);
        s_rescale = inc > 1e20f;
        vact[D.J] = s_rescale ? inc * 1e-20f : inc;
    }
    cta_sync();
    if (s_rescale)
        for (uint32_t j = threadIdx.x; j < D.J; j += blockDim.x) vact[j] *= 1e-20f;
}

// fwd-learning (Algorithm 4) on CTA 0: OR the dependency bitmaps of the
// conflict's literals (plus those of the clashing variable's reason), take
// the highest level involved, and learn the nogood made of the decision
// literals of the levels in the bitmap.  Returns via S.misc:
//   misc[0] = 1 if the bitmap is empty (conflict at the root),
//   misc[1] = backjump target, misc[2] = learned length.
__device__ __forceinline__ void analyze(const Dev &D, const Smem &S, uint32_t g, uint32_t cdl, uint32_t lfill, bool find_clash)
{
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    const uint32_t nw = deps_words(D, cdl);
    for (uint32_t w = tid; w < D.WW; w += nt) S.bm[w] = 0ull;
    if (tid == 0) {
        // length of g and the clashing variable: the one with both values set
        uint32_t len = ng_len(D, g), clash = 0xFFFFFFFFu;
        for (uint32_t q = 0; q < len && find_clash; q++) {
            uint32_t u = ng_lit(D, g, q) >> 1;
            if ((nib(__ldcg(D.asg + (u >> 3)), u) & 3u) == 3u) clash = u;
        }
        S.misc[4] = len;
        S.misc[5] = clash;
    }
    cta_sync();
    const uint32_t len = S.misc[4], clash = S.misc[5];
    for (uint32_t t = tid; t < len * nw; t += nt) {
        uint32_t i = t / nw, w = t % nw;
        uint32_t u = ng_lit(D, g, i) >> 1;
        if (u == clash) continue;
        int32_t L = __ldcg(D.dl + u);
        if (L > 1 && w < deps_words(D, (uint32_t)L)) atomicOr(&S.bm[w], __ldcg(D.deps + (size_t)u * D.WW + w));
    }
    if (clash != 0xFFFFFFFFu) {
        uint32_t r = __ldcg(D.reason + clash);
        if (r == R_COMPLETE) {
            for (uint32_t w = tid; w < nw; w += nt) atomicOr(&S.bm[w], all_levels_word(D, cdl, w));
        } else if (r < R_INPUT) {
            for (uint32_t w = tid; w < nw; w += nt) atomicOr(&S.bm[w], or_deps_word(D, r, clash, w));
        } else if (r == R_DECISION) {
            int32_t L = __ldcg(D.dl + clash);
            for (uint32_t w = tid; w < nw; w += nt)
                if (L > 1 && w < deps_words(D, (uint32_t)L)) atomicOr(&S.bm[w], __ldcg(D.deps + (size_t)clash * D.WW + w));
        }
    }
    cta_sync();
    if (tid == 0) {
        bool overflow = cdl >= D.Wlevels && (S.bm[D.WW - 1] >> 63);
        int top = -1;
        for (int w = (int)nw - 1; w >= 0 && top < 0; w--) {
            unsigned long long m = S.bm[w];
            if (w == (int)D.WW - 1) m &= ~(1ull << 63);
            if (m) top = w * 64 + 63 - __clzll((long long)m);
        }
        if (!overflow && top < 0) {
            S.misc[0] = 1;
        } else {
            uint32_t h = overflow ? cdl : (uint32_t)top + 1u;
            S.misc[0] = 0;
            S.misc[1] = h - 1u;
            if (D.backjump == 1u && !overflow) {
                // the asserting level: the second-highest level of the bitmap
                // (1 if h is its only level); the learned nogood is unit there
                int second = -1;
                for (int w = top >> 6; w >= 0 && second < 0; w--) {
                    unsigned long long m = S.bm[w];
                    if (w == (int)D.WW - 1) m &= ~(1ull << 63);
                    if (w == (top >> 6)) m &= (1ull << (top & 63)) - 1ull;
                    if (m) second = w * 64 + 63 - __clzll((long long)m);
                }
                S.misc[1] = second >= 1 ? (uint32_t)second + 1u : 1u;
            }
            // write the decision literals, levels ascending
            uint32_t n = 0;
            for (uint32_t w = 0; w < nw; w++) {
                unsigned long long m = S.bm[w];
                if (w == D.WW - 1u) m &= ~(1ull << 63);
                while (m) {
                    uint32_t bit = (uint32_t)__ffsll((long long)m) - 1u;
                    m &= m - 1ull;
                    uint32_t level = w * 64u + bit + 1u;
                    if (level < 2u || level > cdl) continue;
                    uint32_t pos = lfill + n;
                    if (pos + 1u < D.lits_cap) D.lits[pos] = mk_lit(__ldcg(D.dec_var + level), false);
                    n++;
                }
            }
            if (overflow) {
                for (uint32_t level = D.Wlevels; level <= cdl; level++) {
                    uint32_t pos = lfill + n;
                    if (pos + 1u < D.lits_cap) D.lits[pos] = mk_lit(__ldcg(D.dec_var + level), false);
                    n++;
                }
            }
            if (n > 0 && lfill + n < D.lits_cap) D.lits[lfill + n - 1u] |= END_BIT;
            S.misc[2] = n;
            if (D.heuristic == 1) {
                for (uint32_t q = 0; q < n && lfill + q < D.lits_cap; q++) {
                    uint32_t bv = (D.lits[lfill + q] & ~END_BIT) >> 1;
                    if (bv >= D.na && (bv - D.na) % 3u == 0u) atomicAdd(D.act + (bv - D.na) / 3u, 1u);
                }
            }
        }
    }
    cta_sync();
    if (D.heuristic == 5 && !S.misc[0]) {
        const float inc = __ldcg(reinterpret_cast<const float *>(D.act) + D.J);
        for (uint32_t q = tid; q < S.misc[2] && lfill + q < D.lits_cap; q += nt)
            vsids_bump(D, (__ldcg(D.lits + lfill + q) & ~END_BIT) >> 1, inc);
        vsids_decay(D);
    }
}

// Register learned nogood number i (its first literal at `id`, len
// literals): the learned list, and its two watched positions (the first
// two literals; a nogood of one literal is always scanned).
__device__ __forceinline__ void add_learned(const Dev &D, uint32_t i, uint32_t id, uint32_t len)
{
    D.learned_ids[i] = id;
    if (D.nwatch) D.nwatch[D.n_long + i] = len > 1u ? make_uint2(0u, 1u) : make_uint2(0u, 0u);
}

// Record of the last conflict analysis, for consistency checks (leader).
__device__ __forceinline__ void debug_analysis(const Dev &D, uint32_t g, uint32_t tend, uint32_t lfill, uint32_t n,
                                               uint32_t target, uint32_t m)
{
    D.stats->dbg_conf = g;
    D.stats->dbg_tend = tend;
    D.stats->dbg_lfill = lfill;
    D.stats->dbg_len = n;
    D.stats->dbg_target = target;
    D.stats->dbg_level = m;
}

// ------------------------------------------------------ res-learning

// State of the resolution chain of res_analyze (uniform over its warp).
struct ResState {
    uint32_t m;             // level the nogood is resolved at
    uint32_t seg0, seg1;    // trail positions of level m
    uint32_t ep;            // stamp of this analysis
    uint32_t out0, nout;    // learned literals below level m: slots out0 ..
    uint32_t kappa;         // highest level among them (1 if none)
    bool err;
    uint32_t why, what;     // failed check (1..10) and the variable or value involved
};

__device__ __forceinline__ void res_fail(ResState &R, uint32_t why, uint32_t what)
{
    if (!R.err) { R.why = why; R.what = what; }
    R.err = true;
}

// The warp adds one literal per lane (has = false on lanes holding none) to
// the nogood being resolved.  Dropped: the variable `skip` (the one resolved
// upon), root-level literals and variables already in the nogood (stamped
// with R.ep).  A literal at level m is marked in the trail-position bitset;
// one below goes to the learned nogood.  Returns the number marked.
__device__ __forceinline__ uint32_t res_add(const Dev &D, ResState &R, bool has, uint32_t l, uint32_t skip)
{
    const uint32_t lane = threadIdx.x & 31u;
    bool cur = false, out = false;
    uint32_t L = 0, bad = 0u;
    if (has) {
        const uint32_t u = l >> 1;
        if (u >= D.nv) {
            bad = 1u;
        } else if (u != skip) {
            const int32_t Ls = __ldcg(D.dl + u);
            L = Ls > 0 ? (uint32_t)Ls : 0u;
            if (L == 0u) {
                bad = 2u;                // unassigned
            } else if (L > R.m) {
                bad = 3u;                // above the conflict level
            } else if (L > 1u && atomicExch(D.stamp + u, R.ep) != R.ep) {
                if (L == R.m) {
                    const uint32_t tp = __ldcg(D.tpos + u);
                    if (tp >= R.seg0 && tp < R.seg1) {
                        atomicOr(D.cand + (tp >> 5), 1u << (tp & 31u));
                        cur = true;
                    } else {
                        bad = 4u;        // trail position outside level m
                    }
                } else {
                    out = true;
                }
            }
        }
    }
    const unsigned bb = __ballot_sync(FULL_MASK, bad != 0u);
    if (bb) {
        const int src = __ffs(bb) - 1;
        res_fail(R, __shfl_sync(FULL_MASK, bad, src), __shfl_sync(FULL_MASK, l >> 1, src));
    }
    const unsigned bc = __ballot_sync(FULL_MASK, cur), bo = __ballot_sync(FULL_MASK, out);
    if (out) {
        const uint32_t pos = R.out0 + R.nout + (uint32_t)__popc(bo & ((1u << lane) - 1u));
        if (pos + 1u < D.lits_cap) D.lits[pos] = l;
    }
    R.nout += (uint32_t)__popc(bo);
    uint32_t k = out ? L : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) k = max(k, __shfl_xor_sync(FULL_MASK, k, o));
    R.kappa = max(R.kappa, k);
    return (uint32_t)__popc(bc);
}

// The literals of nogood `id` but variable `skip`, 32 at a time.
__device__ __forceinline__ uint32_t res_add_nogood(const Dev &D, ResState &R, uint32_t id, uint32_t skip)
{
    const uint32_t lane = threadIdx.x & 31u;
    if (id & BUCKET_ID) {
        const uint32_t len = ng_len(D, id);               // at most BUCKET_MAX < 32
        const bool has = lane < len;
        return res_add(D, R, has, has ? ng_lit(D, id, lane) : 0u, skip);
    }
    uint32_t added = 0;
    for (uint32_t base = 0;; base += 32u) {
        if (id + base + 32u > D.lits_cap + 96u) { res_fail(R, 5u, id); break; }   // no end marker
        const uint32_t w = lit_at(D, id + base + lane);
        const unsigned Bend = __ballot_sync(FULL_MASK, (w & END_BIT) != 0u);
        const unsigned valid = Bend ? ((2u << (__ffs(Bend) - 1)) - 1u) : FULL_MASK;
        added += res_add(D, R, (valid >> lane) & 1u, w & ~END_BIT, skip);
        if (Bend) break;
    }
    return added;
}

// The antecedent of a literal set by CompleteAssignment at level Le: the
// decisions of levels 2 .. Le (each true).
__device__ __forceinline__ uint32_t res_add_decisions(const Dev &D, ResState &R, uint32_t Le, uint32_t skip)
{
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t added = 0;
    for (uint32_t base = 2; base <= Le; base += 32u) {
        const uint32_t lv = base + lane;
        const bool has = lv <= Le;
        added += res_add(D, R, has, has ? mk_lit(__ldcg(D.dec_var + lv), false) : 0u, skip);
    }
    return added;
}

// Conflict analysis by resolution to the first UIP (Algorithm 3), by one
// warp of the analysing CTA.  delta starts as nogood g (every literal of it
// holds; a variable both values were claimed for in the conflict round is
// taken with its first claim) and m is its highest level.  Then, repeatedly:
// sigma = the literal of delta at level m assigned last (highest trail
// position); if no other literal of delta is at level m, sigma is the first
// UIP and delta is learned with kappa = the highest level of the others;
// else delta becomes the resolvent of delta and the reason of sigma (which
// holds the complement of sigma).  Root-level literals are left out of
// delta.  A literal set by CompleteAssignment has no reason nogood: its
// antecedent is taken to be every decision up to its level.  Writes the
// learned nogood at lfill, the first UIP first; S.misc: [0] = 1 conflict at
// the root, 2 internal inconsistency, else 0; [1] = kappa (the backjump
// target); [2] = length; [3] = m.
__device__ __forceinline__ void res_analyze(const Dev &D, const Smem &S, uint32_t g, uint32_t cdl, uint32_t tend,
                                            uint32_t lfill)
{
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) {
        S.misc[4] = ng_len(D, g);
        uint32_t e = atomicAdd(D.epoch, 1u) + 1u;
        S.misc[5] = e;
        S.misc[6] = 0u;
        S.misc[0] = 0u;
    }
    cta_sync();
    if (S.misc[5] == 0u) {
        // the stamp counter wrapped: clear every stamp, restart at 1
        for (uint32_t v = tid; v < D.nv; v += nt) D.stamp[v] = 0u;
        cta_sync();
        if (tid == 0) { *D.epoch = 1u; S.misc[5] = 1u; }
        cta_sync();
    }
    const uint32_t len = S.misc[4], ep = S.misc[5];
    for (uint32_t q = tid; q < len; q += nt) {
        const uint32_t u = ng_lit(D, g, q) >> 1;
        if (u < D.nv) atomicMax(&S.misc[6], (uint32_t)max(__ldcg(D.dl + u), 0));
    }
    cta_sync();
    const uint32_t m = S.misc[6];
    if (m <= 1u) {
        if (tid == 0) S.misc[0] = 1u;
        cta_sync();
        return;
    }
    const uint32_t seg0 = __ldcg(D.level_start + m);
    const uint32_t seg1 = m >= cdl ? tend : __ldcg(D.level_start + m + 1u);
    if (!(seg0 < seg1 && seg1 <= D.nv)) {
        if (tid == 0) { S.misc[0] = 2u; S.misc[1] = 10u; S.misc[2] = seg0; S.misc[3] = m; }
        cta_sync();
        return;
    }
    for (uint32_t w = (seg0 >> 5) + tid; w <= ((seg1 - 1u) >> 5); w += nt) D.cand[w] = 0u;
    cta_sync();
    if (tid < 32u) {
        const uint32_t lane = tid;
        ResState R{m, seg0, seg1, ep, lfill + 1u, 0u, 1u, false, 0u, 0u};
        uint32_t cnt = res_add_nogood(D, R, g, 0xFFFFFFFFu);
        __syncwarp();
        int p = (int)seg1 - 1;
        const int wlo = (int)(seg0 >> 5);
        uint32_t uip = 0xFFFFFFFFu;
        while (!R.err) {
            // the highest marked position <= p: 32 bitset words per step
            int q = -1;
            while (p >= (int)seg0) {
                const int wtop = p >> 5, w = wtop - (int)lane;
                uint32_t bits = 0;
                if (w >= wlo) {
                    bits = __ldcg(D.cand + w);
                    if (w == wtop) bits &= (2u << (p & 31)) - 1u;
                    if (w == wlo) bits &= ~0u << (seg0 & 31u);
                }
                const unsigned bal = __ballot_sync(FULL_MASK, bits != 0u);
                if (bal) {
                    const int src = __ffs(bal) - 1;
                    const uint32_t b = __shfl_sync(FULL_MASK, bits, src);
                    q = (wtop - src) * 32 + 31 - __clz(b);
                    break;
                }
                p = (wtop - 32) * 32 + 31;
            }
            if (q < 0) { res_fail(R, 6u, cnt); break; }
            if (cnt == 0u) { res_fail(R, 7u, (uint32_t)q); break; }
            const uint32_t entry = __ldcg(D.trail + q), e = entry & TRAIL_VAR;
            if (e >= D.nv) { res_fail(R, 8u, (uint32_t)q); break; }
            if (--cnt == 0u) { uip = entry; break; }     // sigma is the only literal at level m
            const uint32_t r = __ldcg(D.reason + e);
            if (r < R_INPUT) {
                cnt += res_add_nogood(D, R, r, e);
            } else if (r == R_COMPLETE) {
                cnt += res_add_decisions(D, R, (uint32_t)max(__ldcg(D.dl + e), 0), e);
            } else {
                res_fail(R, 9u, e);                       // a decision with others at its level
                break;
            }
            __syncwarp();
            p = q - 1;
        }
        const uint32_t n = 1u + R.nout;
        if (lane == 0) {
            if (R.err) {
                S.misc[0] = 2u;
                S.misc[1] = R.why;
                S.misc[2] = R.what;
                S.misc[3] = m;
            } else {
                if (lfill + 1u < D.lits_cap) D.lits[lfill] = mk_lit(uip & TRAIL_VAR, (uip & TRAIL_F) != 0u);
                if (lfill + n < D.lits_cap) D.lits[lfill + n - 1u] |= END_BIT;
                S.misc[1] = R.kappa;
                S.misc[2] = n;
                S.misc[3] = m;
            }
        }
        __syncwarp();
        if (!R.err && D.heuristic == 1) {
            for (uint32_t q = lane; q < n && lfill + q < D.lits_cap; q += 32u) {
                const uint32_t bv = (D.lits[lfill + q] & ~END_BIT) >> 1;
                if (bv >= D.na && (bv - D.na) % 3u == 0u) atomicAdd(D.act + (bv - D.na) / 3u, 1u);
            }
        }
        if (!R.err && D.heuristic == 5) {
            const float inc = __ldcg(reinterpret_cast<const float *>(D.act) + D.J);
            for (uint32_t q = lane; q < n && lfill + q < D.lits_cap; q += 32u)
                vsids_bump(D, (__ldcg(D.lits + lfill + q) & ~END_BIT) >> 1, inc);
        }
    }
    cta_sync();
    if (D.heuristic == 5 && S.misc[0] == 0u) vsids_decay(D);
}

__device__ __forceinline__ View make_view(const Dev &D, uint32_t *vbase, uint32_t cta)
{
    View V;
    V.w = vbase;
    V.na_v = D.view_atoms;
    V.aux_base = ((D.view_atoms + 15u) >> 4) << 4;
    V.bytes = D.view_mode == VIEW_BYTES;
    V.auxlo = __ldg(D.cta_auxlo + cta);
    V.auxn = __ldg(D.cta_auxn + cta);
    return V;
}

// Copy of a control struct read through L2 (other threads update it with
// plain stores and atomics).
template <class T>
__device__ __forceinline__ void ldcg_copy(T *dst, const T *src)
{
    const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
#pragma unroll
    for (uint32_t i = 0; i < sizeof(T) / 4u; i++) d[i] = __ldcg(s + i);
}

__device__ __forceinline__ Smem make_smem(const Dev &D, unsigned long long *raw)
{
    Smem S;
    S.bm = raw;
    S.red = S.bm + D.WW;
    S.misc = reinterpret_cast<uint32_t *>(S.red + 32);
    S.mlp = reinterpret_cast<const __nv_bfloat16 *>(S.misc + 16 + D.view_words);
    return S;
}

// The i-th term (i >= 1) of the Luby sequence 1 1 2 1 1 2 4 1 1 2 ...: 2^(k-1)
// if i = 2^k - 1, else the term at i - 2^(k-1) + 1 for the k with
// 2^(k-1) <= i < 2^k - 1 (Luby, Sinclair and Zuckerman's restart schedule).
__device__ __forceinline__ uint32_t luby(uint32_t i)
{
    for (;;) {
        uint32_t k = 1;
        while (k < 31u && (1u << k) - 1u < i) k++;
        if ((1u << k) - 1u == i || k == 31u) return 1u << (k - 1u);
        i = i - (1u << (k - 1u)) + 1u;
    }
}

// Phase barrier of the solving group: the whole grid (one program on every
// SM) or one CTA (one program of a batch).
template <bool BATCH>
__device__ __forceinline__ bool group_sync(const Dev &D, uint32_t gen)
{
    if (BATCH) {
        cta_sync();
        return true;
    }
    return grid_sync(D.bar, gridDim.x, D.barrier_ns, gen);
}

// Test-only failure injection: CTA D.stall_cta (thread 0) waits on a flag
// that nothing sets, so it does not reach the first phase barrier in time.
// The wait ends when another CTA has given up on that barrier (its error
// flag) or after three times the barrier's limit, whichever comes first.
__device__ __forceinline__ void injected_stall(const Dev &D)
{
    if (blockIdx.x != D.stall_cta || threadIdx.x != 0) return;
    const unsigned long long t0 = globaltimer_ns();
    while (ld_acquire_u32(&D.bar->stall) == 0u) {
        if (ld_acquire_u32(&D.bar->err)) break;
        if (globaltimer_ns() - t0 > 3ull * D.barrier_ns) break;
        __nanosleep(1000);
    }
}

// Algorithm 1 on the device.  rank/size: thread index and thread count of
// the solving group; cta: this CTA's part of the program's static partition;
// cta0/leader: the CTA and thread that run conflict analysis and write the
// next control block.  UNITS: compiled with the frontier by units (used by
// programs with frontier = 2; the kernels without it keep the sweeps free of
// the unit marks).
template <bool BATCH, bool UNITS>
__device__ __forceinline__ void solver_loop(const Dev &D, const Smem &S, const View &V, uint32_t rank,
                                            uint32_t size, bool cta0, bool leader, uint32_t cta)
{
    __shared__ Ctl sC;
    __shared__ Acc sA;
    const uint32_t gtid = rank, nthreads = size;
    // leader-only counters (shared memory, not registers of every thread),
    // written to the stats when the search ends
    __shared__ unsigned long long t_start, t_phase, n_conf, n_phases, ns_bar, ns_sw, ns_an, ns_de, ns_st;
    __shared__ unsigned long long ns_slow, ns_slow_sw, ns_slow_long, ns_slow_buck, t_cta0;
    // restarts: learned nogoods since the last restart, restarts so far
    __shared__ uint32_t r_conf, r_idx;
    if (leader) {
        t_start = globaltimer_ns();
        t_phase = t_start;
        n_conf = n_phases = ns_bar = ns_sw = ns_an = ns_de = ns_st = ns_slow = ns_slow_sw = 0ull;
        ns_slow_long = ns_slow_buck = 0ull;
        r_conf = 0u;
        r_idx = 0u;
    }
    if (threadIdx.x == 0) { s_tlearned = 0ull; s_tbuckets = 0ull; s_wmax[0] = s_wmax[1] = 0ull; t_cta0 = globaltimer_ns(); }

    if (threadIdx.x == 0) ldcg_copy(&sC, D.ctl);
    if (D.heuristic == 2) {
        uint16_t *w = const_cast<uint16_t *>(reinterpret_cast<const uint16_t *>(S.mlp));
        for (uint32_t i = threadIdx.x; i < (uint32_t)MLP_PARAMS; i += blockDim.x) w[i] = __ldg(D.mlp + i);
    }
    cta_sync();
    view_reload(D, V, 4u << (sC.round & 1u));
    unit_table(D, cta);
    if constexpr (UNITS && !BATCH) {
        // frontier by units: the CTA's unit range, no unit queued yet
        if (threadIdx.x == 0 && D.frontier >= 2u) {
            s_ub[0] = __ldg(D.cta_ubase + cta);
            s_ub[1] = __ldg(D.cta_ubase + cta + 1u);
            for (uint32_t w = 0; w < DQ_BITS / 32u; w++) s_dqbits[w] = 0u;
            for (uint32_t w = 0; w < DQ_WAVES; w++) s_wave[w] = 0u;
        }
    }
    cta_sync();

    for (uint32_t k = 0;; k++) {
        if (threadIdx.x == 0) {
            ldcg_copy(&sC, D.ctl + (k & 1u));
            ldcg_copy(&sA, D.acc + ((k + 3u) & 3u));
        }
        cta_sync();
        const Ctl C = sC;
        const Acc A = sA;
        if (leader) { ns_slow += A.tbusy; ns_slow_sw += A.tsweep; ns_slow_long += A.tlong; ns_slow_buck += A.tbuck; }
        if (C.op == OP_DONE) break;
        Acc *acc = D.acc + (k & 3u);
        // the next control block, written by the leader only (kept in
        // shared memory rather than in every thread's registers)
        __shared__ Ctl sN;
        Ctl &N = sN;
        if (leader) N = C;
        int kind = 0;   // 0 sweep, 1 analysis, 2 decision, 3 stability
        const uint32_t tend = C.tb + A.nclaim;
        const uint32_t fresh_cur = 4u << (C.round & 1u);
        const uint32_t fresh_prev = 4u << ((C.round + 1u) & 1u);

        // the propagate-and-check sweep of ROUND and APPLY runs after the
        // switch (one copy of its code)
        bool sw = false, sw_full = true;
        uint32_t sw_cdl = 0, sw_tbase = 0, sw_dec = 0xFFFFFFFFu, sw_fr0 = 0, sw_fr1 = 0;
        switch (C.op) {
        case OP_INIT: {
            SweepCtx X{&D, V, fresh_cur, 1u, tend, acc, true, false, 0xFFFFFFFFu, cta, rank >> 5, size >> 5};
            if (leader && D.heuristic == 5) reinterpret_cast<float *>(D.act)[D.J] = 1.0f;   // the first increment
            for (uint32_t i = gtid; i < D.n_units; i += nthreads) {
                uint32_t id = D.units_base + i;
                uint32_t l = __ldg(D.lits + id) & ~END_BIT;
                uint32_t v = l >> 1;
                uint32_t val = global_val(D, v, fresh_cur);
                uint32_t own = (l & 1u) ? V_F : V_T;
                if (val == 0u) {
                    const uint32_t valbit = (l & 1u) ? V_T : V_F;
                    int r = claim_var(D.asg, v, valbit, fresh_cur);
                    if (r == 0) record_claim(X, v, valbit, id);
                    else if (r == 2) report_conflict(X, id, 1u);
                } else if (val == own) {
                    report_conflict(X, id, 1u);
                }
            }
            if (leader) {
                N.op = OP_ROUND; N.round = C.round + 1u; N.tb = tend; N.tc = C.tc; N.clean = 0; N.full = 1;
            }
            break;
        }
        case OP_ROUND: {
            if (A.ckey != NO_KEY) {
                kind = 1;
                if (D.mode == MODE_PROPAGATE || C.cdl <= 1u) {
                    if (leader) {
                        N.op = OP_DONE;
                        N.conflict = 1;
                        N.status = C.n_models > 0 ? 10 : 20;
                        atomicAdd(&D.stats->conflicts, 1ull);
                        n_conf++;
                    }
                    break;
                }
                if (cta0) {
                    // the conflicts to analyse: the shortest one, then (several
                    // per round) the shortest of each id class, shorter first
                    __shared__ unsigned long long s_keys[4];
                    __shared__ uint32_t s_nk, s_stop;
                    if (leader) {
                        uint32_t nk = 0;
                        s_keys[nk++] = A.ckey;
                        for (int j = 0; j < 3; j++) {
                            unsigned long long key = A.cslot[j];
                            if (key == NO_KEY || key == A.ckey) continue;
                            uint32_t i = nk++;
                            while (i > 1u && s_keys[i - 1u] > key) { s_keys[i] = s_keys[i - 1u]; i--; }
                            s_keys[i] = key;
                        }
                        s_nk = min(nk, max(D.conf_per_round, 1u));
                        s_stop = 0u;
                        atomicAdd(&D.stats->conflict_rounds, 1ull);
                        N.target = 0xFFFFFFFFu;
                    }
                    cta_sync();
                    const uint32_t nk = s_nk;
                    for (uint32_t c = 0; c < nk; c++) {
                        const uint32_t g = (uint32_t)(s_keys[c] & 0xFFFFFFFFull);
                        const uint32_t lf = N.lfill;
                        if (D.learning) res_analyze(D, S, g, C.cdl, tend, lf);
                        else analyze(D, S, g, C.cdl, lf, true);
                        if (leader) {
                            atomicAdd(&D.stats->conflicts, 1ull);
                            n_conf++;
                            if (S.misc[0] == 2u) {
                                N.op = OP_DONE; N.err = -6; N.status = 0;
                                debug_analysis(D, g, tend, lf, 0u, S.misc[1], S.misc[3]);
                                D.stats->dbg_lfill = S.misc[2];
                                s_stop = 1u;
                            } else if (S.misc[0]) {
                                N.op = OP_DONE;
                                N.status = C.n_models > 0 ? 10 : 20;
                                s_stop = 1u;
                            } else {
                                uint32_t n = S.misc[2];
                                if (lf + n + 64u >= D.lits_cap || N.n_learned + 1u >= D.learned_ng_cap) {
                                    N.op = OP_DONE; N.err = -6; N.status = 0;
                                    s_stop = 1u;
                                } else {
                                    add_learned(D, N.n_learned, lf, n);
                                    N.n_learned = N.n_learned + 1u;
                                    N.lfill = lf + n;
                                    N.op = OP_BACKJUMP;
                                    N.target = min(N.target, S.misc[1]);
                                    N.tb = tend;
                                    atomicAdd(&D.stats->learned, 1ull);
                                    atomicAdd(&D.stats->learned_lits, (unsigned long long)n);
                                    debug_analysis(D, g, tend, lf, n, S.misc[1], D.learning ? S.misc[3] : 0u);
                                }
                            }
                        }
                        cta_sync();
                        if (s_stop) break;
                    }
                    if (leader && N.op == OP_BACKJUMP && D.restart_unit &&
                        ++r_conf >= luby(r_idx + 1u) * D.restart_unit) {
                        r_conf = 0u;
                        r_idx++;
                        N.target = 1u;
                        atomicAdd(&D.stats->restarts, 1ull);
                    }
                }
                break;
            }
            if (A.nclaim == 0u && C.clean) {
                // fixpoint
                if (D.mode == MODE_PROPAGATE) {
                    if (leader) { N.op = OP_DONE; N.status = 0; }
                    break;
                }
                if (tend >= D.nv) {
                    kind = 3;
                    if (leader) N.op = OP_STAB_INIT;
                    break;
                }
                kind = 2;
                decide(D, S, acc, gtid, nthreads, C.cdl, tend);
                if (leader) N.op = OP_APPLY;
                break;
            }
            // frontier by units: this round's dirty units of the CTA
            if constexpr (UNITS && !BATCH) {
                if (D.frontier >= 2u) build_unit_queue(D, cta, D.dirty + (C.round & 1u) * D.dirty_words, 0xFFFFFFFFu);
            }
            // make last round's claims visible: clear their fresh bit
            // (grid-wide) and put them in this CTA's view
            for (uint32_t i = C.tc + gtid; i < tend; i += nthreads) {
                uint32_t v = __ldcg(D.trail + i) & TRAIL_VAR;
                if (v >= D.nv) { atomicExch(&D.bar->err, 2u); continue; }   // corrupt trail: stop with an error
                atomicAnd(D.asg + (v >> 3), ~(fresh_prev << ((v & 7u) * 4u)));
            }
            if (tend - C.tc > 4096u) {
                view_reload(D, V, fresh_cur);
            } else {
                for (uint32_t i = C.tc + threadIdx.x; i < tend; i += blockDim.x) {
                    const uint32_t e = __ldcg(D.trail + i);
                    view_set(V, e & TRAIL_VAR, (e & TRAIL_F) ? V_F : V_T);
                }
            }
            cta_sync();
            sw = true; sw_cdl = C.cdl; sw_tbase = tend;
            sw_full = C.full != 0u || D.frontier == 0u || (!UNITS && D.frontier >= 2u);
            sw_fr0 = C.tc; sw_fr1 = tend;
            if (leader) {
                N.op = OP_ROUND; N.round = C.round + 1u; N.tc = tend; N.tb = tend; N.clean = 1; N.full = 0;
                atomicAdd(&D.stats->rounds, 1ull);
                atomicAdd(&D.stats->props, (unsigned long long)(tend - C.tc));
                if (sw_full) atomicAdd(&D.stats->checks, D.static_checks);
                atomicAdd(&D.stats->visits, (sw_full ? D.static_nogoods : 0ull) + D.n_long + C.n_learned);
            }
            break;
        }
        case OP_APPLY: {
            if (A.dkey == 0ull) {
                // CompleteAssignment: falsify the unassigned atoms; their
                // dependency bitmap is every decision level so far
                kind = 2;
                SweepCtx X{&D, V, fresh_cur, C.cdl, tend, acc, true, false, 0xFFFFFFFFu, cta, rank >> 5, size >> 5};
                const uint32_t nw = deps_words(D, C.cdl);
                for (uint32_t p = gtid; p < D.na; p += nthreads) {
                    if ((nib(__ldcg(D.asg + (p >> 3)), p) & 3u) != 0u) continue;
                    if (claim_var(D.asg, p, V_F, fresh_cur) == 0) {
                        record_claim(X, p, V_F, R_COMPLETE);
                        if (C.cdl > 1u)
                            for (uint32_t w = 0; w < nw; w++)
                                D.deps[(size_t)p * D.WW + w] = all_levels_word(D, C.cdl, w);
                    }
                }
                if (leader) {
                    // (frontier by units: completion claims mark no units, so
                    // the next round sweeps everything)
                    N.op = OP_ROUND; N.round = C.round + 1u; N.tb = tend; N.tc = tend; N.clean = 0;
                    N.full = D.frontier >= 2u ? 1u : 0u;
                    atomicAdd(&D.stats->completions, 1ull);
                }
                break;
            }
            const uint32_t j = 0xFFFFFFFFu - (uint32_t)(A.dkey & 0xFFFFFFFFull);
            if (j >= D.J || C.cdl + 1u > D.J + 1u) {
                // a decision key that names no rule: stop with an error
                // rather than write outside the arrays
                if (leader) { N.op = OP_DONE; N.err = -6; N.status = 0; }
                break;
            }
            const uint32_t L = C.cdl + 1u;
            const uint32_t bv = D.na + 3u * j;
            if (leader) {
                D.level_start[L] = tend;
                D.dec_var[L] = bv;
                D.trail[tend] = bv;
                if (D.tpos) D.tpos[bv] = tend;
                D.dl[bv] = (int32_t)L;
                D.reason[bv] = R_DECISION;
                uint32_t nw = deps_words(D, L), bit = level_bit(D, L);
                for (uint32_t w = 0; w < nw; w++)
                    D.deps[(size_t)bv * D.WW + w] = (w == (bit >> 6)) ? (1ull << (bit & 63u)) : 0ull;
                __threadfence();
                atomicOr(D.asg + (bv >> 3), V_T << ((bv & 7u) * 4u));
            }
            if (threadIdx.x == 0) view_set(V, bv, V_T);
            if (UNITS && D.frontier >= 2u) {
                uint32_t *buf = D.dirty + (C.round & 1u) * D.dirty_words;
                if constexpr (UNITS && !BATCH) {
                    build_unit_queue(D, cta, buf, bv);
                } else if (threadIdx.x < 32u) {
                    // one program per CTA: the decision variable's units go
                    // into the bitmap the sweep takes its words from
                    const uint32_t o0 = __ldg(D.occ_uoff + bv), o1 = __ldg(D.occ_uoff + bv + 1u);
                    for (uint32_t o = o0 + threadIdx.x; o < o1; o += 32u) {
                        const uint32_t u = __ldg(D.occ_unit + o);
                        atomicOr(buf + (u >> 5), 1u << (u & 31u));
                    }
                }
            }
            cta_sync();
            sw = true; sw_cdl = L; sw_tbase = tend + 1u; sw_dec = bv;
            sw_full = D.frontier == 0u || (!UNITS && D.frontier >= 2u);
            if (leader) {
                N.op = OP_ROUND; N.cdl = L; N.round = C.round + 1u; N.tc = tend + 1u; N.tb = tend + 1u;
                N.clean = 0; N.full = 0;
                atomicAdd(&D.stats->decisions, 1ull);
                atomicAdd(&D.stats->rounds, 1ull);
                if (sw_full) atomicAdd(&D.stats->checks, D.static_checks);
                atomicAdd(&D.stats->visits, (sw_full ? D.static_nogoods : 0ull) + D.n_long + C.n_learned);
                if ((unsigned long long)L > D.stats->max_level) D.stats->max_level = L;
            }
            break;
        }
        case OP_BACKJUMP: {
            kind = 1;
            const uint32_t newend = __ldcg(D.level_start + C.target + 1u);
            for (uint32_t i = newend + gtid; i < tend; i += nthreads) {
                uint32_t v = __ldcg(D.trail + i) & TRAIL_VAR;
                if (v >= D.nv) { atomicExch(&D.bar->err, 2u); continue; }
                atomicAnd(D.asg + (v >> 3), ~(0xFu << ((v & 7u) * 4u)));
                D.dl[v] = 0;
            }
            for (uint32_t i = newend + threadIdx.x; i < tend; i += blockDim.x)
                view_clear(V, __ldcg(D.trail + i) & TRAIL_VAR);
            if (leader) {
                N.op = OP_ROUND; N.cdl = C.target; N.tc = newend; N.tb = newend; N.clean = 0; N.full = 1;
            }
            break;
        }
        case OP_STAB_INIT: {
            kind = 3;
            const uint32_t words = (D.na + 31u) >> 5;
            for (uint32_t w = gtid; w < words; w += nthreads) D.lm[w] = 0u;
            if (leader) { N.op = OP_STAB_ITER; N.stab_first = 1; N.tb = tend; }
            break;
        }
        case OP_STAB_ITER: {
            kind = 3;
            if (!C.stab_first && A.flag == 0u) {
                // least model reached: look for true atoms outside it
                for (uint32_t p = gtid; p < D.na; p += nthreads) {
                    bool inM = (nib(__ldcg(D.asg + (p >> 3)), p) & 3u) == V_T;
                    bool inLM = (__ldcg(D.lm + (p >> 5)) >> (p & 31u)) & 1u;
                    if (inM && !inLM) atomicMin(&acc->minU, p);
                }
                if (leader) N.op = OP_STAB_RESULT;
                break;
            }
            // one pass of T over the reduct: rules whose negative body avoids
            // M and whose positive body lies in the current set
            for (uint32_t j = gtid; j < D.J; j += nthreads) {
                uint32_t h = (uint32_t)__ldg(D.rule_head + j);
                if ((__ldcg(D.lm + (h >> 5)) >> (h & 31u)) & 1u) continue;
                bool ok = true;
                for (uint32_t q = __ldg(D.rneg_off + j); ok && q < __ldg(D.rneg_off + j + 1); q++) {
                    uint32_t a = __ldg(D.rneg + q);
                    if ((nib(__ldcg(D.asg + (a >> 3)), a) & 3u) == V_T) ok = false;
                }
                for (uint32_t q = __ldg(D.rpos_off + j); ok && q < __ldg(D.rpos_off + j + 1); q++) {
                    uint32_t a = __ldg(D.rpos + q);
                    if (!((__ldcg(D.lm + (a >> 5)) >> (a & 31u)) & 1u)) ok = false;
                }
                if (ok) {
                    atomicOr(D.lm + (h >> 5), 1u << (h & 31u));
                    atomicOr(&acc->flag, 1u);
                }
            }
            if (leader) { N.op = OP_STAB_ITER; N.stab_first = 0; }
            break;
        }
        case OP_STAB_RESULT: {
            kind = 3;
            if (A.minU == 0xFFFFFFFFu) {
                // answer set: record it, then block it with the decision literals
                const long long row = C.n_models;
                const uint32_t words = (D.na + 63u) >> 6;
                if (D.trace && row == 0) {
                    // label each sampled candidate: does its body hold in the answer set
                    const uint32_t nrec = min(__ldcg(&D.stats->trace_n), D.trace_cap);
                    for (uint32_t r = gtid; r < nrec; r += nthreads) {
                        uint32_t *rec = D.trace + (size_t)r * TRACE_WORDS;
                        const uint32_t b = D.na + 3u * rec[16];
                        rec[18] = (nib(__ldcg(D.asg + (b >> 3)), b) & 3u) == V_T ? 1u : 0u;
                        rec[19] = 1u;
                    }
                }
                if (row < D.models_cap) {
                    for (uint32_t w = gtid; w < words; w += nthreads) {
                        unsigned long long m = 0;
                        for (uint32_t q = 0; q < 64u; q++) {
                            uint32_t p = w * 64u + q;
                            if (p < D.na && (nib(__ldcg(D.asg + (p >> 3)), p) & 3u) == V_T) m |= 1ull << q;
                        }
                        D.models[(size_t)row * words + w] = m;
                    }
                }
                if (leader) {
                    atomicAdd(&D.stats->models, 1ull);
                    N.n_models = C.n_models + 1;
                    if ((D.max_models > 0 && N.n_models >= D.max_models) || C.cdl <= 1u) {
                        N.op = OP_DONE; N.status = 10;
                    } else if (C.lfill + C.cdl + 64u >= D.lits_cap || C.n_learned + 1u >= D.learned_ng_cap) {
                        N.op = OP_DONE; N.err = -6; N.status = 10;
                    } else {
                        uint32_t n = 0;
                        for (uint32_t level = 2; level <= C.cdl; level++)
                            D.lits[C.lfill + n++] = mk_lit(__ldcg(D.dec_var + level), false);
                        D.lits[C.lfill + n - 1u] |= END_BIT;
                        add_learned(D, C.n_learned, C.lfill, n);
                        N.n_learned = C.n_learned + 1u;
                        N.lfill = C.lfill + n;
                        N.op = OP_BACKJUMP;
                        N.target = C.cdl - 1u;
                        atomicAdd(&D.stats->learned, 1ull);
                        atomicAdd(&D.stats->learned_lits, (unsigned long long)n);
                    }
                }
                break;
            }
            // not an answer set: loop nogood {Tp} u {Fb_j : head(j) in U,
            // body+(j) disjoint from U} for U = M \ LM(reduct), p = min U
            const uint32_t p = A.minU;
            for (uint32_t j = gtid; j < D.J; j += nthreads) {
                uint32_t h = (uint32_t)__ldg(D.rule_head + j);
                bool hU = ((nib(__ldcg(D.asg + (h >> 3)), h) & 3u) == V_T) && !((__ldcg(D.lm + (h >> 5)) >> (h & 31u)) & 1u);
                if (!hU) continue;
                bool ext = true;
                for (uint32_t q = __ldg(D.rpos_off + j); ext && q < __ldg(D.rpos_off + j + 1); q++) {
                    uint32_t a = __ldg(D.rpos + q);
                    bool aU = ((nib(__ldcg(D.asg + (a >> 3)), a) & 3u) == V_T) && !((__ldcg(D.lm + (a >> 5)) >> (a & 31u)) & 1u);
                    if (aU) ext = false;
                }
                if (ext) {
                    uint32_t pos = C.lfill + 1u + atomicAdd(&acc->nlits, 1u);
                    if (pos + 64u < D.lits_cap) D.lits[pos] = mk_lit(D.na + 3u * j, true);
                }
            }
            if (leader) {
                D.lits[C.lfill] = mk_lit(p, false);
                N.op = OP_ANALYZE_ID;
                N.conf_id = C.lfill;
                atomicAdd(&D.stats->loops, 1ull);
            }
            break;
        }
        case OP_ANALYZE_ID: {
            kind = 1;
            const uint32_t len = 1u + A.nlits;
            if (C.lfill + len + C.cdl + 64u >= D.lits_cap || C.n_learned + 2u >= D.learned_ng_cap) {
                if (leader) { N.op = OP_DONE; N.err = -6; N.status = C.n_models > 0 ? 10 : 0; }
                break;
            }
            if (cta0) {
                if (leader) {
                    D.lits[C.lfill + len - 1u] |= END_BIT;
                    add_learned(D, C.n_learned, C.lfill, len);
                    __threadfence();
                }
                cta_sync();
                const uint32_t lf = C.lfill + len;
                if (D.learning) res_analyze(D, S, C.conf_id, C.cdl, tend, lf);
                else analyze(D, S, C.conf_id, C.cdl, lf, false);
                if (leader) {
                    atomicAdd(&D.stats->conflicts, 1ull);
                    n_conf++;
                    atomicAdd(&D.stats->learned, 1ull);
                    atomicAdd(&D.stats->learned_lits, (unsigned long long)len);
                    if (S.misc[0] == 2u) {
                        N.op = OP_DONE; N.err = -6; N.status = 0;
                        debug_analysis(D, C.conf_id, tend, lf, 0u, S.misc[1], S.misc[3]);
                        D.stats->dbg_lfill = S.misc[2];
                    } else if (S.misc[0]) {
                        N.op = OP_DONE;
                        N.status = C.n_models > 0 ? 10 : 20;
                        N.n_learned = C.n_learned + 1u;
                        N.lfill = lf;
                    } else {
                        uint32_t n = S.misc[2];
                        add_learned(D, C.n_learned + 1u, lf, n);
                        N.n_learned = C.n_learned + 2u;
                        N.lfill = lf + n;
                        N.op = OP_BACKJUMP;
                        N.target = S.misc[1];
                        atomicAdd(&D.stats->learned, 1ull);
                        atomicAdd(&D.stats->learned_lits, (unsigned long long)n);
                        debug_analysis(D, C.conf_id, tend, lf, n, S.misc[1], D.learning ? S.misc[3] : 0u);
                        if (D.restart_unit && ++r_conf >= luby(r_idx + 1u) * D.restart_unit) {
                            r_conf = 0u;
                            r_idx++;
                            N.target = 1u;
                            atomicAdd(&D.stats->restarts, 1ull);
                        }
                    }
                }
            }
            break;
        }
        default:
            if (leader) { N.op = OP_DONE; N.err = -6; }
            break;
        }
        if (sw) {
            const unsigned long long ts = threadIdx.x == 0 ? globaltimer_ns() : 0ull;
            SweepCtx X{&D, V, fresh_cur, sw_cdl, sw_tbase, acc, true, true, sw_dec, cta, rank >> 5, size >> 5};
            if (UNITS && D.frontier >= 2u) X.dmark = D.dirty + ((C.round + 1u) & 1u) * D.dirty_words;
            sweep<UNITS ? (BATCH ? 2 : 1) : 0>(X, C.n_learned, sw_full, sw_fr0, sw_fr1, 0u,
                                               D.frontier >= 2u ? D.dirty + (C.round & 1u) * D.dirty_words : nullptr);
            if (threadIdx.x == 0) atomicMax(&acc->tsweep, globaltimer_ns() - ts);
        }

        if (leader) {
            if (D.mode == MODE_SOLVE && N.op != OP_DONE) {
                unsigned long long now = globaltimer_ns();
                bool over_time = D.time_budget_ns > 0 && (long long)(now - t_start) > D.time_budget_ns;
                bool over_conf = D.conflict_budget > 0 && (long long)n_conf >= D.conflict_budget;
                if (over_time || over_conf) { N.op = OP_DONE; N.status = N.n_models > 0 ? 10 : 0; }
            }
            D.ctl[(k + 1u) & 1u] = N;
            Acc z;
            z.ckey = NO_KEY; z.cslot[0] = z.cslot[1] = z.cslot[2] = NO_KEY; z.dkey = 0; z.nclaim = 0; z.flag = 0; z.minU = 0xFFFFFFFFu; z.nlits = 0; z.checks = 0; z.visits = 0;
            z.tbusy = 0; z.tsweep = 0; z.tlong = 0; z.tbuck = 0;
            D.acc[(k + 1u) & 3u] = z;
            // fold long-nogood checks of the previous phase into the stats
            if (A.checks) atomicAdd(&D.stats->checks, A.checks);
            if (A.visits) atomicAdd(&D.stats->visits, A.visits);
            unsigned long long now = globaltimer_ns();
            unsigned long long dt = now - t_phase;
            t_phase = now;
            if (kind == 0) ns_sw += dt;
            else if (kind == 1) ns_an += dt;
            else if (kind == 2) ns_de += dt;
            else ns_st += dt;
            n_phases++;
            __threadfence();
        }
        const unsigned long long tb0 = threadIdx.x == 0 ? globaltimer_ns() : 0ull;
        if (threadIdx.x == 0) atomicMax(&acc->tbusy, tb0 - t_cta0);
        if (!BATCH && k == 0 && D.stall_cta != 0xFFFFFFFFu) injected_stall(D);
        if (!group_sync<BATCH>(D, k)) break;
        if (threadIdx.x == 0) t_cta0 = globaltimer_ns();
        if (leader) ns_bar += t_cta0 - tb0;
    }
    if (leader) {
        const Ctl F = sC;
        D.stats->pad = F.tc;
        D.stats->ns_total = globaltimer_ns() - t_start;
        D.stats->ns_sweep = ns_sw;
        D.stats->ns_analysis = ns_an;
        D.stats->ns_decision = ns_de;
        D.stats->ns_stab = ns_st;
        D.stats->phases = n_phases;
        D.stats->ns_barrier = ns_bar;
        D.stats->ns_learned = s_tlearned;
        D.stats->ns_buckets = s_tbuckets;
        D.stats->ns_slowest = ns_slow;
        D.stats->ns_slowest_sweep = ns_slow_sw;
        D.stats->ns_slowest_long = ns_slow_long;
        D.stats->ns_slowest_buckets = ns_slow_buck;
        int err = F.err;
        if (__ldcg(&D.bar->err)) err = -6;
        D.result[0] = F.status;
        D.result[1] = F.n_models;
        D.result[2] = err;
        D.result[3] = F.conflict;
    }
}

// The dynamic shared-memory limit is a property of each kernel, shared by
// every program: it is set to the largest size any program may use, and
// occupancy is computed for a program's own size.
constexpr int MAX_DYN_SMEM = 220 * 1024;

}  // namespace aspgpu
