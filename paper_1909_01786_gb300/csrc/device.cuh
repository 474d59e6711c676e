// Device-side data layout and small helpers of the solver (internal).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace aspgpu {

// reason markers (anything else is the id of the reason nogood = the offset
// of its first literal in the literal array)
constexpr uint32_t R_DECISION = 0xFFFFFFFFu;
constexpr uint32_t R_COMPLETE = 0xFFFFFFFEu;
constexpr uint32_t R_INPUT = 0xFFFFFFFDu;

// Assignment: one 4-bit code per variable, 8 per 32-bit word.
//   bit 0: true, bit 1: false, bit 2 / bit 3: claimed in an even / odd
//   round and not yet committed ("fresh").  A fresh variable reads as
//   unassigned during the round that claimed it, so every sweep classifies
//   nogoods against the assignment as it stood when the round began (plus
//   clash detection through the atomic claim), and dependency bitmaps are
//   only ever computed from committed variables.
constexpr uint32_t V_T = 1u, V_F = 2u;

// Trail entries: the variable, with TRAIL_F set if it was made false (so a
// round can put the previous round's claims into its views without reading
// the codes).
constexpr uint32_t TRAIL_F = 0x80000000u;
constexpr uint32_t TRAIL_VAR = 0x7FFFFFFFu;

enum Op : uint32_t {
    OP_INIT = 1,      // InitialPropagation: apply the unit nogoods at level 1
    OP_ROUND,         // commit last round's claims, then propagate-and-check sweep
    OP_APPLY,         // apply the chosen decision (or complete the assignment) + sweep
    OP_BACKJUMP,      // unassign every trail entry above the target level
    OP_STAB_INIT,     // stability check: clear the least-model bitset
    OP_STAB_ITER,     // one pass of the immediate-consequence operator of the reduct
    OP_STAB_RESULT,   // answer set found -> record it and block it; else loop nogood
    OP_ANALYZE_ID,    // conflict analysis of the loop nogood just written
    OP_DONE
};

enum Mode : uint32_t { MODE_SOLVE = 0, MODE_PROPAGATE = 1 };

// Shared-memory view of a CTA (values ASP_VIEW_PLAIN/PACKED/BYTES)
enum ViewMode : uint32_t { VIEW_PLAIN = 1, VIEW_PACKED = 2, VIEW_BYTES = 3 };

constexpr unsigned long long NO_KEY = ~0ull;

// learned heuristic: 16 features -> 64 hidden (ReLU) -> 1, parameters
// W1[64][16], b1[64], w2[64], b2
constexpr int N_FEATURES = 16, N_HIDDEN = 64;
constexpr int MLP_PARAMS = N_FEATURES * N_HIDDEN + 2 * N_HIDDEN + 1;
// trace record: 16 feature words (float bits), rule, level, label, labelled
constexpr int TRACE_WORDS = 20;
// a candidate rule is sampled into the trace when its hash has these bits clear
constexpr uint32_t TRACE_SAMPLE_MASK = 7u;

struct Ctl {              // double-buffered control block (phase parity)
    uint32_t op, cdl, tc, tb;   // tc: trail entries committed; tb: base of last claims
    // (a claim's level, reason and dependency bitmap are written when it is
    // made; "committing" only clears its fresh bit and makes it visible to
    // every CTA's shared-memory view)
    uint32_t round, clean, target, conf_id;
    uint32_t n_learned, lfill, stab_first, trace_n;
    long long n_models;
    int32_t status, err;
    int32_t conflict;
    uint32_t full;              // the next round sweeps every nogood (else the frontier)
};

struct Acc {              // per-phase accumulators, indexed by phase % 4
    unsigned long long ckey;    // min over conflicts of (length << 32 | nogood id)
    unsigned long long cslot[3]; // the same over conflicts with id % 3 == 0, 1, 2 (several
                                 // conflicts per round)
    unsigned long long dkey;    // max over candidate rules of (score << 32 | ~j)
    uint32_t nclaim;            // variables claimed in the phase
    uint32_t flag;              // something changed (least-model iteration)
    uint32_t minU;              // smallest unfounded true atom
    uint32_t nlits;             // literals appended to the loop nogood
    unsigned long long checks;  // literals classified by long/learned sweeps (and by unit
                                // frontiers' bucket units)
    unsigned long long visits;  // bucket nogoods classified by unit frontiers
    unsigned long long tbusy;   // max over CTAs of the time from phase start to barrier arrival
    unsigned long long tsweep;  // max over CTAs of the time in the sweep
    unsigned long long tlong;   // max over warps of the sweep's long and learned nogoods
    unsigned long long tbuck;   // max over warps of the sweep's bucket units
};

struct DevStats {
    unsigned long long rounds, checks, props, conflicts, decisions, completions;
    unsigned long long learned, learned_lits, loops, models, max_level;
    unsigned long long ns_total, ns_sweep, ns_analysis, ns_decision, ns_stab;
    unsigned long long phases, pad;
    // time inside sweeps seen by CTA 0: static buckets, long and learned
    // nogoods, and waiting at the phase barrier
    unsigned long long ns_buckets, ns_learned, ns_barrier, pad2;
    // sums over phases of the slowest CTA's busy time and sweep time
    unsigned long long ns_slowest, ns_slowest_sweep;
    unsigned long long restarts, conflict_rounds;
    // nogoods classified by the sweeps (every sweep: the long and learned
    // nogoods, plus the bucket nogoods when it is a full sweep)
    unsigned long long visits;
    unsigned int trace_n, pad4;    // trace records written (atomic)
    // the last conflict analysis: conflicting nogood, trail length (claims of
    // the conflict round included), learned nogood id and length, backjump
    // target, and the level the nogood was resolved at (0 for fwd-learning)
    unsigned long long dbg_conf, dbg_tend, dbg_lfill, dbg_len, dbg_target, dbg_level;
    // sums over phases of the slowest warp's time on long and learned
    // nogoods and on bucket units (any CTA)
    unsigned long long ns_slowest_long, ns_slowest_buckets;
};

// Grid barrier: arrivals counted since the launch began (zeroed by the host
// before each launch; barrier g is complete once count >= (g + 1) * CTAs);
// err is set by a CTA that gave up
// waiting; stall is a flag that nothing sets (the test-only stalled CTA
// waits on it).
struct Barrier { unsigned long long count; unsigned int err, stall; };

struct Dev {
    uint32_t na, J, nv, asg_words;
    uint32_t n_long, n_units, units_base, pad1;
    // bucket L (2..15): literal q of nogood k at lits[bk_base[L] + q*bk_n[L] + k]
    uint32_t bk_base[16], bk_n[16];
    uint32_t lits_static, lits_cap, learned_ng_cap, pad0;
    uint32_t WW, Wlevels, mode, heuristic;
    // fwd-learning backjump: 0 to h-1 (h = highest level of the conflict's
    // bitmap), 1 to the second-highest level (the asserting level);
    // restart_unit: Luby restarts every luby(i) x restart_unit learned
    // nogoods (0 = none)
    uint32_t backjump, restart_unit;
    // conflicts analysed per conflicting round (1..4): the shortest, then
    // the shortest of each class id % 3; the lowest target wins
    uint32_t conf_per_round;
    // test-only failure injection: this CTA does not arrive at the first
    // phase barrier (0xFFFFFFFF = none); it waits, bounded, on a flag that
    // nothing sets until another CTA gives up on the barrier
    uint32_t stall_cta;
    // static partition of the buckets over the CTAs by groups (atoms and
    // their rules; constraints): CTA g owns nogoods [cta_boff[L*(G+1)+g],
    // cta_boff[L*(G+1)+g+1]) of bucket L, and keeps in shared memory the
    // atoms [0, view_atoms) and the auxiliary variables
    // [cta_auxlo, cta_auxlo + cta_auxn) those nogoods refer to
    uint32_t G, view_atoms, view_words, view_mode;
    const uint32_t *cta_boff;    // [16 * (G+1)]
    const uint32_t *cta_auxlo;   // [G]
    const uint32_t *cta_auxn;    // [G]
    // view_mode PACKED or BYTES: the buckets again (same offsets), each
    // literal rewritten for its owner CTA as (view entry << 2) | xmask with
    // xmask = 3 for a false literal, 0 for a true one
    const uint32_t *vlits;
    long long max_models, models_cap, conflict_budget, time_budget_ns;
    unsigned long long static_checks;    // literals of the buckets (read every sweep)
    unsigned long long static_nogoods;   // nogoods of the buckets
    unsigned long long barrier_ns;       // grid barrier: give up after this wait
    uint32_t *lits;                      // buckets | long | units | learned
    const uint32_t *long_ids;
    uint32_t *learned_ids;
    // watched literals of the long and learned nogoods (Algorithm 2): two
    // positions per nogood, long nogood i at i, learned nogood i at n_long + i
    uint2 *nwatch;
    const int32_t *rule_head;
    const uint32_t *rpos_off, *rpos, *rneg_off, *rneg, *score;
    // per rule: conflicts it took part in (heuristic 1), or its VSIDS-style
    // activity as a float with the increment after the J rules (heuristic 5)
    uint32_t *act;
    const uint32_t *head_first;   // heuristic 5: rules of atom p are [head_first[p], head_first[p+1])
    // learned decision heuristic (heuristic 2): static rule features
    // [J][8], MLP weights (bf16 bits, MLP_PARAMS), decision trace
    const float *rfeat;
    const uint16_t *mlp;
    const float *prior;       // heuristic 3: per-rule score computed at load
    uint32_t *trace;          // [trace_cap][TRACE_WORDS]
    uint32_t trace_cap;
    // frontier propagation (Algorithm 2's idea): a round checks only the
    // bucket nogoods of the variables assigned in the previous round, found
    // through occ_off/occ (per variable, the ids of the bucket nogoods it
    // occurs in); full sweeps after (re)starts and backjumps
    uint32_t frontier;
    const uint32_t *occ_off, *occ;
    // frontier = 2 (frontier by bucket units): the sweep units of the static
    // partition are numbered globally, CTA g's being [cta_ubase[g],
    // cta_ubase[g+1]); occ_unit[occ_uoff[v] .. occ_uoff[v+1]) are the units
    // whose nogoods hold variable v.  A claim sets the bits of v's units in
    // the next round's dirty bitmap (two bitmaps of dirty_words words,
    // alternating by round); each round's sweep checks the units whose bit
    // is set and clears them.
    const uint32_t *cta_ubase, *occ_uoff, *occ_unit;
    uint32_t *dirty;
    uint32_t dirty_words, pad3;
    uint32_t *asg;
    int32_t *dl;
    uint32_t *reason;
    unsigned long long *deps;
    uint32_t *trail, *level_start, *dec_var, *lm;
    // learning = 1 (Algorithm 3, resolution to the first UIP): trail
    // position of each assigned variable (written with its trail entry), a
    // per-variable stamp marking the variables of the nogood being resolved,
    // a bitset over trail positions of its literals at the conflict level,
    // and the stamp counter (one word, never reset: stamps of earlier
    // analyses, in this solve or an earlier one, are all smaller)
    uint32_t learning;
    uint32_t *tpos, *stamp, *cand, *epoch;
    Ctl *ctl;
    Acc *acc;
    DevStats *stats;
    Barrier *bar;
    unsigned long long *models;
    long long *result;
};

}  // namespace aspgpu
