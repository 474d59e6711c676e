// Host-side nogood store built from a ground program (internal to libaspgpu).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace aspgpu {

// Literal word: bits 0..30 = (var << 1) | sign (sign 1 = F), bit 31 = last
// literal of its nogood (in the CSR regions).  Variables stay below 2^30 - 1.
constexpr uint32_t END_BIT = 0x80000000u;
constexpr uint32_t PAD_LIT = 0x7FFFFFFFu;
constexpr int32_t MAX_VARS = (1 << 30) - 2;
// Static nogoods of length 2..BUCKET_MAX live in one bucket per length,
// stored structure-of-arrays (literal q of nogood k of bucket L at
// plane q, index k), so one lane classifies one nogood and a warp reads each
// plane with one coalesced load.  Longer ones go to a CSR region.
constexpr int BUCKET_MAX = 15;
// Nogood ids: a CSR nogood is the offset of its first literal (< 2^31); a
// bucket nogood is BUCKET_ID | (L-1) << 27 | k.
constexpr uint32_t BUCKET_ID = 0x80000000u;

#if defined(__CUDACC__)
#define ASPGPU_HD __host__ __device__
#else
#define ASPGPU_HD
#endif
ASPGPU_HD inline uint32_t mk_lit(uint32_t v, bool is_false) { return (v << 1) | (is_false ? 1u : 0u); }
ASPGPU_HD inline uint32_t bucket_nogood_id(uint32_t L, uint32_t k) { return BUCKET_ID | ((L - 1u) << 27) | k; }
// Groups of 32 nogoods per unit of sweep work, by bucket length: about 16
// literal loads in flight per lane.
ASPGPU_HD constexpr uint32_t unit_groups(uint32_t L) { return L <= 2u ? 8u : L <= 4u ? 4u : L <= 8u ? 2u : 1u; }

struct HostStore {
    int32_t n_atoms = 0, n_rules = 0, n_headed = 0;
    int64_t n_vars = 0;
    int32_t n_groups = 0;                    // atoms, then one group per constraint
    // bucket L: nogoods in group order, row-major while building
    std::vector<uint32_t> bucket_rows[BUCKET_MAX + 1];
    std::vector<uint32_t> bucket_group[BUCKET_MAX + 1];
    std::vector<uint32_t> long_lits;         // CSR with END bits
    std::vector<uint32_t> long_rel;          // start of each long nogood in long_lits
    std::vector<uint32_t> units;             // literals of unit nogoods
    bool has_empty_nogood = false;
    int64_t n_nogoods = 0, n_literals = 0;
    std::vector<uint64_t> group_lits;        // literals per group (load balance)
    // headed rules sorted by head atom (ties in input order); rule j of
    // this order owns the variables b_j, t_j, n_j = n_atoms + 3j + {0,1,2}
    std::vector<int32_t> rule_index;                 // input index of rule j
    std::vector<int32_t> rule_head;                  // [n_headed]
    std::vector<uint32_t> rpos_off, rpos, rneg_off, rneg;
    std::vector<uint32_t> score;                     // static decision score per headed rule
    std::vector<uint32_t> score_jw;                  // Jeroslow-Wang score per headed rule (x 2^16)
    std::vector<float> rfeat;                        // [n_headed][8] static features of each rule
};

// static features per rule for the learned decision heuristic
constexpr int RULE_STATIC_FEATURES = 8;

// Returns 0 or a negative ASP_E_* code with a message in err.  compact:
// for a rule with an empty positive (negative) body, leave out the nogoods
// that the unit nogood {Ft_r} ({Fn_r}) satisfies at the root and drop the
// literal Tt_r (Tn_r) from {Fb_r, Tt_r, Tn_r}.
int build_store(int32_t n_atoms, int32_t n_rules, const int32_t *head,
                const int64_t *pos_off, const int32_t *pos,
                const int64_t *neg_off, const int32_t *neg,
                HostStore &out, std::string &err, bool compact = false);

}  // namespace aspgpu
