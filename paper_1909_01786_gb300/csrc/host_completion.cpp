// Host-side views of the nogood store that asp_load_ground builds (Section 2:
// completion nogoods and constraint nogoods; Section 4: the decision scores),
// without a device: the same build_store that loading runs, written out for
// inspection and for tests that run on machines without a GPU.
#include <cstring>
#include <string>

#include "aspgpu.h"
#include "store.h"

namespace aspgpu {
int internal_fail(int code, const char *msg);
}  // namespace aspgpu

namespace {

using aspgpu::HostStore;

int build(int32_t n_atoms, int32_t n_rules, const int32_t *head, const int64_t *pos_off, const int32_t *pos,
          const int64_t *neg_off, const int32_t *neg, int32_t compact, HostStore &S)
{
    std::string err;
    const int rc = aspgpu::build_store(n_atoms, n_rules, head, pos_off, pos, neg_off, neg, S, err, compact != 0);
    if (rc != ASP_OK) return aspgpu::internal_fail(rc, err.c_str());
    return ASP_OK;
}

}  // namespace

extern "C" int asp_debug_completion(int32_t n_atoms, int32_t n_rules, const int32_t *head,
                                    const int64_t *pos_off, const int32_t *pos,
                                    const int64_t *neg_off, const int32_t *neg, int32_t compact,
                                    int64_t *n_vars, int64_t *n_nogoods, int64_t *n_literals,
                                    int64_t *off, int32_t *lits, int64_t lits_cap)
{
    using namespace aspgpu;
    if (!n_vars || !n_nogoods || !n_literals) return internal_fail(ASP_E_ARG, "null count pointer");
    HostStore S;
    const int rc = build(n_atoms, n_rules, head, pos_off, pos, neg_off, neg, compact, S);
    if (rc != ASP_OK) return rc;
    *n_vars = S.n_vars;
    *n_nogoods = S.n_nogoods;
    *n_literals = S.n_literals;
    if (!off && !lits) return ASP_OK;
    if (!off || !lits) return internal_fail(ASP_E_ARG, "off and lits must both be given");
    if (lits_cap < S.n_literals) return internal_fail(ASP_E_CAPACITY, "lits holds fewer than n_literals entries");
    int64_t i = 0, n = 0;
    auto emit = [&](const uint32_t *l, int64_t len) {
        off[i++] = n;
        for (int64_t q = 0; q < len; q++) lits[n++] = (int32_t)(l[q] & ~END_BIT);
    };
    // buckets by length (group order inside a bucket; rows are row-major on
    // the host), then the longer nogoods, the unit nogoods and the empty one
    for (int L = 2; L <= BUCKET_MAX; L++) {
        const std::vector<uint32_t> &rows = S.bucket_rows[L];
        for (size_t t = 0; t + (size_t)L <= rows.size(); t += (size_t)L) emit(rows.data() + t, L);
    }
    for (size_t k = 0; k < S.long_rel.size(); k++) {
        const size_t s0 = S.long_rel[k];
        const size_t s1 = k + 1 < S.long_rel.size() ? S.long_rel[k + 1] : S.long_lits.size();
        emit(S.long_lits.data() + s0, (int64_t)(s1 - s0));
    }
    for (uint32_t u : S.units) emit(&u, 1);
    // one empty nogood per empty constraint (the store keeps only the flag)
    while (S.has_empty_nogood && i < S.n_nogoods) emit(nullptr, 0);
    off[i] = n;
    if (i != S.n_nogoods || n != S.n_literals) return internal_fail(ASP_E_ARG, "store counts disagree with its regions");
    return ASP_OK;
}

extern "C" int asp_debug_rule_scores(int32_t n_atoms, int32_t n_rules, const int32_t *head,
                                     const int64_t *pos_off, const int32_t *pos,
                                     const int64_t *neg_off, const int32_t *neg, int32_t compact,
                                     int32_t *n_headed, int32_t *rule_index, uint32_t *score_occ,
                                     uint32_t *score_jw, int64_t cap)
{
    using namespace aspgpu;
    if (!n_headed) return internal_fail(ASP_E_ARG, "null count pointer");
    HostStore S;
    const int rc = build(n_atoms, n_rules, head, pos_off, pos, neg_off, neg, compact, S);
    if (rc != ASP_OK) return rc;
    *n_headed = S.n_headed;
    if (!rule_index && !score_occ && !score_jw) return ASP_OK;
    if (cap < S.n_headed) return internal_fail(ASP_E_CAPACITY, "output arrays hold fewer than n_headed entries");
    const size_t J = (size_t)S.n_headed;
    if (rule_index && J) std::memcpy(rule_index, S.rule_index.data(), J * sizeof(int32_t));
    if (score_occ && J) std::memcpy(score_occ, S.score.data(), J * sizeof(uint32_t));
    if (score_jw && J) std::memcpy(score_jw, S.score_jw.data(), J * sizeof(uint32_t));
    return ASP_OK;
}
