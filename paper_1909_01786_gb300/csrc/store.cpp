// Completion nogoods of a ground normal program, packed for the device
// (Section 2 for the nogoods; Section 4 for the store sorted by length).
//
// Rules with a head are renumbered in order of their head atom, so rules(p)
// is a contiguous range.  Nogoods are generated group by group: for each atom
// p, the nogoods of each rule of p followed by p's own nogood
// {Tp} u {Fb_r : r in rules(p)}; then one group per constraint.  Each nogood
// goes to the bucket of its exact length (2..BUCKET_MAX; Section 4 uses one
// kernel per length class), keeping group order inside a bucket, so the
// nogoods of a range of groups refer to a contiguous range of auxiliary
// variables b_r, t_r, n_r, which a CTA keeps in shared memory.  Unit nogoods
// go to a separate list that InitialPropagation applies once (Algorithm 1);
// longer nogoods go to a CSR region.
#include "store.h"

#include <algorithm>
#include <cmath>
#include <cstring>

#include "aspgpu.h"

namespace aspgpu {

namespace {

struct Packer {
    HostStore &S;
    uint32_t group = 0;

    explicit Packer(HostStore &s) : S(s) {}

    void add(const uint32_t *l, int64_t len) {
        S.n_nogoods++;
        S.n_literals += len;
        if (len == 0) { S.has_empty_nogood = true; return; }
        if (len == 1) { S.units.push_back(l[0]); return; }
        S.group_lits[group] += (uint64_t)len;
        if (len > BUCKET_MAX) {
            S.long_rel.push_back((uint32_t)S.long_lits.size());
            for (int64_t i = 0; i < len; i++) S.long_lits.push_back(l[i] | (i == len - 1 ? END_BIT : 0u));
            return;
        }
        S.bucket_rows[len].insert(S.bucket_rows[len].end(), l, l + len);
        S.bucket_group[len].push_back(group);
    }
};

}  // namespace

int build_store(int32_t n_atoms, int32_t n_rules, const int32_t *head,
                const int64_t *pos_off, const int32_t *pos,
                const int64_t *neg_off, const int32_t *neg,
                HostStore &S, std::string &err, bool compact)
{
    if (n_atoms < 0 || n_rules < 0) { err = "negative size"; return ASP_E_ARG; }
    if (n_rules > 0 && (!head || !pos_off || !neg_off)) { err = "null rule array"; return ASP_E_ARG; }
    if (n_rules > 0 && (pos_off[0] != 0 || neg_off[0] != 0)) { err = "offsets must start at 0"; return ASP_E_ARG; }
    int64_t n_headed = 0;
    for (int32_t r = 0; r < n_rules; r++) {
        if (pos_off[r + 1] < pos_off[r] || neg_off[r + 1] < neg_off[r]) { err = "offsets not monotone"; return ASP_E_ARG; }
        if (head[r] < -1 || head[r] >= n_atoms) { err = "head atom out of range"; return ASP_E_RANGE; }
        n_headed += head[r] >= 0;
    }
    if ((pos_off && pos_off[n_rules] > 0 && !pos) || (neg_off && neg_off[n_rules] > 0 && !neg)) {
        err = "null body array"; return ASP_E_ARG;
    }
    for (int64_t k = 0; n_rules > 0 && k < pos_off[n_rules]; k++)
        if (pos[k] < 0 || pos[k] >= n_atoms) { err = "body atom out of range"; return ASP_E_RANGE; }
    for (int64_t k = 0; n_rules > 0 && k < neg_off[n_rules]; k++)
        if (neg[k] < 0 || neg[k] >= n_atoms) { err = "body atom out of range"; return ASP_E_RANGE; }
    int64_t nv = (int64_t)n_atoms + 3 * n_headed;
    if (nv > MAX_VARS) { err = "too many variables (atoms + 3 x rules >= 2^30)"; return ASP_E_RANGE; }

    S = HostStore();
    S.n_atoms = n_atoms;
    S.n_rules = n_rules;
    S.n_headed = (int32_t)n_headed;
    S.n_vars = nv;
    const uint32_t J = (uint32_t)n_headed, A = (uint32_t)n_atoms;
    auto bvar = [&](uint32_t j) { return A + 3 * j; };
    auto tvar = [&](uint32_t j) { return A + 3 * j + 1; };
    auto nvar = [&](uint32_t j) { return A + 3 * j + 2; };

    // headed rules sorted by head atom (ties in input order), bodies
    // deduplicated: rules(p) is then a contiguous index range
    std::vector<int32_t> order;
    order.reserve(J);
    for (int32_t r = 0; r < n_rules; r++) if (head[r] >= 0) order.push_back(r);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return head[a] < head[b]; });
    S.rule_index = order;
    S.rule_head.reserve(J);
    S.rpos_off.push_back(0);
    S.rneg_off.push_back(0);
    std::vector<uint32_t> mark((size_t)n_atoms + 1, 0);
    uint32_t stamp = 0;
    for (int32_t r : order) {
        S.rule_head.push_back(head[r]);
        ++stamp;
        for (int64_t k = pos_off[r]; k < pos_off[r + 1]; k++)
            if (mark[pos[k]] != stamp) { mark[pos[k]] = stamp; S.rpos.push_back((uint32_t)pos[k]); }
        S.rpos_off.push_back((uint32_t)S.rpos.size());
        ++stamp;
        for (int64_t k = neg_off[r]; k < neg_off[r + 1]; k++)
            if (mark[neg[k]] != stamp) { mark[neg[k]] = stamp; S.rneg.push_back((uint32_t)neg[k]); }
        S.rneg_off.push_back((uint32_t)S.rneg.size());
    }

    // p -> OR_{r in rules(p)} b_r needs rules(p): contiguous after sorting
    std::vector<uint32_t> first((size_t)n_atoms + 1, 0);
    for (uint32_t j = 0; j < J; j++) first[S.rule_head[j] + 1]++;
    for (int32_t p = 0; p < n_atoms; p++) first[p + 1] += first[p];

    int64_t n_constraints = (int64_t)n_rules - (int64_t)n_headed;
    S.n_groups = (int32_t)(n_atoms + n_constraints);
    S.group_lits.assign((size_t)S.n_groups + 1, 0);
    Packer pk(S);
    std::vector<uint32_t> buf;
    auto rule_nogoods = [&](uint32_t j) {
        uint32_t b = bvar(j), t = tvar(j), n = nvar(j);
        uint32_t x[3];
        // b_r <-> t_r & n_r : {Fb,Tt,Tn} {Tb,Ft} {Tb,Fn}.  Compact: with an
        // empty B+ (B-) the unit nogood {Ft} ({Fn}) below makes t_r (n_r)
        // true at the root, so {Tb,Ft} ({Tb,Fn}) can never be violated and
        // Tt (Tn) always holds in {Fb,Tt,Tn}.
        const bool t_const = compact && S.rpos_off[j + 1] == S.rpos_off[j];
        const bool n_const = compact && S.rneg_off[j + 1] == S.rneg_off[j];
        int m = 0;
        x[m++] = mk_lit(b, true);
        if (!t_const) x[m++] = mk_lit(t, false);
        if (!n_const) x[m++] = mk_lit(n, false);
        pk.add(x, m);
        if (!t_const) { x[0] = mk_lit(b, false); x[1] = mk_lit(t, true); pk.add(x, 2); }
        if (!n_const) { x[0] = mk_lit(b, false); x[1] = mk_lit(n, true); pk.add(x, 2); }
        // t_r <-> body+ : {Tt,Fp} per p, {Ft} u {Tp}
        buf.assign(1, mk_lit(t, true));
        for (uint32_t k = S.rpos_off[j]; k < S.rpos_off[j + 1]; k++) {
            x[0] = mk_lit(t, false); x[1] = mk_lit(S.rpos[k], true); pk.add(x, 2);
            buf.push_back(mk_lit(S.rpos[k], false));
        }
        pk.add(buf.data(), (int64_t)buf.size());
        // n_r <-> not body- : {Tn,Tq} per q, {Fn} u {Fq}
        buf.assign(1, mk_lit(n, true));
        for (uint32_t k = S.rneg_off[j]; k < S.rneg_off[j + 1]; k++) {
            x[0] = mk_lit(n, false); x[1] = mk_lit(S.rneg[k], false); pk.add(x, 2);
            buf.push_back(mk_lit(S.rneg[k], true));
        }
        pk.add(buf.data(), (int64_t)buf.size());
        // head <- b_r : {Fhead, Tb}
        x[0] = mk_lit((uint32_t)S.rule_head[j], true); x[1] = mk_lit(b, false); pk.add(x, 2);
    };
    for (int32_t p = 0; p < n_atoms; p++) {
        pk.group = (uint32_t)p;
        for (uint32_t j = first[p]; j < first[p + 1]; j++) rule_nogoods(j);
        // p -> OR_{r in rules(p)} b_r : {Tp} u {Fb_r}
        buf.assign(1, mk_lit((uint32_t)p, false));
        for (uint32_t j = first[p]; j < first[p + 1]; j++) buf.push_back(mk_lit(bvar(j), true));
        pk.add(buf.data(), (int64_t)buf.size());
    }
    // constraints {Tp1..Tpm, Fpm+1..Fpn} (repeated literals once)
    uint32_t cgroup = (uint32_t)n_atoms;
    for (int32_t r = 0; r < n_rules; r++) {
        if (head[r] >= 0) continue;
        pk.group = cgroup++;
        buf.clear();
        for (int64_t k = pos_off[r]; k < pos_off[r + 1]; k++) buf.push_back(mk_lit((uint32_t)pos[k], false));
        for (int64_t k = neg_off[r]; k < neg_off[r + 1]; k++) buf.push_back(mk_lit((uint32_t)neg[k], true));
        std::sort(buf.begin(), buf.end());
        buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
        pk.add(buf.data(), (int64_t)buf.size());
    }
    // static decision score: occurrences of the head atom in the nogoods
    std::vector<uint32_t> occ((size_t)n_atoms + 1, 0);
    auto count = [&](uint32_t w) {
        uint32_t v = (w & ~END_BIT) >> 1;
        if (v < A) occ[v]++;
    };
    for (int L = 2; L <= BUCKET_MAX; L++) for (uint32_t w : S.bucket_rows[L]) count(w);
    for (uint32_t w : S.long_lits) count(w);
    for (uint32_t u : S.units) count(u);
    S.score.resize(J);
    for (uint32_t j = 0; j < J; j++) S.score[j] = occ[S.rule_head[j]];

    // Jeroslow-Wang score (Section 4 names it among the decision
    // heuristics): a nogood delta is the clause "not all of delta", which a
    // literal l satisfies when its complement is in delta, weighted 2^-|delta|.
    // Deciding Tb_r makes b_r true and then head(r) true, so the score of rule
    // r is the sum of 2^-|delta| over the nogoods holding Fb_r or F head(r),
    // in fixed point (x 2^16, saturating).
    std::vector<uint64_t> jw_f((size_t)nv + 1, 0);     // per variable: sum over nogoods with its F literal
    auto jw_add = [&](const uint32_t *l, size_t len) {
        const uint64_t w = len < 17 ? (1ull << (16 - len)) : 0ull;
        for (size_t q = 0; q < len; q++) {
            const uint32_t lit = l[q] & ~END_BIT;
            if (lit & 1u) jw_f[lit >> 1] += w;
        }
    };
    for (int L = 2; L <= BUCKET_MAX; L++) {
        const std::vector<uint32_t> &rows = S.bucket_rows[L];
        for (size_t t = 0; t + (size_t)L <= rows.size(); t += (size_t)L) jw_add(rows.data() + t, (size_t)L);
    }
    for (size_t i = 0; i < S.long_rel.size(); i++) {
        const size_t s0 = S.long_rel[i];
        const size_t s1 = i + 1 < S.long_rel.size() ? S.long_rel[i + 1] : S.long_lits.size();
        jw_add(S.long_lits.data() + s0, s1 - s0);
    }
    for (uint32_t u : S.units) jw_add(&u, 1);
    S.score_jw.resize(J);
    for (uint32_t j = 0; j < J; j++) {
        const uint64_t sc = jw_f[bvar(j)] + jw_f[(uint32_t)S.rule_head[j]];
        S.score_jw[j] = (uint32_t)std::min<uint64_t>(sc, 0x7FFFFFFFull);
    }

    // static features of each rule (inputs of the learned heuristic):
    // log1p occurrences of the head, |B+|, |B-|, log1p |rules(head)|,
    // log1p positive and negative body occurrences of the head, log1p of the
    // positive body occurrences of the atoms the rule falsifies, 1
    std::vector<uint32_t> posocc((size_t)n_atoms + 1, 0), negocc((size_t)n_atoms + 1, 0);
    for (uint32_t a : S.rpos) posocc[a]++;
    for (uint32_t a : S.rneg) negocc[a]++;
    S.rfeat.assign((size_t)J * RULE_STATIC_FEATURES, 0.0f);
    for (uint32_t j = 0; j < J; j++) {
        float *f = S.rfeat.data() + (size_t)j * RULE_STATIC_FEATURES;
        const uint32_t h = (uint32_t)S.rule_head[j];
        uint64_t blocked = 0;
        for (uint32_t k = S.rneg_off[j]; k < S.rneg_off[j + 1]; k++) blocked += posocc[S.rneg[k]];
        f[0] = std::log1p((float)occ[h]);
        f[1] = (float)(S.rpos_off[j + 1] - S.rpos_off[j]);
        f[2] = (float)(S.rneg_off[j + 1] - S.rneg_off[j]);
        f[3] = std::log1p((float)(first[h + 1] - first[h]));
        f[4] = std::log1p((float)posocc[h]);
        f[5] = std::log1p((float)negocc[h]);
        f[6] = std::log1p((float)blocked);
        f[7] = 1.0f;
    }

    for (int L = 2; L <= BUCKET_MAX; L++)
        if (S.bucket_group[L].size() >= (1u << 27)) { err = "too many nogoods of one length (>= 2^27)"; return ASP_E_RANGE; }
    if ((uint64_t)S.n_literals >= 0x7FFF0000ull) { err = "nogood store exceeds 2^31 literals"; return ASP_E_RANGE; }
    return ASP_OK;
}

}  // namespace aspgpu
