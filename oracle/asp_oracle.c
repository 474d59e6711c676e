/*
 * CPU oracle for answer-set computation of ground normal programs.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, written to be checked against the
 * paper by eye.  Only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it; the solver library never does, and this file
 * shares no code, header or table with it.
 *
 * Paper: Dovier, Formisano, Vella, "GPU-based parallelism for ASP-solving"
 * (arXiv 1909.01786).
 *
 *   O1  answer-set definition, brute force:
 *       M is an answer set iff M = LM(reduct(P, M)) and M violates no
 *       constraint (Section 1, "Answer Set Programming": answer set = the
 *       subset-minimal model of the reduct; immediate-consequence operator T_P
 *       whose least fixpoint is LM, read with body-(r) ∩ I = ∅ -- the printed
 *       "body+(r) ∩ I = ∅" is a typesetting slip).
 *   O2  a simple conflict-driven nogood-learning solver (Section 2):
 *       completion nogoods (Section 2, list of nogoods for b_r, t_r, n_r and
 *       p <-> OR b_r, plus constraint nogoods), unit propagation (Section 2,
 *       "delta \ A = {Fp} => add Tp"), ASP-computation decisions (Section 2,
 *       select Tb_r for an applicable rule of an unassigned head; when none
 *       exists falsify the unassigned heads), first-UIP resolution learning
 *       (Section 4.2, Algorithm 3), and a final reduct check (the paper's
 *       method does no unfounded-set check; atoms forced true only by
 *       propagation can lack support, so a total assignment is accepted only
 *       if it passes O1's check; otherwise a loop nogood is added).
 *   UP  the unit-propagation closure of a partial assignment under the
 *       completion nogoods, by the naive fixpoint of the definition.
 *   The completion also comes in a compact variant (for empty positive or
 *   negative bodies, the nogoods that the unit nogood {Ft_r} / {Fn_r}
 *   settles at the root are left out); O2 uses the full one.
 *
 * Variables: atoms 0..na-1, then for the j-th rule with a head (in rule
 * order) b_j = na+3j, t_j = na+3j+1, n_j = na+3j+2.
 * Literals: +(v+1) is Tv, -(v+1) is Fv.  A nogood is violated when all of its
 * literals hold.  Decision levels start at 1 (the root, Algorithm 1).
 *
 * Parity pins: none of these functions is "parity unpinned"; the tests pin O1
 * against the minimal-model definition by subset brute force and hand cases,
 * O2 against O1, UP against the fixpoint/derivation properties, the encoder
 * against closed-form counts and a hand-written listing.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

typedef struct {
    int32_t na, nr;
    const int32_t *head;
    const int64_t *pos_off;
    const int32_t *pos;
    const int64_t *neg_off;
    const int32_t *neg;
} oprog;

/* ------------------------------------------------------------------ O1 */

/* Least model of the reduct P^M: rules whose negative body meets M are
 * dropped, the negative bodies of the others are deleted; iterate T_P^M from
 * the empty set until nothing changes. */
static void least_model_of_reduct(const oprog *P, const uint8_t *M, uint8_t *LM)
{
    memset(LM, 0, (size_t)P->na);
    int changed = 1;
    while (changed) {
        changed = 0;
        for (int32_t r = 0; r < P->nr; r++) {
            int32_t h = P->head[r];
            if (h < 0 || LM[h]) continue;
            int blocked = 0;
            for (int64_t k = P->neg_off[r]; k < P->neg_off[r + 1]; k++)
                if (M[P->neg[k]]) blocked = 1;
            if (blocked) continue;
            int body = 1;
            for (int64_t k = P->pos_off[r]; k < P->pos_off[r + 1]; k++)
                if (!LM[P->pos[k]]) body = 0;
            if (body) { LM[h] = 1; changed = 1; }
        }
    }
}

static int violates_a_constraint(const oprog *P, const uint8_t *M)
{
    for (int32_t r = 0; r < P->nr; r++) {
        if (P->head[r] >= 0) continue;
        int body = 1;
        for (int64_t k = P->pos_off[r]; k < P->pos_off[r + 1]; k++)
            if (!M[P->pos[k]]) body = 0;
        for (int64_t k = P->neg_off[r]; k < P->neg_off[r + 1]; k++)
            if (M[P->neg[k]]) body = 0;
        if (body) return 1;
    }
    return 0;
}

int oracle_is_answer_set(const oprog *P, const uint8_t *M)
{
    uint8_t *LM = (uint8_t *)malloc((size_t)P->na + 1);
    least_model_of_reduct(P, M, LM);
    int same = memcmp(LM, M, (size_t)P->na) == 0;
    free(LM);
    return same && !violates_a_constraint(P, M);
}

void oracle_least_model_of_reduct(const oprog *P, const uint8_t *M, uint8_t *LM)
{
    least_model_of_reduct(P, M, LM);
}

/* All answer sets by enumerating every subset of the atoms (na <= 26).
 * Models are written as rows of na bytes; returns the number found (rows
 * beyond cap are counted but not stored). */
int64_t oracle_brute_force(const oprog *P, uint8_t *models, int64_t cap)
{
    if (P->na > 26) return -1;
    uint8_t *M = (uint8_t *)malloc((size_t)P->na + 1);
    int64_t found = 0;
    for (uint64_t mask = 0; mask < (1ull << P->na); mask++) {
        for (int32_t i = 0; i < P->na; i++) M[i] = (uint8_t)((mask >> i) & 1u);
        if (oracle_is_answer_set(P, M)) {
            if (found < cap) memcpy(models + found * P->na, M, (size_t)P->na);
            found++;
        }
    }
    free(M);
    return found;
}

/* ------------------------------------------------------------ nogood store */

typedef struct {
    int64_t n, cap_ng;
    int64_t *off;          /* [n+1] */
    int32_t *lit;
    int64_t nlit, cap_lit;
} ngdb;

static void db_init(ngdb *d)
{
    memset(d, 0, sizeof(*d));
    d->cap_ng = 1024; d->cap_lit = 4096;
    d->off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(d->cap_ng + 1));
    d->lit = (int32_t *)malloc(sizeof(int32_t) * (size_t)d->cap_lit);
    d->off[0] = 0;
}

static void db_free(ngdb *d) { free(d->off); free(d->lit); }

static int64_t db_add(ngdb *d, const int32_t *lits, int64_t len)
{
    while (d->nlit + len > d->cap_lit) {
        d->cap_lit *= 2;
        d->lit = (int32_t *)realloc(d->lit, sizeof(int32_t) * (size_t)d->cap_lit);
    }
    if (d->n + 1 > d->cap_ng) {
        d->cap_ng *= 2;
        d->off = (int64_t *)realloc(d->off, sizeof(int64_t) * (size_t)(d->cap_ng + 1));
    }
    memcpy(d->lit + d->nlit, lits, sizeof(int32_t) * (size_t)len);
    d->nlit += len;
    d->n++;
    d->off[d->n] = d->nlit;
    return d->n - 1;
}

static int64_t rules_with_head(const oprog *P)
{
    int64_t c = 0;
    for (int32_t r = 0; r < P->nr; r++) c += P->head[r] >= 0;
    return c;
}

#define TLIT(v) ((int32_t)(v) + 1)
#define FLIT(v) (-((int32_t)(v) + 1))

/* Completion nogoods and constraint nogoods (Section 2).  Body atoms are
 * taken as sets (repeated atoms in one body count once).
 * compact != 0: the compact variant.  A rule with no positive body atom has
 * t_r fixed true by its unit nogood {Ft_r}; then {Tb_r, Ft_r} can never hold
 * and Tt_r always holds, so that nogood is left out and Tt_r is left out of
 * {Fb_r, Tt_r, Tn_r}.  Likewise for n_r when the negative body is empty. */
static void build_completion(const oprog *P, ngdb *d, int compact)
{
    int32_t na = P->na;
    int32_t buf_cap = 16;
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)buf_cap);
    uint8_t *seen = (uint8_t *)calloc((size_t)na + 1, 1);
    int64_t j = 0;
    /* rules(p) for the per-atom nogood */
    int64_t *cnt = (int64_t *)calloc((size_t)na + 1, sizeof(int64_t));
    for (int32_t r = 0; r < P->nr; r++) if (P->head[r] >= 0) cnt[P->head[r]]++;
    for (int32_t r = 0; r < P->nr; r++) {
        int64_t need = 2 + (P->pos_off[r + 1] - P->pos_off[r]) + (P->neg_off[r + 1] - P->neg_off[r]);
        if (need > buf_cap) { buf_cap = (int32_t)need * 2; buf = (int32_t *)realloc(buf, sizeof(int32_t) * (size_t)buf_cap); }
        if (P->head[r] < 0) {
            /* constraint nogood {Tp1..Tpm, Fpm+1..Fpn} */
            int32_t L = 0;
            for (int64_t k = P->pos_off[r]; k < P->pos_off[r + 1]; k++) {
                int32_t a = P->pos[k];
                int dup = 0;
                for (int32_t q = 0; q < L; q++) if (buf[q] == TLIT(a)) dup = 1;
                if (!dup) buf[L++] = TLIT(a);
            }
            for (int64_t k = P->neg_off[r]; k < P->neg_off[r + 1]; k++) {
                int32_t a = P->neg[k];
                int dup = 0;
                for (int32_t q = 0; q < L; q++) if (buf[q] == FLIT(a)) dup = 1;
                if (!dup) buf[L++] = FLIT(a);
            }
            db_add(d, buf, L);
            continue;
        }
        int32_t b = na + 3 * (int32_t)j, t = b + 1, n = b + 2;
        int32_t x[3];
        int pos_empty = P->pos_off[r + 1] == P->pos_off[r];
        int neg_empty = P->neg_off[r + 1] == P->neg_off[r];
        /* b_r <-> t_r & n_r */
        if (!compact) {
            x[0] = FLIT(b); x[1] = TLIT(t); x[2] = TLIT(n); db_add(d, x, 3);
            x[0] = TLIT(b); x[1] = FLIT(t); db_add(d, x, 2);
            x[0] = TLIT(b); x[1] = FLIT(n); db_add(d, x, 2);
        } else {
            int32_t m = 0;
            x[m++] = FLIT(b);
            if (!pos_empty) x[m++] = TLIT(t);
            if (!neg_empty) x[m++] = TLIT(n);
            db_add(d, x, m);
            if (!pos_empty) { x[0] = TLIT(b); x[1] = FLIT(t); db_add(d, x, 2); }
            if (!neg_empty) { x[0] = TLIT(b); x[1] = FLIT(n); db_add(d, x, 2); }
        }
        /* t_r <-> conjunction of body+ */
        int32_t L = 0;
        buf[L++] = FLIT(t);
        for (int64_t k = P->pos_off[r]; k < P->pos_off[r + 1]; k++) {
            int32_t a = P->pos[k];
            if (seen[a] & 1) continue;
            seen[a] |= 1;
            x[0] = TLIT(t); x[1] = FLIT(a); db_add(d, x, 2);
            buf[L++] = TLIT(a);
        }
        for (int64_t k = P->pos_off[r]; k < P->pos_off[r + 1]; k++) seen[P->pos[k]] &= (uint8_t)~1u;
        db_add(d, buf, L);
        /* n_r <-> conjunction of negated body- */
        L = 0;
        buf[L++] = FLIT(n);
        for (int64_t k = P->neg_off[r]; k < P->neg_off[r + 1]; k++) {
            int32_t a = P->neg[k];
            if (seen[a] & 2) continue;
            seen[a] |= 2;
            x[0] = TLIT(n); x[1] = TLIT(a); db_add(d, x, 2);
            buf[L++] = FLIT(a);
        }
        for (int64_t k = P->neg_off[r]; k < P->neg_off[r + 1]; k++) seen[P->neg[k]] &= (uint8_t)~2u;
        db_add(d, buf, L);
        /* head <- b_r */
        x[0] = FLIT(P->head[r]); x[1] = TLIT(b); db_add(d, x, 2);
        j++;
    }
    /* p -> OR of b_r over rules(p): {Tp} u {Fb_r} */
    int64_t *first = (int64_t *)malloc(sizeof(int64_t) * ((size_t)na + 1));
    int64_t *rl = (int64_t *)malloc(sizeof(int64_t) * (size_t)(j + 1));
    first[0] = 0;
    for (int32_t p = 0; p < na; p++) first[p + 1] = first[p] + cnt[p];
    int64_t *fill = (int64_t *)calloc((size_t)na + 1, sizeof(int64_t));
    j = 0;
    for (int32_t r = 0; r < P->nr; r++) {
        if (P->head[r] < 0) continue;
        int32_t h = P->head[r];
        rl[first[h] + fill[h]++] = j++;
    }
    for (int32_t p = 0; p < na; p++) {
        int64_t L = 1 + cnt[p];
        if (L > buf_cap) { buf_cap = (int32_t)L * 2; buf = (int32_t *)realloc(buf, sizeof(int32_t) * (size_t)buf_cap); }
        buf[0] = TLIT(p);
        for (int64_t q = 0; q < cnt[p]; q++) buf[1 + q] = FLIT(na + 3 * (int32_t)rl[first[p] + q]);
        db_add(d, buf, L);
    }
    free(first); free(rl); free(fill); free(cnt); free(seen); free(buf);
}

/* Export the oracle's own completion (compact != 0: the compact variant):
 * pass NULL buffers to get the sizes. */
int oracle_completion(const oprog *P, int compact, int64_t *n_nogoods, int64_t *n_lits, int64_t *n_vars,
                      int64_t *off_out, int32_t *lit_out)
{
    ngdb d;
    db_init(&d);
    build_completion(P, &d, compact);
    *n_nogoods = d.n;
    *n_lits = d.nlit;
    *n_vars = P->na + 3 * rules_with_head(P);
    if (off_out) memcpy(off_out, d.off, sizeof(int64_t) * (size_t)(d.n + 1));
    if (lit_out) memcpy(lit_out, d.lit, sizeof(int32_t) * (size_t)d.nlit);
    db_free(&d);
    return 0;
}

/* ---------------------------------------------------- UP closure (naive) */

static int lit_holds(const int8_t *val, int32_t l) { return l > 0 ? val[l - 1] == 1 : val[-l - 1] == -1; }
static int lit_opposed(const int8_t *val, int32_t l) { return l > 0 ? val[l - 1] == -1 : val[-l - 1] == 1; }

/* Unit-propagation closure of `partial` (per variable: 1 true, -1 false,
 * 0 unassigned) under the completion nogoods, by the definition: repeat over
 * all nogoods -- violated => conflict; exactly one literal not in A and the
 * rest in A => add its complement -- until nothing changes.
 * Writes the closure, the derivation order (variables, signed as literals
 * that were added) and each derived literal's reason nogood index.
 * Returns 1 on conflict (closure then holds the state when it was found),
 * 0 otherwise. */
int oracle_up_closure(const oprog *P, int compact, const int8_t *partial, int8_t *closure,
                      int32_t *order, int64_t *reasons, int64_t *n_derived)
{
    ngdb d;
    db_init(&d);
    build_completion(P, &d, compact);
    int64_t nv = P->na + 3 * rules_with_head(P);
    memcpy(closure, partial, (size_t)nv);
    int64_t nd = 0;
    int conflict = 0;
    int changed = 1;
    while (changed && !conflict) {
        changed = 0;
        for (int64_t g = 0; g < d.n && !conflict; g++) {
            int64_t n_out = 0;
            int32_t out = 0;
            int sat = 0;
            for (int64_t k = d.off[g]; k < d.off[g + 1]; k++) {
                int32_t l = d.lit[k];
                if (lit_opposed(closure, l)) { sat = 1; break; }
                if (!lit_holds(closure, l)) { n_out++; out = l; }
            }
            if (sat) continue;
            if (n_out == 0) { conflict = 1; break; }
            if (n_out == 1) {
                int32_t add = -out;
                closure[(add > 0 ? add : -add) - 1] = (int8_t)(add > 0 ? 1 : -1);
                if (order) order[nd] = add;
                if (reasons) reasons[nd] = g;
                nd++;
                changed = 1;
            }
        }
    }
    *n_derived = nd;
    db_free(&d);
    return conflict;
}

/* ------------------------------------------------------------------ O2 */

typedef struct {
    const oprog *P;
    int32_t na, nv, nrr;
    int32_t *rule_of;     /* j -> rule index r */
    ngdb db;
    int64_t n_static;
    /* occurrence lists: per variable, nogood ids (grown) */
    int64_t **occ;
    int32_t *occ_n, *occ_cap;
    int8_t *val;
    int32_t *lvl;
    int64_t *reason;       /* nogood index, -1 = decision / unassigned */
    int64_t *tpos;         /* trail position */
    int32_t *trail;        /* variables in assignment order */
    int64_t trail_n, qhead;
    int64_t *lim;          /* lim[l] = trail size when level l started */
    int32_t cdl;
    /* scratch */
    uint8_t *mark;
    int32_t *tmp;
    int64_t tmp_cap;
    int64_t conflicts, decisions, propagations;
    int64_t literal_checks;    /* literals read and classified (instrumentation) */
} cdnl;

static void occ_push(cdnl *S, int32_t v, int64_t g)
{
    if (S->occ_n[v] == S->occ_cap[v]) {
        S->occ_cap[v] = S->occ_cap[v] ? 2 * S->occ_cap[v] : 4;
        S->occ[v] = (int64_t *)realloc(S->occ[v], sizeof(int64_t) * (size_t)S->occ_cap[v]);
    }
    S->occ[v][S->occ_n[v]++] = g;
}

static int64_t add_nogood(cdnl *S, const int32_t *lits, int64_t len)
{
    int64_t g = db_add(&S->db, lits, len);
    for (int64_t k = 0; k < len; k++) occ_push(S, (lits[k] > 0 ? lits[k] : -lits[k]) - 1, g);
    return g;
}

static void assign(cdnl *S, int32_t lit, int64_t reason)
{
    int32_t v = (lit > 0 ? lit : -lit) - 1;
    S->val[v] = (int8_t)(lit > 0 ? 1 : -1);
    S->lvl[v] = S->cdl;
    S->reason[v] = reason;
    S->tpos[v] = S->trail_n;
    S->trail[S->trail_n++] = v;
}

static void backjump(cdnl *S, int32_t level)
{
    while (S->trail_n > S->lim[level + 1]) {
        int32_t v = S->trail[--S->trail_n];
        S->val[v] = 0;
        S->lvl[v] = 0;
        S->reason[v] = -1;
    }
    S->qhead = S->trail_n;
    S->cdl = level;
}

/* 0 = satisfied or open, 1 = unit (out = the single literal not in A),
 * 2 = violated */
static int classify(cdnl *S, int64_t g, int32_t *out)
{
    int64_t n_out = 0;
    for (int64_t k = S->db.off[g]; k < S->db.off[g + 1]; k++) {
        int32_t l = S->db.lit[k];
        S->literal_checks++;
        if (lit_opposed(S->val, l)) return 0;
        if (!lit_holds(S->val, l)) { n_out++; *out = l; if (n_out > 1) return 0; }
    }
    return n_out == 0 ? 2 : 1;
}

/* Check nogoods [from, to): assign units, return the first violated one. */
static int64_t check_range(cdnl *S, int64_t from, int64_t to)
{
    for (int64_t g = from; g < to; g++) {
        int32_t out = 0;
        int c = classify(S, g, &out);
        if (c == 2) return g;
        if (c == 1) { assign(S, -out, g); S->propagations++; }
    }
    return -1;
}

/* Queue-driven unit propagation: each newly assigned variable re-examines
 * the nogoods it occurs in.  Returns a violated nogood or -1 at fixpoint. */
static int64_t propagate(cdnl *S)
{
    while (S->qhead < S->trail_n) {
        int32_t v = S->trail[S->qhead++];
        for (int32_t i = 0; i < S->occ_n[v]; i++) {
            int64_t g = S->occ[v][i];
            int32_t out = 0;
            int c = classify(S, g, &out);
            if (c == 2) return g;
            if (c == 1) { assign(S, -out, g); S->propagations++; }
        }
    }
    return -1;
}

static int32_t lit_var(int32_t l) { return (l > 0 ? l : -l) - 1; }

/* First-UIP learning (Algorithm 3): resolve the violated nogood with the
 * reason of its last-assigned literal while another of its literals has the
 * same decision level.  Returns the learned nogood length in S->tmp and sets
 * *kappa (the highest level among the others, at least 1) and *uip. */
static int64_t first_uip(cdnl *S, int64_t g, int32_t *kappa, int32_t *uip)
{
    int64_t len = 0;
    /* delta as a marked set of literals */
    for (int64_t k = S->db.off[g]; k < S->db.off[g + 1]; k++) {
        int32_t l = S->db.lit[k], v = lit_var(l);
        if (!S->mark[v]) { S->mark[v] = 1; S->tmp[len++] = l; }
    }
    for (;;) {
        int64_t last = -1;
        for (int64_t i = 0; i < len; i++)
            if (last < 0 || S->tpos[lit_var(S->tmp[i])] > S->tpos[lit_var(S->tmp[last])]) last = i;
        int32_t sigma = S->tmp[last];
        int32_t ls = S->lvl[lit_var(sigma)];
        int32_t k = 1;
        for (int64_t i = 0; i < len; i++)
            if (i != last && S->lvl[lit_var(S->tmp[i])] > k) k = S->lvl[lit_var(S->tmp[i])];
        int others_at_ls = 0;
        for (int64_t i = 0; i < len; i++)
            if (i != last && S->lvl[lit_var(S->tmp[i])] == ls) others_at_ls = 1;
        if (!others_at_ls) {
            *kappa = k;
            *uip = sigma;
            break;
        }
        /* resolve with epsilon = reason(sigma), which contains -sigma */
        int64_t e = S->reason[lit_var(sigma)];
        S->mark[lit_var(sigma)] = 0;
        S->tmp[last] = S->tmp[--len];
        for (int64_t q = S->db.off[e]; q < S->db.off[e + 1]; q++) {
            int32_t l = S->db.lit[q], v = lit_var(l);
            if (v == lit_var(sigma)) continue;
            if (!S->mark[v]) {
                if (len + 1 > S->tmp_cap) {
                    S->tmp_cap *= 2;
                    S->tmp = (int32_t *)realloc(S->tmp, sizeof(int32_t) * (size_t)S->tmp_cap);
                }
                S->mark[v] = 1;
                S->tmp[len++] = l;
            }
        }
    }
    for (int64_t i = 0; i < len; i++) S->mark[lit_var(S->tmp[i])] = 0;
    return len;
}

/* Handle a violated nogood.  Returns 1 when no (further) model exists. */
static int handle_conflict(cdnl *S, int64_t g)
{
    S->conflicts++;
    int32_t m = 1;
    for (int64_t k = S->db.off[g]; k < S->db.off[g + 1]; k++)
        if (S->lvl[lit_var(S->db.lit[k])] > m) m = S->lvl[lit_var(S->db.lit[k])];
    if (m <= 1) return 1;
    if (m < S->cdl) backjump(S, m);
    int32_t kappa = 1, uip = 0;
    int64_t len = first_uip(S, g, &kappa, &uip);
    int64_t learned = add_nogood(S, S->tmp, len);
    backjump(S, kappa);
    assign(S, -uip, learned);
    S->propagations++;
    return 0;
}

/* Loop nogood for an unfounded set U containing p: {Tp} u {Fb_r : head(r) in
 * U, body+(r) disjoint from U}.  Every answer set satisfies it (loop formula
 * of U). */
static int64_t loop_nogood(cdnl *S, const uint8_t *inU, int32_t p)
{
    const oprog *P = S->P;
    int64_t len = 0;
    int64_t need = 1 + S->nrr;
    if (need > S->tmp_cap) { S->tmp_cap = need; S->tmp = (int32_t *)realloc(S->tmp, sizeof(int32_t) * (size_t)S->tmp_cap); }
    S->tmp[len++] = TLIT(p);
    for (int32_t j = 0; j < S->nrr; j++) {
        int32_t r = S->rule_of[j];
        if (!inU[P->head[r]]) continue;
        int ext = 1;
        for (int64_t k = P->pos_off[r]; k < P->pos_off[r + 1]; k++)
            if (inU[P->pos[k]]) ext = 0;
        if (ext) S->tmp[len++] = FLIT(S->na + 3 * j);
    }
    return add_nogood(S, S->tmp, len);
}

/* Returns 10 (SAT: at least one model), 20 (UNSAT or all enumerated with
 * none), 0 (budget exhausted).  models: rows of na bytes. */
int oracle_cdnl(const oprog *P, int64_t max_models, int64_t conflict_budget, double time_budget_s,
                uint8_t *models, int64_t cap, int64_t *n_models, int64_t *stats)
{
    cdnl S;
    memset(&S, 0, sizeof(S));
    S.P = P;
    S.na = P->na;
    S.nrr = (int32_t)rules_with_head(P);
    S.nv = S.na + 3 * S.nrr;
    S.rule_of = (int32_t *)malloc(sizeof(int32_t) * ((size_t)S.nrr + 1));
    for (int32_t r = 0, j = 0; r < P->nr; r++) if (P->head[r] >= 0) S.rule_of[j++] = r;
    db_init(&S.db);
    build_completion(P, &S.db, 0);
    S.n_static = S.db.n;
    size_t nv = (size_t)S.nv + 1;
    S.occ = (int64_t **)calloc(nv, sizeof(int64_t *));
    S.occ_n = (int32_t *)calloc(nv, sizeof(int32_t));
    S.occ_cap = (int32_t *)calloc(nv, sizeof(int32_t));
    for (int64_t g = 0; g < S.db.n; g++)
        for (int64_t k = S.db.off[g]; k < S.db.off[g + 1]; k++) occ_push(&S, lit_var(S.db.lit[k]), g);
    S.val = (int8_t *)calloc(nv, 1);
    S.lvl = (int32_t *)calloc(nv, sizeof(int32_t));
    S.reason = (int64_t *)malloc(sizeof(int64_t) * nv);
    for (size_t v = 0; v < nv; v++) S.reason[v] = -1;
    S.tpos = (int64_t *)calloc(nv, sizeof(int64_t));
    S.trail = (int32_t *)malloc(sizeof(int32_t) * nv);
    S.lim = (int64_t *)calloc(nv + 2, sizeof(int64_t));
    S.mark = (uint8_t *)calloc(nv, 1);
    S.tmp_cap = (int64_t)nv + 16;
    S.tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)S.tmp_cap);
    uint8_t *M = (uint8_t *)calloc((size_t)S.na + 1, 1);
    uint8_t *LM = (uint8_t *)calloc((size_t)S.na + 1, 1);
    uint8_t *inU = (uint8_t *)calloc((size_t)S.na + 1, 1);
    clock_t t0 = clock();

    int64_t found = 0;
    int status = 20;
    S.cdl = 1;
    S.lim[1] = 0;
    /* initial propagation: every nogood once, then the queue */
    int64_t conf = check_range(&S, 0, S.db.n);
    if (conf < 0) conf = propagate(&S);
    if (conf >= 0) goto done;               /* violation at level 1 */
    for (;;) {
        if (conf >= 0) {
            if (handle_conflict(&S, conf)) break;
            /* learned nogoods may be unit after backjumping */
            conf = check_range(&S, S.n_static, S.db.n);
            if (conf < 0) conf = propagate(&S);
            if ((conflict_budget > 0 && S.conflicts >= conflict_budget) ||
                (time_budget_s > 0 && (double)(clock() - t0) / CLOCKS_PER_SEC > time_budget_s)) {
                status = found ? 10 : 0;
                goto done_budget;
            }
            continue;
        }
        if (S.trail_n == S.nv) {
            /* total assignment: accept only an answer set */
            for (int32_t p = 0; p < S.na; p++) M[p] = S.val[p] == 1;
            least_model_of_reduct(P, M, LM);
            int32_t pick = -1;
            for (int32_t p = 0; p < S.na; p++) {
                inU[p] = M[p] && !LM[p];
                if (inU[p] && pick < 0) pick = p;
            }
            if (pick >= 0) {
                conf = loop_nogood(&S, inU, pick);
                continue;
            }
            if (found < cap) memcpy(models + found * S.na, M, (size_t)S.na);
            found++;
            if (max_models > 0 && found >= max_models) break;
            /* blocking nogood {Tp : p in M} */
            int64_t len = 0;
            for (int32_t p = 0; p < S.na; p++) if (M[p]) S.tmp[len++] = TLIT(p);
            conf = add_nogood(&S, S.tmp, len);
            continue;
        }
        /* decision: an applicable rule of an unassigned head (lowest index) */
        int32_t pick = -1;
        for (int32_t j = 0; j < S.nrr && pick < 0; j++) {
            int32_t r = S.rule_of[j], h = P->head[r];
            int32_t t = S.na + 3 * j + 1, n = S.na + 3 * j + 2, b = S.na + 3 * j;
            if (S.val[h] == 0 && S.val[t] == 1 && S.val[n] != -1 && S.val[b] == 0) pick = j;
        }
        if (pick >= 0) {
            S.cdl++;
            S.lim[S.cdl] = S.trail_n;
            S.decisions++;
            assign(&S, TLIT(S.na + 3 * pick), -1);
        } else {
            /* no applicable rule: the unassigned atoms U form an unfounded
             * set; falsify each p in U with its loop nogood as the reason */
            int any = 0;
            for (int32_t p = 0; p < S.na; p++) { inU[p] = S.val[p] == 0; any |= inU[p]; }
            if (!any) {
                /* only auxiliary variables open: cannot happen at a fixpoint,
                 * kept as a guard */
                status = 0;
                goto done_budget;
            }
            for (int32_t p = 0; p < S.na; p++) {
                if (!inU[p]) continue;
                int64_t g = loop_nogood(&S, inU, p);
                assign(&S, FLIT(p), g);
            }
        }
        conf = propagate(&S);
    }
done:
    status = found ? 10 : 20;
done_budget:
    *n_models = found;
    if (stats) {
        stats[0] = S.decisions;
        stats[1] = S.conflicts;
        stats[2] = S.propagations;
        stats[3] = S.db.n - S.n_static;
        stats[4] = S.literal_checks;
    }
    for (int32_t v = 0; v < S.nv; v++) free(S.occ[v]);
    free(S.occ); free(S.occ_n); free(S.occ_cap);
    free(S.val); free(S.lvl); free(S.reason); free(S.tpos); free(S.trail); free(S.lim);
    free(S.mark); free(S.tmp); free(S.rule_of); free(M); free(LM); free(inU);
    db_free(&S.db);
    return status;
}
