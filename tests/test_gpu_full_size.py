"""Parity at full size, in the launch configuration the benchmark times (needs
a GB300).

The benchmark's workload is the large random program (100k atoms, 400k
rules, seed 0) loaded with the library's default options (view chosen by
size, one CTA per SM, full sweeps, fwd-learning).  At that size the oracle
still computes two outputs exactly, and they are compared here:

- the unit-propagation closure (the fixpoint of propagate-and-check, Section
  4) of partial assignments several decisions deep, literal by literal,
  against the oracle's UP closure (also on the 400k-atom program whose store
  is larger than L2);
- fwd-learning (Section 4.2, Algorithm 4) at the k-th conflict of the
  search: every variable in the cone of the violated nogood (its variables,
  their reasons' variables, and so on down to the decisions) has a reason
  that is a nogood of the oracle's own completion (or a learned one), unit
  on that variable, and a dependency bitmap equal to the OR over that
  reason's other variables above the root (mk_dl_bitmap); a decision's
  bitmap is its own level.  With the cone checked, the learned nogood must be
  the decision literals of the levels in the OR over the violated nogood,
  the backjump target h-1 (the second-highest level under the asserting
  option), and the nogood unit there; also under the unit frontier;
- first-UIP resolution learning (Algorithm 3) at the k-th conflict: the
  learned nogood and target equal the oracle's first_uip on the GPU's state."""
import numpy as np
import pytest

import oracle
from synth.programs import large_random_program

pytestmark = pytest.mark.gpu

CONE_CAP = 200_000        # variables of the cone checked one by one


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1909_01786_gb300 import aspgpu
    aspgpu.lib()
    return aspgpu


def _rule_maps(prog):
    """Input index of the library's rule j (headed rules by head atom, ties in
    input order) and the oracle's ordinal of each input rule (headed rules in
    input order)."""
    headed = np.nonzero(prog.head >= 0)[0]
    order = headed[np.argsort(prog.head[headed], kind="stable")]
    ordinal = np.full(prog.head.shape[0], -1, np.int64)
    ordinal[headed] = np.arange(headed.shape[0])
    return order, ordinal


def _oracle_to_library(prog, nv):
    """Library variable of each oracle variable (atoms are shared; b, t, n of
    a rule sit at n_atoms + 3 x (rule number) + 0/1/2 on both sides, with
    different rule numberings)."""
    order, ordinal = _rule_maps(prog)
    na = prog.n_atoms
    o2g = np.arange(nv, dtype=np.int64)
    oj = ordinal[order]
    j = np.arange(order.shape[0])
    for q in range(3):
        o2g[na + 3 * oj + q] = na + 3 * j + q
    return o2g


class _Completion:
    """The oracle's completion nogoods in the library's literal encoding
    ((variable << 1) | is_false), with a variable -> nogoods index for
    membership tests."""

    def __init__(self, prog):
        nv, off, lits = oracle.completion(prog)
        o2g = _oracle_to_library(prog, nv)
        var = o2g[np.abs(lits).astype(np.int64) - 1]
        self.nv, self.off, self.o2g = nv, off, o2g
        self.enc = 2 * var + (lits < 0)
        ng = np.repeat(np.arange(off.shape[0] - 1), np.diff(off))
        order = np.argsort(var, kind="stable")
        self.by_var, self.ng_of = var[order], ng[order]

    def contains(self, lits):
        want = sorted({int(l) for l in lits})
        x = want[0] >> 1
        lo, hi = np.searchsorted(self.by_var, [x, x + 1])
        for g in np.unique(self.ng_of[lo:hi]):
            if sorted(set(self.enc[self.off[g]:self.off[g + 1]].tolist())) == want:
                return True
        return False


@pytest.fixture(scope="module")
def large(gpu):
    prog = large_random_program(0)
    return prog, _Completion(prog)


def _closure_case(gpu, prog, comp, P, k, seed):
    """Root closure plus k open atoms set at random, propagated by the GPU and
    by the oracle; returns whether the oracle saw a conflict."""
    nv = P.n_vars
    zero = np.zeros(nv, np.int8)
    _, root = P.propagate(zero)
    rng = np.random.default_rng(seed)
    open_atoms = np.nonzero(root[:prog.n_atoms] == 0)[0]
    pick = rng.choice(open_atoms, size=k, replace=False)
    partial = root.copy()
    partial[pick] = rng.choice(np.array([-1, 1], np.int8), size=k)
    conflict, clo = P.propagate(partial)
    opart = partial[comp.o2g]              # oracle variable i is library variable o2g[i]
    oconf, oclo, _, _ = oracle.up_closure(prog, opart)
    assert conflict == oconf, (k, seed)
    if not oconf:
        lib_from_oracle = np.zeros(nv, np.int8)
        lib_from_oracle[comp.o2g] = oclo
        diff = np.nonzero(clo != lib_from_oracle)[0]
        assert diff.shape[0] == 0, (k, seed, diff[:10])
        assert (clo != 0).sum() > (root != 0).sum()
    return oconf


@pytest.mark.parametrize("k,seed", [(1, 0), (4, 1), (16, 2), (64, 3), (64, 4), (256, 5), (1024, 6)])
def test_closure_of_deep_partial_assignments_100k(gpu, large, k, seed):
    prog, comp = large
    P = gpu.Program(prog)
    _closure_case(gpu, prog, comp, P, k, seed)
    P.close()


def test_closure_of_deep_partial_assignments_store_larger_than_l2(gpu):
    """400k atoms, 1.6M rules (126 MB store, packed views): the store streams
    from DRAM on every sweep."""
    prog = large_random_program(0, n_atoms=400_000, n_rules=1_600_000)
    comp = _Completion(prog)
    P = gpu.Program(prog)
    outcomes = [_closure_case(gpu, prog, comp, P, k, 10 + k) for k in (2, 32)]
    assert not all(outcomes)
    P.close()


def _deps_levels(row, L):
    """Levels of the dependency bitmap of a variable at level L (bit j-1
    stands for level j).  Only the first ceil(L / 64) words of a row are
    written when the variable is assigned; the words after them are left
    from earlier use of the memory and are not read."""
    out = set()
    for w, word in enumerate(row[:(int(L) + 63) // 64].tolist()):
        while word:
            b = (word & -word).bit_length() - 1
            word &= word - 1
            out.add(64 * w + b + 1)
    return frozenset(out)


def _check_fwd_conflict(gpu, P, comp, k, asserting=False):
    """The cone of the last conflict's violated nogood, reason by reason, and
    the learned nogood and target of Algorithm 4 from it (see the module
    docstring); returns (cone size, learned length, target)."""
    s = P.stats()
    lc = P.last_conflict()
    assert lc is not None and "learned" in lc
    words = (int(s["max_level"]) + 63) // 64 + 1
    st = P.state(deps_words=words)
    level, reason, deps = st["level"], st["reason"], st["deps"]
    nv = P.n_vars
    # values on the trail up to the conflict: -1 open, 0 true, 1 false
    val = np.full(nv, -1, np.int8)
    tl = lc["trail"].astype(np.int64)
    tv = tl >> 1
    assert np.unique(tv).shape[0] == tv.shape[0], "a variable twice on the trail"
    val[tv] = (tl & 1).astype(np.int8)
    dec = {}
    for v in tv[reason[tv] == gpu.R_DECISION].tolist():
        L = int(level[v])
        assert L not in dec, f"two decisions at level {L}"
        dec[L] = v
    learned = {int(i) for i in P.learned_ids()}

    def holds(l):
        return val[l >> 1] == (l & 1)

    # the cone of the violated nogood, checked variable by variable
    g = [int(l) for l in P.nogood(lc["conflict"])]
    assert comp.contains(g) or lc["conflict"] in learned
    assert all(holds(l) for l in g), "a literal of the violated nogood does not hold"
    todo = [l >> 1 for l in g if level[l >> 1] > 1]
    seen = set(todo)
    checked = 0
    while todo and checked < CONE_CAP:
        v = todo.pop()
        L = int(level[v])
        r = int(reason[v])
        have = _deps_levels(deps[v], L)
        checked += 1
        if r == gpu.R_DECISION:
            assert have == {L}, (v, L, sorted(have))
            continue
        if r == gpu.R_COMPLETE:
            assert have == frozenset(range(2, L + 1)), (v, L)
            continue
        ng = [int(l) for l in P.nogood(r)]
        assert comp.contains(ng) or r in learned, f"reason {r} of {v} is neither completion nor learned"
        mine = [l for l in ng if l >> 1 == v]
        assert mine == [(v << 1) | (1 - int(val[v]))], (v, r, ng)
        want = set()
        for l in ng:
            u = l >> 1
            if u == v:
                continue
            assert holds(l), (v, r, l)
            if level[u] > 1:
                want |= _deps_levels(deps[u], level[u])
                if u not in seen:
                    seen.add(u)
                    todo.append(u)
        assert have == want, (v, L, sorted(have ^ want)[:10])
    assert not todo, f"cone larger than {CONE_CAP} variables"
    # the learned nogood (Algorithm 4) and the backjump target
    levels = set()
    for l in g:
        if level[l >> 1] > 1:
            levels |= _deps_levels(deps[l >> 1], level[l >> 1])
    assert levels
    h = max(levels)
    got = [int(l) for l in P.nogood(lc["learned"])]
    assert len(got) == lc["length"] == len(set(got))
    assert set(got) == {dec[L] << 1 for L in levels}
    if asserting:
        below = sorted(L for L in levels if L < h)
        assert lc["target"] == (below[-1] if below else 1)
    else:
        assert lc["target"] == h - 1
    # unit at the target: only the decision of level h is above it
    at_h = [l for l in got if level[l >> 1] > lc["target"]]
    assert at_h == [dec[h] << 1]
    return checked, len(got), lc["target"]


# (conflict k, options): the benchmark's defaults, then the unit frontier
# (the fastest propagation-round mode of the benchmark's comparison, also on
# 76 CTAs), the asserting-level backjump, and the Jeroslow-Wang and
# decaying-activity decision scores
FWD_CASES = [(1, {}), (3, {}), (8, {}), (25, {}),
             (4, {"frontier": 2}), (15, {"frontier": 2}), (7, {"frontier": 2, "grid_ctas": 76}),
             (6, {"backjump": 1}),
             (5, {"heuristic": 4}), (9, {"heuristic": 5})]


@pytest.mark.parametrize("k,opts", FWD_CASES, ids=[f"k{k}-{'-'.join(f'{a}{b}' for a, b in o.items()) or 'default'}"
                                                   for k, o in FWD_CASES])
def test_fwd_learning_at_full_size(gpu, large, k, opts):
    prog, comp = large
    P = gpu.Program(prog, conflict_budget=k, time_budget_ms=60_000, **opts)
    status, _, _ = P.solve(1, cap=1)
    if status != gpu.UNKNOWN or P.stats()["conflicts"] != k:
        pytest.skip("search ended before the k-th conflict")
    cone, n, target = _check_fwd_conflict(gpu, P, comp, k, asserting=opts.get("backjump") == 1)
    print(f"fwd k={k} {opts}: cone of {cone} variables, learned nogood of {n} decisions, target {target}")
    P.close()


@pytest.mark.parametrize("k", [1, 4, 12])
def test_resolution_learning_at_full_size(gpu, large, k):
    """First-UIP resolution learning (Algorithm 3, the paper's baseline
    analysis) at the k-th conflict of the benchmark's search: the learned
    nogood, its first literal and the target equal the oracle's first_uip run
    on the GPU's own state (trail order, levels, reasons, violated nogood);
    the GPU leaves root-level literals out of the nogood."""
    prog, comp = large
    P = gpu.Program(prog, learning=gpu.LEARN_RES, conflict_budget=k, time_budget_ms=60_000)
    status, _, _ = P.solve(1, cap=1)
    if status != gpu.UNKNOWN or P.stats()["conflicts"] != k:
        pytest.skip("search ended before the k-th conflict")
    lc = P.last_conflict()
    assert lc is not None and "learned" in lc
    st = P.state()
    level, reason = st["level"], st["reason"]
    tl = lc["trail"].astype(np.int64)
    tv = tl >> 1
    pos = np.full(P.n_vars, -1, np.int64)
    pos[tv] = np.arange(tv.shape[0])
    is_false = np.zeros(P.n_vars, bool)
    is_false[tv] = (tl & 1) == 1
    dec = {int(level[v]): int(v) for v in tv[reason[tv] == gpu.R_DECISION].tolist()}
    learned_ids = {int(i) for i in P.learned_ids()}

    def lits(arr):
        return [(int(l) >> 1, bool(int(l) & 1)) for l in arr]

    def antecedent(v):
        r = int(reason[v])
        if r == gpu.R_DECISION:
            return None
        if r == gpu.R_COMPLETE:
            return [(v, not bool(is_false[v]))] + [(dec[L], False) for L in range(2, int(level[v]) + 1)]
        ng = P.nogood(r)
        assert comp.contains(ng) or r in learned_ids, f"reason {r} of {v} is neither completion nor learned"
        return lits(ng)

    delta = lits(P.nogood(lc["conflict"]))
    d, kappa, uip = oracle.first_uip(delta, pos, level, antecedent)
    got = lits(P.nogood(lc["learned"]))
    assert len(got) == lc["length"] == len(set(got))
    assert got[0] == uip
    assert set(got) == {l for l in d if level[l[0]] > 1}
    assert lc["target"] == max(kappa, 1)
    print(f"res k={k}: learned nogood of {len(got)} literals, target {lc['target']}")
    P.close()
