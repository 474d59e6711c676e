"""fwd-learning (Section 4.2, Algorithm 4) pinned as a function (needs a GB300).

At the k-th conflict of a search -- the solve stops on its conflict budget
right after the analysis, before the backjump -- the dependency bitmaps and
the learned nogood are recomputed on the CPU from the search state:

- every reason the search recorded is a nogood of the oracle's own
  completion (its variables mapped to the library's numbering) or a nogood
  the search learned earlier, and it was unit: its other literals hold and
  its literal on the assigned variable is the complement of the assignment;
- Deps[x] = OR of Deps[u] over the reason's other variables u with level > 1
  (mk_dl_bitmap); a decision at level L depends on L alone; an atom set false
  by CompleteAssignment on every level 2..L (the reading for atoms without a
  reason);
- the learned nogood is the decision literals of the levels in
  OR(Deps[u] : u in the violated nogood, level > 1) (when two claims clashed
  on a variable, the trail holds the first, and its Deps brings in the
  clashing reason);
- the backjump target is h-1 for the highest of those levels h, or the second
  highest (1 if none) under the asserting option, and the learned nogood is
  then unit at the target.

Brute-force pins on small programs: no answer set violates a nogood that was
learned before it was found."""
import json
import os

import numpy as np
import pytest

import oracle
from synth.programs import coloring_program, program_seed, random_program, tiny_program

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1909_01786_gb300 import aspgpu
    aspgpu.lib()
    return aspgpu


def _gpu_rule_order(prog):
    """Input index of the library's rule j (headed rules sorted by head atom,
    ties in input order), as the header documents."""
    headed = np.nonzero(prog.head >= 0)[0]
    return headed[np.argsort(prog.head[headed], kind="stable")]


def _oracle_nogoods_in_gpu_vars(prog):
    """The oracle's completion nogoods as frozensets of (variable, is_false)
    in the library's variable numbering (both put b, t, n of rule j at
    n_atoms + 3j + 0/1/2; the rule numbering differs)."""
    nv, off, lits = oracle.completion(prog)
    na = prog.n_atoms
    order = _gpu_rule_order(prog)
    headed = np.nonzero(prog.head >= 0)[0]
    ordinal = {int(r): i for i, r in enumerate(headed)}      # input rule -> oracle rule ordinal
    o2g = np.arange(nv)
    for j, r_in in enumerate(order):
        oj = ordinal[int(r_in)]
        for q in range(3):
            o2g[na + 3 * oj + q] = na + 3 * j + q
    out = set()
    for i in range(off.shape[0] - 1):
        ng = frozenset((int(o2g[abs(int(l)) - 1]), int(l) < 0) for l in lits[off[i]:off[i + 1]])
        out.add(ng)
    return out


def _lits(arr):
    return [(int(l) >> 1, bool(int(l) & 1)) for l in arr]


class _Recompute:
    """The search state at the last conflict, and Deps recomputed from it."""

    def __init__(self, gpu, P, prog, completion):
        self.gpu, self.P = gpu, P
        lc = P.last_conflict()
        assert lc is not None and "learned" in lc
        self.lc = lc
        st = P.state()
        self.level, self.reason = st["level"], st["reason"]
        self.trail = _lits(lc["trail"])
        self.value = {}                      # var -> is_false
        self.pos = {}
        for i, (v, f) in enumerate(self.trail):
            assert v not in self.value, f"variable {v} twice on the trail"
            self.value[v] = f
            self.pos[v] = i
        self.dec = {}
        for v, _ in self.trail:
            if self.reason[v] == gpu.R_DECISION:
                L = int(self.level[v])
                assert L not in self.dec, f"two decisions at level {L}"
                self.dec[L] = v
        self.learned = {int(i) for i in P.learned_ids()}
        self.completion = completion
        self._cache = {}
        self._ng = {}
        self.reasons_checked = 0

    def nogood(self, nid):
        if nid not in self._ng:
            self._ng[nid] = _lits(self.P.nogood(nid))
        return self._ng[nid]

    def holds(self, lit):
        v, f = lit
        return v in self.value and self.value[v] == f

    def check_reason(self, x):
        """x's reason: a completion or learned nogood, unit on x."""
        r = int(self.reason[x])
        ng = self.nogood(r)
        s = frozenset(ng)
        assert s in self.completion or r in self.learned, f"reason {r} of {x} is neither completion nor learned"
        mine = [l for l in ng if l[0] == x]
        assert mine == [(x, not self.value[x])], (x, r, ng)
        for l in ng:
            if l[0] != x:
                assert self.holds(l), (x, r, l)
        self.reasons_checked += 1
        return ng

    def deps(self, x):
        """Deps[x] as a set of levels >= 2 (explicit stack, reasons first)."""
        if x in self._cache:
            return self._cache[x]
        stack = [(x, False)]
        on = set()
        while stack:
            v, ready = stack.pop()
            if v in self._cache:
                continue
            L = int(self.level[v])
            r = int(self.reason[v])
            if L <= 1:
                self._cache[v] = frozenset()
                continue
            if r == self.gpu.R_DECISION:
                self._cache[v] = frozenset([L])
                continue
            if r == self.gpu.R_COMPLETE:
                self._cache[v] = frozenset(range(2, L + 1))
                continue
            ng = self.check_reason(v) if not ready else self.nogood(r)
            others = [u for (u, _) in ng if u != v and int(self.level[u]) > 1]
            if not ready:
                assert v not in on, f"cyclic reasons at {v}"
                on.add(v)
                stack.append((v, True))
                stack.extend((u, False) for u in others if u not in self._cache)
                continue
            acc = set()
            for u in others:
                acc |= self._cache[u]
            self._cache[v] = frozenset(acc)
        return self._cache[x]


def _conflict_levels(R):
    """Levels of the learned nogood by Algorithm 4's reading: the OR of Deps
    over the violated nogood.  When two claims clashed on a variable c, the
    trail holds the first claim, under which every literal of the nogood
    holds, and Deps[c] is the OR over c's reason: the union is the OR over
    the nogood and the reason of the clash, as the analysis takes it."""
    g = R.nogood(R.lc["conflict"])
    assert frozenset(g) in R.completion or R.lc["conflict"] in R.learned
    acc = set()
    for (u, f) in g:
        assert R.holds((u, f)), ("a literal of the violated nogood does not hold", u, f)
        if int(R.level[u]) > 1:
            acc |= R.deps(u)
    return acc, g


def _check_at_conflict(gpu, P, prog, completion, mode, deps_words=64):
    R = _Recompute(gpu, P, prog, completion)
    levels, g = _conflict_levels(R)
    assert levels, "the analysed conflict involves no decision level"
    h = max(levels)
    want = {(R.dec[L], False) for L in levels}
    got = _lits(P.nogood(R.lc["learned"]))
    assert len(got) == R.lc["length"] == len(set(got))
    assert set(got) == want
    if mode == gpu.BACKJUMP_H_MINUS_1:
        assert R.lc["target"] == h - 1
    else:
        below = sorted(L for L in levels if L < h)
        assert R.lc["target"] == (below[-1] if below else 1)
    # unit at the target: every literal but the decision of level h holds
    # there, and that one is unassigned after the backjump
    t = R.lc["target"]
    at_h = [(v, f) for (v, f) in got if int(R.level[v]) > t]
    assert at_h == [(R.dec[h], False)]
    # Deps of every assigned variable above the root equal the recomputation
    st = P.state(deps_words=deps_words)
    deps = st["deps"]
    compared = 0
    for v, _ in R.trail:
        L = int(R.level[v])
        if L <= 1:
            continue
        nw = min(deps_words, (L + 63) // 64)
        have = set()
        for w in range(nw):
            word = int(deps[v, w])
            while word:
                b = (word & -word).bit_length() - 1
                word &= word - 1
                have.add(64 * w + b + 1)
        assert have == set(R.deps(v)), (v, L, sorted(have), sorted(R.deps(v)))
        compared += 1
    return compared, R.reasons_checked


CASES = [(300, 900, 0), (800, 2000, 1), (2000, 5000, 2), (5000, 12000, 3)]


@pytest.mark.parametrize("atoms,rules,seed", CASES)
@pytest.mark.parametrize("k", [1, 2, 4, 9, 23])
@pytest.mark.parametrize("mode", [0, 1])
def test_fwd_learned_nogood_recomputed(gpu, atoms, rules, seed, k, mode):
    prog = random_program(atoms, rules, program_seed(705, seed))
    P = gpu.Program(prog, backjump=mode, conflict_budget=k, time_budget_ms=60_000)
    status, _, _ = P.solve(1, cap=1)
    s = P.stats()
    if status != gpu.UNKNOWN or s["conflicts"] != k:
        pytest.skip("search ended before the k-th conflict")
    compared, reasons = _check_at_conflict(gpu, P, prog, _completion(prog), mode)
    assert compared > 0 and reasons > 0


@pytest.mark.parametrize("grid", [1, 5, 0])
@pytest.mark.parametrize("k", [3, 11])
@pytest.mark.parametrize("fr", [0, 1, 2, 3])
def test_fwd_learned_nogood_recomputed_grids_and_frontiers(gpu, grid, k, fr):
    prog = random_program(2000, 5000, program_seed(705, 2))
    P = gpu.Program(prog, conflict_budget=k, grid_ctas=grid, frontier=fr, time_budget_ms=60_000)
    status, _, _ = P.solve(1, cap=1)
    if status != gpu.UNKNOWN or P.stats()["conflicts"] != k:
        pytest.skip("search ended before the k-th conflict")
    _check_at_conflict(gpu, P, prog, _completion(prog), 0)


@pytest.mark.parametrize("k", [2, 7, 19])
def test_fwd_learned_nogood_recomputed_colouring(gpu, k):
    """Colouring programs reach loop nogoods and models less often; their
    conflicts come from the edge constraints."""
    prog = coloring_program(300, 4.5, seed_index=3)
    P = gpu.Program(prog, conflict_budget=k, time_budget_ms=60_000)
    status, _, _ = P.solve(1, cap=1)
    if status != gpu.UNKNOWN or P.stats()["conflicts"] != k:
        pytest.skip("search ended before the k-th conflict")
    _check_at_conflict(gpu, P, prog, _completion(prog), 0)


def _completion(prog):
    return _oracle_nogoods_in_gpu_vars(prog)


# ------------------------------------------------------------ brute force

def _extend(prog, M):
    """The total assignment of an interpretation M over the library's
    variables: atoms from M; b_j = body of rule j holds, t_j = its positive
    body holds, n_j = none of its negative body holds (the completion's
    definitions of the auxiliary atoms, Section 2)."""
    order = _gpu_rule_order(prog)
    na = prog.n_atoms
    X = np.zeros(na + 3 * order.shape[0], bool)
    X[:na] = np.asarray(M, bool)
    for j, r in enumerate(order):
        pos = prog.pos[prog.pos_off[r]:prog.pos_off[r + 1]]
        neg = prog.neg[prog.neg_off[r]:prog.neg_off[r + 1]]
        t = bool(X[pos].all()) if pos.size else True
        n = not bool(X[neg].any()) if neg.size else True
        X[na + 3 * j] = t and n
        X[na + 3 * j + 1] = t
        X[na + 3 * j + 2] = n
    return X


def _violated(ng, X):
    return all(X[v] == (not f) for (v, f) in ng)


def _answer_sets_golden():
    data = json.load(open(os.path.join(GOLDEN, "tiny_answer_sets.json")))
    return {r["index"]: r["answer_sets"] for r in data["programs"]}


def _masks_to_rows(masks, n):
    return [np.array([(m >> a) & 1 for a in range(n)], np.uint8) for m in masks]


def _learned_sound(gpu, prog, all_sets, max_first=4, **kw):
    """Runs with max_models = 1..max_first: every nogood learned in the run
    before the i-th model is violated by no answer set other than the i-1
    models found before it.  Returns the number of nogoods checked."""
    ext = [(_extend(prog, M), frozenset(np.nonzero(M)[0].tolist())) for M in all_sets]
    checked = 0
    for i in range(1, min(max_first, len(all_sets)) + 1):
        P = gpu.Program(prog, **kw)
        status, models, n = P.solve(i, cap=i)
        assert status == gpu.SAT and n == i
        found = [frozenset(np.nonzero(m)[0].tolist()) for m in models]
        earlier = set(found[:-1])
        for nid in P.learned_ids():
            ng = _lits(P.nogood(int(nid)))
            for X, key in ext:
                if key in earlier:
                    continue
                assert not _violated(ng, X), (i, int(nid), ng, sorted(key))
            checked += 1
        P.close()
    return checked


def test_learned_nogoods_violate_no_answer_set_tiny(gpu):
    """Every tiny program with an answer set (brute force over 2^20, stored):
    fwd-learning, both backjump targets."""
    golden = _answer_sets_golden()
    picked = [i for i in sorted(golden) if golden[i]]
    assert len(picked) >= 200
    checked = 0
    for i in picked:
        prog = tiny_program(i)
        sets = _masks_to_rows(golden[i], prog.n_atoms)
        for mode in (0, 1):
            checked += _learned_sound(gpu, prog, sets, backjump=mode)
    assert checked >= 100, checked


def test_learned_nogoods_violate_no_answer_set_denser_tiny(gpu):
    """20 atoms, 60 rules, 4 constraints: more conflicts before each model
    (brute force over 2^20 in the test)."""
    checked = runs = 0
    for i in range(40):
        prog = tiny_program(5000 + i, n_rules=60, n_constraints=4)
        sets = list(oracle.brute_force(prog))
        if not sets:
            continue
        runs += 1
        for mode in (0, 1):
            checked += _learned_sound(gpu, prog, sets, backjump=mode)
    assert runs >= 4 and checked > 0, (runs, checked)


def _sat_colourings(n, count):
    out = []
    for seed in range(40):
        prog = coloring_program(n, 3.0, seed_index=seed)
        ost, om, _ = oracle.cdnl(prog, time_budget_s=60)
        assert ost in (oracle.SAT, oracle.UNSAT)
        if ost == oracle.SAT:
            out.append((prog, list(om)))
        if len(out) == count:
            break
    return out


@pytest.mark.parametrize("n", [8, 10])
def test_learned_nogoods_violate_no_answer_set_colouring(gpu, n):
    """Small 3-colourings (the first three seeds with a colouring), every
    answer set by the oracle's CDNL enumeration (itself pinned against brute
    force): conflicts and blocking nogoods mix."""
    cases = _sat_colourings(n, 3)
    assert len(cases) == 3
    checked = 0
    for prog, om in cases:
        checked += _learned_sound(gpu, prog, om, max_first=6)
    assert checked > 0
