"""Pins of the oracle's first-UIP analysis (Section 4.2, Algorithm 3),
independent of the GPU path: a conflict resolved by hand, and conflicts of
a small sequential solver over the oracle's completion nogoods, where the
learned nogood must (a) hold under the assignment, (b) have exactly one
literal at the conflict level, the first UIP, which must be the dominator of
the conflict in the implication graph closest to it (the textbook definition
of the first UIP), and (c) be violated by no supported model of the program
(brute force over atom assignments)."""
import json
import os

import numpy as np
import pytest

import oracle
from synth.programs import tiny_program

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_hand_example():
    with open(os.path.join(GOLDEN, "first_uip_example.json")) as f:
        ex = json.load(f)
    pos = {v: i for i, v in enumerate(ex["trail"])}
    ante = {v: [tuple(l) for l in lits] for v, lits in ex["antecedent"].items()}
    d, kappa, uip = oracle.first_uip([tuple(l) for l in ex["conflict"]], pos, ex["level"], lambda v: ante.get(v))
    assert d == {tuple(l) for l in ex["learned"]}
    assert kappa == ex["kappa"] and uip == tuple(ex["uip"])


def test_decision_sharing_a_level_is_an_error():
    # the decision is assigned last at its level only if the state is broken
    pos = {"c": 1, "d": 0}
    with pytest.raises(ValueError):
        oracle.first_uip([("c", False), ("d", False)], pos, {"c": 4, "d": 4}, lambda v: None)


class _Solver:
    """Sequential unit propagation over the oracle's completion nogoods with
    trail positions, levels and antecedents (test scaffolding)."""

    def __init__(self, prog):
        self.nv, off, lits = oracle.completion(prog)
        self.ng = [[(abs(int(l)) - 1, int(l) < 0) for l in lits[off[i]:off[i + 1]]] for i in range(len(off) - 1)]
        self.val = np.zeros(self.nv, np.int8)     # 1 true, -1 false
        self.level = np.zeros(self.nv, np.int64)
        self.pos = np.full(self.nv, -1, np.int64)
        self.ante = [None] * self.nv
        self.trail = []
        self.cdl = 1

    def holds(self, lit):
        v, f = lit
        return self.val[v] == (-1 if f else 1)

    def assign(self, lit_true, ante):
        v, f = lit_true
        self.val[v] = -1 if f else 1
        self.level[v] = self.cdl
        self.pos[v] = len(self.trail)
        self.ante[v] = ante
        self.trail.append(v)

    def propagate(self):
        """Returns a violated nogood index or None at fixpoint."""
        changed = True
        while changed:
            changed = False
            for i, g in enumerate(self.ng):
                open_ = [l for l in g if self.val[l[0]] == 0]
                if any(self.val[l[0]] != 0 and not self.holds(l) for l in g):
                    continue
                if not open_:
                    return i
                if len(open_) == 1:
                    v, f = open_[0]
                    self.assign((v, not f), i)
                    changed = True
        return None

    def backjump(self, k):
        while self.trail and self.level[self.trail[-1]] > k:
            v = self.trail.pop()
            self.val[v] = 0
            self.level[v] = 0
            self.pos[v] = -1
            self.ante[v] = None
        self.cdl = k


def _dominators(S, m, conflict_vars):
    """Level-m variables every path from a level-m source (a variable with no
    level-m antecedent literal) to the conflict passes through."""
    nodes = [v for v in S.trail if S.level[v] == m]
    preds = {}
    for v in nodes:
        a = S.ante[v]
        preds[v] = [] if a is None else [u for (u, _) in S.ng[a] if u != v and S.level[u] == m]
    sources = {v for v in nodes if not preds[v]}
    dom = []
    for u in nodes:
        seen, stack, hit = set(), [w for w in conflict_vars if w != u], False
        while stack:
            w = stack.pop()
            if w in seen:
                continue
            seen.add(w)
            if w in sources:
                hit = True
                break
            stack.extend(x for x in preds[w] if x != u)
        if not hit:
            dom.append(u)
    return dom


def _wave_first_uip(delta, pos, level, ng, ante, w):
    """Resolution in waves: with cnt literals of the conflict level marked,
    resolve the min(cnt - 1, w) highest at once (their reasons' literals
    join; a variable is taken once); stop at one marked literal."""
    m = max(level[v] for (v, _) in delta)
    seen, marked, low = set(), {}, set()

    def add(lits, skip):
        for (v, f) in lits:
            if v == skip or v in seen or level[v] <= 0:
                continue
            seen.add(v)
            if level[v] == m:
                marked[v] = (v, f)
            else:
                low.add((v, f))

    add(delta, None)
    while len(marked) > 1:
        top = sorted(marked, key=lambda v: -pos[v])[:min(len(marked) - 1, w)]
        for v in top:
            del marked[v]
        for v in top:
            add(ng[ante[v]], v)
    (uip,) = marked.values()
    kappa = max([level[v] for (v, _) in low] + [0])
    return low | {uip}, kappa, uip


def _another_order(S, rng):
    """Trail positions of a random topological order of the implication
    graph, level by level."""
    depth = {}
    for v in S.trail:                                   # antecedents come first
        a = S.ante[v]
        ps = [] if a is None else [u for (u, _) in S.ng[a] if u != v and S.level[u] == S.level[v]]
        depth[v] = 1 + max([depth[u] for u in ps], default=-1)
    key = {v: (int(S.level[v]), depth[v], float(rng.random())) for v in S.trail}
    pos = np.full(S.nv, -1, np.int64)
    for i, v in enumerate(sorted(S.trail, key=lambda v: key[v])):
        pos[v] = i
    return pos


def _supported_models(prog, nv):
    na = prog.n_atoms
    out = []
    for mask in range(1 << na):
        part = np.zeros(nv, np.int8)
        part[:na] = [1 if (mask >> i) & 1 else -1 for i in range(na)]
        conf, clo, _, _ = oracle.up_closure(prog, part)
        if not conf and (clo != 0).all():
            out.append(clo)
    return out


@pytest.mark.parametrize("index", range(0, 300, 3))
def test_learned_nogoods_of_a_sequential_search(index):
    prog = tiny_program(index, n_atoms=9, n_rules=18, n_constraints=2)
    if _Solver(prog).propagate() is not None:
        return
    models = _supported_models(prog, _Solver(prog).nv)
    for run in range(4):
        _search(prog, models, np.random.default_rng(1000 * index + run))


def _search(prog, models, rng):
    S = _Solver(prog)
    S.propagate()
    analysed = 0
    while analysed < 6:
        free = [v for v in range(S.nv) if S.val[v] == 0]
        if not free:
            break
        S.cdl += 1
        v = int(rng.choice(free))
        S.assign((v, bool(rng.integers(2))), None)
        g = S.propagate()
        while g is not None:
            m = max(int(S.level[u]) for (u, _) in S.ng[g])
            if m <= 1:
                return
            if m < S.cdl:
                S.backjump(m)
            d, kappa, uip = oracle.first_uip(S.ng[g], S.pos, S.level,
                                            lambda u: None if S.ante[u] is None else S.ng[S.ante[u]])
            analysed += 1
            # (a) the learned nogood holds under the assignment
            assert all(S.holds(l) for l in d)
            # (b) one literal at the conflict level, the closest dominator
            at_m = [l for l in d if S.level[l[0]] == m]
            assert at_m == [uip] and kappa < m
            assert kappa == max([int(S.level[u]) for (u, _) in d if (u, _) != uip] + [0])
            dom = _dominators(S, m, [u for (u, _) in S.ng[g] if S.level[u] == m])
            assert uip[0] == max(dom, key=lambda u: S.pos[u])
            # (d) the same result under another trail order that respects
            # the implication graph (concurrent claims may land in any such
            # order): levels first, then depth below the level's sources,
            # random among equals
            d2, k2, u2 = oracle.first_uip(S.ng[g], _another_order(S, rng), S.level,
                                          lambda u: None if S.ante[u] is None else S.ng[S.ante[u]])
            assert (d2, k2, u2) == (d, kappa, uip)
            # (e) resolving up to w of the highest marked literals at once,
            # never the lowest, reaches the same nogood
            for w in (2, 5, 32):
                assert _wave_first_uip(S.ng[g], S.pos, S.level, S.ng, S.ante, w) == (d, kappa, uip)
            # (c) no supported model violates it
            for M in models:
                assert not all(M[u] == (-1 if f else 1) for (u, f) in d)
            # learn, backjump, assert the complement of the UIP
            S.ng.append(sorted(d))
            S.backjump(max(kappa, 1))
            S.assign((uip[0], not uip[1]), len(S.ng) - 1)
            g = S.propagate()
            if g is not None and max(int(S.level[u]) for (u, _) in S.ng[g]) <= 1:
                return
