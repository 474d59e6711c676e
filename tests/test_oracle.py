"""Pins for the CPU oracle (no GPU).

Each check compares the oracle against something other than itself: hand
results, the subset-minimal-model definition by subset enumeration, the
supported-model characterisation of the completion, brute force over total
assignments, closed-form counts, or invariants of the semantics.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from synth.programs import from_rules, random_program, tiny_program, program_seed

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _named_program(atoms, rules):
    idx = {a: i for i, a in enumerate(atoms)}
    return from_rules(len(atoms), [(-1 if h is None else idx[h], [idx[a] for a in p], [idx[a] for a in n])
                                   for h, p, n in rules])


def _as_sets(models, atoms=None):
    out = set()
    for m in models:
        s = frozenset(int(i) for i in np.nonzero(m)[0])
        out.add(s if atoms is None else frozenset(atoms[i] for i in s))
    return out


# ------------------------------------------------------------- hand cases

HAND = json.load(open(os.path.join(GOLDEN, "hand_cases.json")))["cases"]


@pytest.mark.parametrize("case", HAND, ids=[c["name"] for c in HAND])
def test_hand_cases_brute_force(case):
    prog = _named_program(case["atoms"], case["rules"])
    got = _as_sets(oracle.brute_force(prog), case["atoms"])
    assert got == {frozenset(s) for s in case["answer_sets"]}


@pytest.mark.parametrize("case", HAND, ids=[c["name"] for c in HAND])
def test_hand_cases_cdnl(case):
    prog = _named_program(case["atoms"], case["rules"])
    status, models, _ = oracle.cdnl(prog)
    want = {frozenset(s) for s in case["answer_sets"]}
    assert _as_sets(models, case["atoms"]) == want
    assert len(models) == len(want)
    assert status == (oracle.SAT if want else oracle.UNSAT)


# ------------------------------------- reduct definition by subset search

def _minimal_model_of_reduct(prog, M):
    """Paper's definition taken literally: M is an answer set iff M is a
    model of every constraint and M is a subset-minimal model of the reduct
    (rules with body- meeting M dropped, body- deleted from the rest)."""
    rules = list(prog.rules())
    Ms = set(np.nonzero(M)[0].tolist())
    reduct = [(h, set(p)) for h, p, n in rules if h >= 0 and not (set(n) & Ms)]

    def is_model(I):
        return all(h in I or not p <= I for h, p in reduct)

    for h, p, n in rules:
        if h < 0 and set(p) <= Ms and not (set(n) & Ms):
            return False
    if not is_model(Ms):
        return False
    lst = sorted(Ms)
    for k in range(len(lst)):
        for sub in itertools.combinations(lst, k):
            if is_model(set(sub)):
                return False
    return True


@pytest.mark.parametrize("seed", range(40))
def test_is_answer_set_matches_minimal_model_definition(seed):
    prog = random_program(6, 7 + seed % 5, program_seed(101, seed))
    for mask in range(1 << prog.n_atoms):
        M = np.array([(mask >> i) & 1 for i in range(prog.n_atoms)], dtype=np.uint8)
        assert oracle.is_answer_set(prog, M) == _minimal_model_of_reduct(prog, M), mask


def test_least_model_of_definite_chain():
    # a. b <- a. c <- b. d <- e.   LM = {a,b,c}
    prog = from_rules(5, [(0, [], []), (1, [0], []), (2, [1], []), (3, [4], [])])
    lm = oracle.least_model_of_reduct(prog, np.zeros(5, np.uint8))
    assert lm.tolist() == [1, 1, 1, 0, 0]


# ------------------------------------------------ enumeration invariants

@pytest.mark.parametrize("seed", range(60))
def test_cdnl_equals_brute_force_small(seed):
    prog = random_program(9, 8 + seed % 10, program_seed(102, seed))
    bf = _as_sets(oracle.brute_force(prog))
    status, models, _ = oracle.cdnl(prog)
    assert _as_sets(models) == bf
    assert len(models) == len(bf)          # no duplicates
    assert status == (oracle.SAT if bf else oracle.UNSAT)


@pytest.mark.parametrize("index", list(range(6)) + list(range(100, 2400, 100)))
def test_cdnl_equals_brute_force_tiny_config(index):
    prog = tiny_program(index)
    bf = _as_sets(oracle.brute_force(prog))
    _, models, _ = oracle.cdnl(prog)
    assert _as_sets(models) == bf and len(models) == len(bf)


@pytest.mark.parametrize("seed", range(20))
def test_answer_sets_form_an_antichain(seed):
    prog = random_program(10, 12, program_seed(103, seed))
    sets = list(_as_sets(oracle.brute_force(prog)))
    for a in sets:
        for b in sets:
            assert not (a < b)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_max_models_returns_that_many_distinct(k):
    # four independent even loops: 16 answer sets
    rules = []
    for i in range(4):
        rules += [(2 * i, [], [2 * i + 1]), (2 * i + 1, [], [2 * i])]
    prog = from_rules(8, rules)
    status, models, _ = oracle.cdnl(prog, max_models=k)
    assert status == oracle.SAT and len(models) == k and len(_as_sets(models)) == k
    assert all(oracle.is_answer_set(prog, m) for m in models)
    _, allm, _ = oracle.cdnl(prog)
    assert len(allm) == 16


# ------------------------------------------------------------ completion

def _names(prog_atoms, n_atoms, head):
    """Oracle variable index -> name (atoms, then b/t/n of headed rules)."""
    names = list(prog_atoms)
    j = 0
    for h in head:
        if h >= 0:
            names += [f"b_r{j}", f"t_r{j}", f"n_r{j}"]
            j += 1
    return names


def test_completion_golden_listing():
    g = json.load(open(os.path.join(GOLDEN, "completion_three_rules.json")))
    prog = _named_program(g["atoms"], g["rules"])
    nv, off, lits = oracle.completion(prog)
    names = _names(g["atoms"], prog.n_atoms, prog.head)
    assert nv == len(names)
    got = sorted(sorted(("T" if l > 0 else "F") + names[abs(l) - 1] for l in lits[off[i]:off[i + 1]])
                 for i in range(off.shape[0] - 1))
    want = sorted(sorted(x) for x in g["nogoods"])
    assert got == want


@pytest.mark.parametrize("seed", range(10))
def test_completion_closed_form_counts(seed):
    prog = random_program(50, 200, program_seed(104, seed))
    nv, off, lits = oracle.completion(prog)
    lens = np.diff(off)
    # per rule with k body atoms: 6 + k nogoods, 11 + 3k literals;
    # per atom one nogood of 1 + |rules(p)| literals
    k = np.diff(prog.pos_off) + np.diff(prog.neg_off)
    nr = prog.n_rules
    assert nv == prog.n_atoms + 3 * nr
    assert lens.shape[0] == int((6 + k).sum()) + prog.n_atoms
    assert lens.sum() == int((11 + 3 * k).sum()) + prog.n_atoms + nr
    per_atom = lens[-prog.n_atoms:]
    assert (per_atom == 1 + np.bincount(prog.head, minlength=prog.n_atoms)).all()


def _supported_models(prog):
    """Models M with M = T_P(M) (T read with body+ in M, body- disjoint from
    M) that violate no constraint: the models of the Clark completion."""
    out = set()
    rules = list(prog.rules())
    for mask in range(1 << prog.n_atoms):
        M = {i for i in range(prog.n_atoms) if (mask >> i) & 1}
        T = {h for h, p, n in rules if h >= 0 and set(p) <= M and not (set(n) & M)}
        bad = any(h < 0 and set(p) <= M and not (set(n) & M) for h, p, n in rules)
        if T == M and not bad:
            out.add(frozenset(M))
    return out


def _nogood_solutions(nv, off, lits, fixed=None):
    """All total assignments (tuples of +-1) violating no nogood."""
    sols = []
    ngs = [lits[off[i]:off[i + 1]] for i in range(off.shape[0] - 1)]
    for bits in itertools.product((1, -1), repeat=nv):
        if fixed is not None and any(f != 0 and f != b for f, b in zip(fixed, bits)):
            continue
        if all(not all((bits[abs(l) - 1] == (1 if l > 0 else -1)) for l in g) for g in ngs):
            sols.append(bits)
    return sols


@pytest.mark.parametrize("seed", range(12))
def test_completion_solutions_are_supported_models(seed):
    prog = random_program(4, 3, program_seed(105, seed))
    nv, off, lits = oracle.completion(prog)
    sols = _nogood_solutions(nv, off, lits)
    proj = {frozenset(i for i in range(prog.n_atoms) if s[i] == 1) for s in sols}
    assert proj == _supported_models(prog)
    # aux atoms are functions of the atoms: one solution per supported model
    assert len(sols) == len(proj)


# ------------------------------------------------------------ UP closure

def _classify(g, val):
    n_out, sat = 0, False
    for l in g:
        v = val[abs(l) - 1]
        if v == (-1 if l > 0 else 1):
            return "sat"
        if v != (1 if l > 0 else -1):
            n_out += 1
    return "violated" if n_out == 0 else ("unit" if n_out == 1 else "open")


@pytest.mark.parametrize("seed", range(30))
def test_up_closure_is_derived_fixpoint(seed):
    prog = random_program(12, 30, program_seed(106, seed))
    nv, off, lits = oracle.completion(prog)
    ngs = [lits[off[i]:off[i + 1]] for i in range(off.shape[0] - 1)]
    rng = np.random.default_rng(seed)
    partial = np.zeros(nv, np.int8)
    pick = rng.choice(prog.n_atoms, size=3, replace=False)
    partial[pick] = rng.choice([-1, 1], size=3)
    conflict, clo, order, reasons = oracle.up_closure(prog, partial)
    # every derived literal was forced by a nogood unit at that point
    val = partial.copy()
    for lit, g in zip(order, reasons):
        assert _classify(ngs[g], val) == "unit"
        v = abs(lit) - 1
        assert val[v] == 0
        assert (-lit) in ngs[g] or lit in [-x for x in ngs[g]]
        val[v] = 1 if lit > 0 else -1
    assert (val == clo).all()
    kinds = [_classify(g, clo) for g in ngs]
    if conflict:
        assert "violated" in kinds
    else:
        assert "violated" not in kinds and "unit" not in kinds


@pytest.mark.parametrize("seed", range(12))
def test_up_closure_sound_by_brute_force(seed):
    prog = random_program(4, 3, program_seed(107, seed))
    nv, off, lits = oracle.completion(prog)
    rng = np.random.default_rng(seed)
    partial = np.zeros(nv, np.int8)
    partial[rng.integers(0, prog.n_atoms)] = rng.choice([-1, 1])
    conflict, clo, _, _ = oracle.up_closure(prog, partial)
    sols = _nogood_solutions(nv, off, lits, fixed=partial)
    if conflict:
        assert sols == []
    for s in sols:   # every solution extending the partial contains the closure
        assert all(c == 0 or c == x for c, x in zip(clo, s))


def test_c8_needs_stability_check():
    """p <- q. q <- p. :- not p.  Propagation alone makes everything true at
    the root; the reduct check must reject it (no answer set)."""
    prog = from_rules(2, [(0, [1], []), (1, [0], []), (-1, [], [0])])
    nv, _, _ = oracle.completion(prog)
    conflict, clo, _, _ = oracle.up_closure(prog, np.zeros(nv, np.int8))
    assert not conflict and (clo != 0).all() and clo[0] == 1 and clo[1] == 1
    assert not oracle.is_answer_set(prog, np.array([1, 1], np.uint8))
    status, models, _ = oracle.cdnl(prog)
    assert status == oracle.UNSAT and len(models) == 0


def test_crosscheck_script_on_a_slice():
    """The committed O2-vs-O1 cross-check (run on 4 x 10^4 programs of the
    tiny family and 10^4 denser ones offline) passes on a slice of each."""
    from oracle import crosscheck
    assert crosscheck.main(["--count", "12", "--first", "9000", "--workers", "2"]) == 0
    assert crosscheck.main(["--count", "8", "--first", "9000", "--workers", "2", "--rules", "60",
                            "--constraints", "4"]) == 0
