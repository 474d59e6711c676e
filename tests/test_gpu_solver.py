"""GPU solver against the CPU oracle (needs a GB300).

Answer sets are compared as sets (the search order is not unique); SAT/UNSAT
must agree; every returned model must pass the oracle's reduct check; the
propagation fixpoint is unique, so it is compared literal by literal.
"""
import json
import os

import numpy as np
import pytest

import oracle
from synth.programs import (coloring_program, from_rules, program_seed, random_program,
                            tiny_program)

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


def _sets(models):
    return {frozenset(np.nonzero(m)[0].tolist()) for m in models}


def _named(atoms, rules):
    idx = {a: i for i, a in enumerate(atoms)}
    return from_rules(len(atoms), [(-1 if h is None else idx[h], [idx[a] for a in p], [idx[a] for a in n])
                                   for h, p, n in rules])


HAND = json.load(open(os.path.join(GOLDEN, "hand_cases.json")))["cases"]


@pytest.mark.parametrize("case", HAND, ids=[c["name"] for c in HAND])
def test_hand_cases(gpu, case):
    prog = _named(case["atoms"], case["rules"])
    P = gpu.Program(prog)
    status, models, n = P.solve(0, cap=64)
    names = case["atoms"]
    got = {frozenset(names[i] for i in s) for s in _sets(models)}
    want = {frozenset(s) for s in case["answer_sets"]}
    assert got == want and n == len(want)
    assert status == (gpu.SAT if want else gpu.UNSAT)


@pytest.mark.parametrize("index", list(range(0, 1000, 37)))
def test_tiny_programs_full_enumeration(gpu, index):
    """20 atoms, 40 rules, 3 constraints: all answer sets vs brute force over 2^20."""
    prog = tiny_program(index)
    want = _sets(oracle.brute_force(prog))
    status, models, n = gpu.Program(prog).solve(0, cap=1 << 12)
    assert _sets(models) == want and n == len(want)
    assert status == (gpu.SAT if want else gpu.UNSAT)


@pytest.mark.parametrize("seed", range(40))
def test_small_random_programs(gpu, seed):
    prog = random_program(10, 6 + seed % 14, program_seed(201, seed))
    want = _sets(oracle.brute_force(prog))
    _, models, n = gpu.Program(prog).solve(0, cap=1 << 12)
    assert _sets(models) == want and n == len(want)


MEDIUM = [(120, 480, s) for s in range(6)] + [(300, 900, s) for s in range(4)] + [(2000, 4000, s) for s in range(4)]


@pytest.mark.parametrize("na,nr,seed", MEDIUM)
def test_medium_programs_sat_agreement_and_validity(gpu, na, nr, seed):
    """Random programs the oracle decides quickly: SAT/UNSAT must agree and
    every model must be an answer set."""
    prog = random_program(na, nr, program_seed(202, 1000 * na + seed))
    ost, omodels, _ = oracle.cdnl(prog, max_models=1, time_budget_s=60)
    assert ost in (oracle.SAT, oracle.UNSAT)
    P = gpu.Program(prog, time_budget_ms=60_000)
    status, models, n = P.solve(3, cap=3)
    assert status == (gpu.SAT if ost == oracle.SAT else gpu.UNSAT)
    for m in models:
        assert oracle.is_answer_set(prog, m)
    assert len(_sets(models)) == len(models)


@pytest.mark.parametrize("k", [1, 5, 40])
def test_max_models(gpu, k):
    rules = []
    for i in range(6):                       # six independent even loops: 64 answer sets
        rules += [(2 * i, [], [2 * i + 1]), (2 * i + 1, [], [2 * i])]
    prog = from_rules(12, rules)
    status, models, n = gpu.Program(prog).solve(k, cap=k)
    assert status == gpu.SAT and n == k and len(_sets(models)) == k
    assert all(oracle.is_answer_set(prog, m) for m in models)


def test_small_coloring_enumeration(gpu):
    prog = coloring_program(12, 3.0, seed_index=5)
    _, om, _ = oracle.cdnl(prog)
    status, models, n = gpu.Program(prog).solve(0, cap=1 << 14)
    assert _sets(models) == _sets(om) and n == len(om)


# ------------------------------------------------------ propagation parity

def _gpu_to_oracle_perm(prog):
    """oracle variable index for each GPU variable.  Both layouts are
    documented: both interleave b,t,n per rule after the atoms; the GPU
    numbers headed rules by head atom (ties in input order), the oracle in
    input order."""
    na = prog.n_atoms
    headed = np.nonzero(prog.head >= 0)[0]
    J = headed.shape[0]
    o = np.argsort(prog.head[headed], kind="stable")     # GPU rule j -> input ordinal
    perm = np.arange(na + 3 * J)
    j = np.arange(J)
    for q in range(3):
        perm[na + 3 * j + q] = na + 3 * o + q
    return perm


@pytest.mark.parametrize("seed", range(25))
def test_propagation_fixpoint_equals_oracle(gpu, seed):
    prog = random_program(60 + seed * 7, 200 + seed * 31, program_seed(203, seed))
    P = gpu.Program(prog)
    perm = _gpu_to_oracle_perm(prog)
    rng = np.random.default_rng(seed)
    for trial in range(4):
        partial = np.zeros(P.n_vars, np.int8)
        k = int(rng.integers(1, 12))
        pick = rng.choice(prog.n_atoms, size=k, replace=False)
        partial[pick] = rng.choice([-1, 1], size=k)
        conflict, clo = P.propagate(partial)
        opart = np.zeros(P.n_vars, np.int8)
        opart[perm] = partial
        oconf, oclo, _, _ = oracle.up_closure(prog, opart)
        assert conflict == oconf
        if not oconf:
            assert (clo == oclo[perm]).all()


def test_propagation_on_large_store(gpu):
    """Full-size program (100k atoms, 400k rules): root-level closure."""
    from synth.programs import large_random_program
    prog = large_random_program(0)
    P = gpu.Program(prog)
    perm = _gpu_to_oracle_perm(prog)
    conflict, clo = P.propagate(np.zeros(P.n_vars, np.int8))
    oconf, oclo, _, _ = oracle.up_closure(prog, np.zeros(P.n_vars, np.int8))
    assert conflict == oconf
    if not oconf:
        assert (clo == oclo[perm]).all()


# ------------------------------------------------ dependency bitmaps

@pytest.mark.parametrize("seed", range(6))
def test_dependency_bitmaps_follow_reasons(gpu, seed):
    """After a search, each propagated variable above the root has
    Deps = OR of the Deps of its reason's other literals with level > 1, and
    each decision at level L has exactly bit L-1 (Section 4.2)."""
    prog = random_program(1500, 3000 + 300 * seed, program_seed(204, seed))
    P = gpu.Program(prog, conflict_budget=2000, time_budget_ms=20_000)
    status, _, _ = P.solve(1, cap=1)   # any outcome: the committed trail is checked
    st = P.state(deps_words=64)
    lvl, rea, deps = st["level"], st["reason"], st["deps"]
    W = deps.shape[1]
    checked = 0
    for v in st["trail"]:
        L = int(lvl[v])
        if L <= 1:
            continue
        nw = min(W, (L + 63) // 64)
        if rea[v] == gpu.R_DECISION:
            want = np.zeros(nw, np.uint64)
            want[(L - 1) // 64] = np.uint64(1) << np.uint64((L - 1) % 64)
        elif rea[v] == gpu.R_COMPLETE:
            continue
        else:
            want = np.zeros(nw, np.uint64)
            for lit in P.nogood(int(rea[v])):
                u = lit >> 1
                if u == v or lvl[u] <= 1:
                    continue
                want |= deps[u, :nw] & _mask(min(W, (int(lvl[u]) + 63) // 64), nw)
        assert (deps[v, :nw] == want).all(), v
        checked += 1
    if status == gpu.SAT:
        assert checked > 0


def _mask(words, nw):
    m = np.zeros(nw, np.uint64)
    m[:words] = np.uint64(0xFFFFFFFFFFFFFFFF)
    return m
