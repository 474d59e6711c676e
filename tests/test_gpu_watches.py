"""Watched literals on long nogoods (Algorithm 2 watches two literals of a
nogood, long learned ones included; needs a GB300).

Long nogoods (more than 15 literals: here the nogood {Tp} u {Fb_r : r in
rules(p)} of atoms with many rules, and the learned nogoods) are checked
through two watched positions and scanned only when a watched literal holds.
Every round checks every such nogood, so a missed propagation would show as
a closure different from the oracle's unique UP closure, or as a repeated or
missing answer set under enumeration (blocking nogoods are long learned
nogoods)."""
import numpy as np
import pytest

import oracle
from synth.programs import program_seed, random_program, tiny_program

from test_gpu_solver import _gpu_to_oracle_perm, _sets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1909_01786_gb300 import aspgpu
    aspgpu.lib()
    return aspgpu


@pytest.mark.parametrize("fr", [0, 1, 2])
@pytest.mark.parametrize("seed", range(8))
def test_closure_with_long_atom_nogoods(gpu, fr, seed):
    prog = random_program(60 + 10 * seed, 1200 + 150 * seed, program_seed(630, seed))   # ~20 rules per atom
    P = gpu.Program(prog, frontier=fr)
    assert P.stats()["n_long_nogoods"] > 0
    perm = _gpu_to_oracle_perm(prog)
    rng = np.random.default_rng(seed)
    for trial in range(6):
        partial = np.zeros(P.n_vars, np.int8)
        k = int(rng.integers(1, 20))
        pick = rng.choice(prog.n_atoms, size=k, replace=False)
        partial[pick] = rng.choice([-1, 1], size=k)
        conflict, clo = P.propagate(partial)
        opart = np.zeros(P.n_vars, np.int8)
        opart[perm] = partial
        oconf, oclo, _, _ = oracle.up_closure(prog, opart)
        assert conflict == oconf
        if not oconf:
            assert (clo == oclo[perm]).all()


@pytest.mark.parametrize("seed", range(6))
def test_search_with_long_atom_nogoods(gpu, seed):
    prog = random_program(150 + 30 * seed, 2000 + 300 * seed, program_seed(631, seed))
    ost, om, _ = oracle.cdnl(prog, max_models=4, time_budget_s=60)
    assert ost in (oracle.SAT, oracle.UNSAT)
    st, models, n = gpu.Program(prog, time_budget_ms=60_000).solve(4, cap=4)
    assert st == (gpu.SAT if ost == oracle.SAT else gpu.UNSAT)
    assert n == len(om) or n == 4
    assert len(_sets(models)) == len(models)
    for m in models:
        assert oracle.is_answer_set(prog, m)


@pytest.mark.parametrize("learning", [0, 1])
def test_enumeration_respects_long_blocking_nogoods(gpu, learning):
    """Every answer set once, with many long blocking nogoods: six
    independent even loops plus tiny programs."""
    from synth.programs import from_rules
    rules = []
    for i in range(9):                       # nine independent even loops: 512 answer sets
        rules += [(2 * i, [], [2 * i + 1]), (2 * i + 1, [], [2 * i])]
    prog = from_rules(18, rules)
    st, models, n = gpu.Program(prog, learning=learning).solve(0, cap=1024)
    assert st == gpu.SAT and n == 512 and len(_sets(models)) == 512
    for i in range(0, 1000, 97):
        p = tiny_program(i)
        want = _sets(oracle.brute_force(p))
        _, m2, n2 = gpu.Program(p, learning=learning).solve(0, cap=256)
        assert _sets(m2) == want and n2 == len(want)
