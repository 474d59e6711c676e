"""Compact completion, the Jeroslow-Wang score and the decaying activity
(VSIDS-style) decision heuristic (needs a GB300).

Compact completion leaves out, for empty positive or negative bodies, the
nogoods that the units {Ft_r} / {Fn_r} settle at the root: the library's
nogood and literal counts equal the oracle's compact completion, unit
propagation reaches the oracle's closure, and the answer sets are unchanged.
The Jeroslow-Wang score and the decaying activity (Section 4 names
Jeroslow-Wang and activity among the decision heuristics) only order
decisions: answers equal the oracle's, under fwd-learning and first-UIP
resolution learning alike."""
import json
import os

import numpy as np
import pytest

import oracle
from synth.programs import coloring_program, program_seed, random_program, tiny_program

from test_gpu_solver import _gpu_to_oracle_perm, _sets

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


def _golden():
    data = json.load(open(os.path.join(GOLDEN, "tiny_answer_sets.json")))
    return {r["index"]: r["answer_sets"] for r in data["programs"]}


def _masks(models, n):
    w = np.int64(1) << np.arange(n, dtype=np.int64)
    return sorted(int((np.asarray(m[:n], np.int64) * w).sum()) for m in models)


@pytest.mark.parametrize("seed", range(6))
def test_compact_counts_equal_the_oracle(gpu, seed):
    prog = random_program(500 + 300 * seed, 1500 + 900 * seed, program_seed(620, seed))
    _, off, lits = oracle.completion(prog, compact=True)
    s = gpu.Program(prog, compact=True).stats()
    assert s["n_nogoods"] == off.shape[0] - 1
    assert s["n_literals"] == lits.shape[0]
    full = gpu.Program(prog).stats()
    assert s["n_literals"] < full["n_literals"]


@pytest.mark.parametrize("seed", range(12))
def test_compact_closure_equals_the_oracle(gpu, seed):
    prog = random_program(60 + seed * 7, 200 + seed * 31, program_seed(621, seed))
    P = gpu.Program(prog, compact=True)
    perm = _gpu_to_oracle_perm(prog)
    rng = np.random.default_rng(seed)
    for trial in range(4):
        partial = np.zeros(P.n_vars, np.int8)
        k = int(rng.integers(0, 12))
        pick = rng.choice(prog.n_atoms, size=k, replace=False)
        partial[pick] = rng.choice([-1, 1], size=k)
        conflict, clo = P.propagate(partial)
        opart = np.zeros(P.n_vars, np.int8)
        opart[perm] = partial
        oconf, oclo, _, _ = oracle.up_closure(prog, opart, compact=True)
        assert conflict == oconf
        if not oconf:
            assert (clo == oclo[perm]).all()


@pytest.mark.parametrize("heuristic,compact", [(0, True), (4, False), (4, True), (5, False)])
def test_tiny_programs_enumerate_the_brute_force(gpu, heuristic, compact):
    golden = _golden()
    for i in range(0, 1000, 7):
        prog = tiny_program(i)
        status, models, n = gpu.Program(prog, heuristic=heuristic, compact=compact).solve(0, cap=256)
        assert _masks(models, prog.n_atoms) == golden[i] and n == len(golden[i]), i
        assert status == (gpu.SAT if golden[i] else gpu.UNSAT)


@pytest.mark.parametrize("heuristic,compact", [(4, False), (4, True), (1, True), (5, False)])
@pytest.mark.parametrize("seed", range(5))
def test_medium_programs_agree_with_the_oracle(gpu, heuristic, compact, seed):
    prog = random_program(300 + 400 * seed, 900 + 800 * seed, program_seed(622, seed))
    ost, _, _ = oracle.cdnl(prog, max_models=1, time_budget_s=60)
    assert ost in (oracle.SAT, oracle.UNSAT)
    P = gpu.Program(prog, heuristic=heuristic, compact=compact, time_budget_ms=60_000)
    st, models, _ = P.solve(1, cap=1)
    assert st == (gpu.SAT if ost == oracle.SAT else gpu.UNSAT)
    for m in models:
        assert oracle.is_answer_set(prog, m)


def test_colouring_enumeration_under_jw_and_compact(gpu):
    prog = coloring_program(40, 4.5, seed_index=7)
    ost, om, _ = oracle.cdnl(prog, time_budget_s=120)
    assert ost == oracle.SAT
    for heuristic, compact in ((4, False), (4, True), (0, True), (5, False)):
        st, models, cnt = gpu.Program(prog, heuristic=heuristic, compact=compact,
                                      time_budget_ms=120_000).solve(0, cap=1 << 12)
        assert _sets(models) == _sets(om) and cnt == len(om), (heuristic, compact)


def test_compact_batched(gpu):
    golden = _golden()
    idx = list(range(3, 1000, 11))
    P = [gpu.Program(tiny_program(i), compact=True, heuristic=4) for i in idx]
    st, nm, models = gpu.solve_batch(P, max_models_each=0, cap_each=64)
    for k, i in enumerate(idx):
        assert _masks(models[k], 20) == golden[i] and nm[k] == len(golden[i]), i


@pytest.mark.parametrize("learning,restarts", [(0, 0), (1, 0), (1, 16)])
@pytest.mark.parametrize("seed", range(4))
def test_vsids_search_answers(gpu, learning, restarts, seed):
    prog = random_program(500 + 300 * seed, 1100 + 600 * seed, program_seed(623, seed))
    ost, _, _ = oracle.cdnl(prog, max_models=1, time_budget_s=60)
    assert ost in (oracle.SAT, oracle.UNSAT)
    P = gpu.Program(prog, heuristic=gpu.HEUR_VSIDS, learning=learning, restart_conflicts=restarts,
                    time_budget_ms=60_000)
    st, models, _ = P.solve(1, cap=1)
    assert st == (gpu.SAT if ost == oracle.SAT else gpu.UNSAT)
    for m in models:
        assert oracle.is_answer_set(prog, m)


def test_vsids_colouring_enumeration_with_resolution_and_restarts(gpu):
    prog = coloring_program(40, 4.5, seed_index=7)
    ost, om, _ = oracle.cdnl(prog, time_budget_s=120)
    st, models, cnt = gpu.Program(prog, heuristic=gpu.HEUR_VSIDS, learning=gpu.LEARN_RES, restart_conflicts=8,
                                  time_budget_ms=120_000).solve(0, cap=1 << 12)
    assert _sets(models) == _sets(om) and cnt == len(om)
