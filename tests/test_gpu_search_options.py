"""Search options beyond the paper's defaults (needs a GB300): the
asserting-level backjump of fwd-learning and Luby restarts.  Both keep the
oracle's answers; the backjump targets and restart counts follow their
definitions exactly."""
import numpy as np
import pytest

import oracle
from synth.programs import coloring_program, program_seed, random_program, tiny_program

from test_gpu_solver import _sets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1909_01786_gb300 import aspgpu
    aspgpu.lib()
    return aspgpu


def _luby(i):
    """Luby et al.'s sequence, by its recursive definition (i >= 1)."""
    k = 1
    while (1 << k) - 1 < i:
        k += 1
    if (1 << k) - 1 == i:
        return 1 << (k - 1)
    return _luby(i - (1 << (k - 1)) + 1)


def test_luby_prefix():
    assert [_luby(i) for i in range(1, 16)] == [1, 1, 2, 1, 1, 2, 4, 1, 1, 2, 1, 1, 2, 4, 8]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("atoms,rules,seed", [(800, 2000, 0), (3000, 7500, 1), (20000, 50000, 2)])
@pytest.mark.parametrize("k", [1, 3, 8, 21])
def test_backjump_target(gpu, mode, atoms, rules, seed, k):
    """At the k-th conflict: the learned nogood is decision literals; the
    target is h-1 (mode 0) or the second-highest of their levels (mode 1)."""
    prog = random_program(atoms, rules, program_seed(801, seed))
    P = gpu.Program(prog, backjump=mode, conflict_budget=k, time_budget_ms=60_000)
    status, _, _ = P.solve(1, cap=1)
    if status != gpu.UNKNOWN or P.stats()["conflicts"] != k:
        pytest.skip("search ended before the k-th conflict")
    lc = P.last_conflict()
    st = P.state()
    levels = sorted(int(st["level"][int(l) >> 1]) for l in P.nogood(lc["learned"]))
    assert all(st["reason"][int(l) >> 1] == gpu.R_DECISION for l in P.nogood(lc["learned"]))
    if mode == 0:
        assert lc["target"] == levels[-1] - 1
    else:
        assert lc["target"] == (levels[-2] if len(levels) > 1 else 1)


@pytest.mark.parametrize("index", [3, 77, 151, 402, 555, 918])
@pytest.mark.parametrize("backjump,restarts", [(1, 0), (0, 1), (1, 2)])
def test_tiny_full_enumeration(gpu, index, backjump, restarts):
    prog = tiny_program(index)
    want = _sets(oracle.brute_force(prog))
    P = gpu.Program(prog, backjump=backjump, restart_conflicts=restarts)
    status, models, n = P.solve(0, cap=1 << 12)
    assert _sets(models) == want and n == len(want)
    assert status == (gpu.SAT if want else gpu.UNSAT)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("backjump,restarts,learning", [(1, 0, 0), (0, 4, 0), (1, 4, 0), (0, 4, 1)])
def test_search_answers(gpu, seed, backjump, restarts, learning):
    prog = random_program(600 + 200 * seed, 1400 + 400 * seed, program_seed(802, seed))
    ost, _, _ = oracle.cdnl(prog, max_models=1, time_budget_s=30)
    assert ost in (oracle.SAT, oracle.UNSAT)
    P = gpu.Program(prog, backjump=backjump, restart_conflicts=restarts, learning=learning,
                    time_budget_ms=60_000)
    st, models, _ = P.solve(1, cap=1)
    assert st == (gpu.SAT if ost == oracle.SAT else gpu.UNSAT)
    for m in models:
        assert oracle.is_answer_set(prog, m)


@pytest.mark.parametrize("unit", [1, 3])
@pytest.mark.parametrize("learning", [0, 1])
def test_restart_count_follows_luby(gpu, unit, learning):
    """With every conflict learned (a budget-bound search without models),
    restarts = the number of prefixes of unit x (1 1 2 1 1 2 4 ...) that fit
    in the conflicts."""
    prog = random_program(20000, 50000, program_seed(803, 0))
    budget = 60
    P = gpu.Program(prog, restart_conflicts=unit, learning=learning, conflict_budget=budget,
                    time_budget_ms=60_000)
    status, _, _ = P.solve(1, cap=1)
    s = P.stats()
    if status != gpu.UNKNOWN or s["conflicts"] != budget or s["loop_nogoods"] or s["models"]:
        pytest.skip("search ended early or met loops/models")
    want, total, i = 0, 0, 1
    while total + unit * _luby(i) <= budget:
        total += unit * _luby(i)
        want += 1
        i += 1
    assert s["restarts"] == want


def test_colouring_enumeration_with_restarts(gpu):
    prog = coloring_program(40, 4.5, seed_index=7)
    ost, om, _ = oracle.cdnl(prog, time_budget_s=120)
    assert ost in (oracle.SAT, oracle.UNSAT)
    P = gpu.Program(prog, backjump=1, restart_conflicts=2, time_budget_ms=120_000)
    st, models, cnt = P.solve(0, cap=1 << 14)
    assert _sets(models) == _sets(om) and cnt == len(om)


def test_bad_options_are_rejected(gpu):
    with pytest.raises(gpu.AspError):
        gpu.Program(tiny_program(1), backjump=5)
    with pytest.raises(gpu.AspError):
        gpu.Program(tiny_program(1), restart_conflicts=-1)


# ---- several conflicts per round (Section 4.2: "one or more" conflicts)

@pytest.mark.parametrize("index", [3, 77, 151, 402, 555, 918])
@pytest.mark.parametrize("learning", [0, 1])
def test_tiny_full_enumeration_several_conflicts(gpu, index, learning):
    prog = tiny_program(index)
    want = _sets(oracle.brute_force(prog))
    P = gpu.Program(prog, conflicts_per_round=4, learning=learning)
    status, models, n = P.solve(0, cap=1 << 12)
    assert _sets(models) == want and n == len(want)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("learning,backjump,restarts", [(0, 0, 0), (1, 0, 0), (0, 1, 8)])
def test_search_answers_several_conflicts(gpu, seed, learning, backjump, restarts):
    prog = random_program(600 + 200 * seed, 1400 + 400 * seed, program_seed(804, seed))
    ost, _, _ = oracle.cdnl(prog, max_models=1, time_budget_s=30)
    assert ost in (oracle.SAT, oracle.UNSAT)
    P = gpu.Program(prog, conflicts_per_round=4, learning=learning, backjump=backjump,
                    restart_conflicts=restarts, time_budget_ms=60_000)
    st, models, _ = P.solve(1, cap=1)
    assert st == (gpu.SAT if ost == oracle.SAT else gpu.UNSAT)
    for m in models:
        assert oracle.is_answer_set(prog, m)


def test_several_conflicts_are_analysed(gpu):
    """With one conflict per round every conflicting round is one analysis;
    with up to four, some rounds analyse more (each learns a nogood)."""
    tot = {1: [0, 0], 4: [0, 0]}
    for seed in range(4):
        prog = random_program(20000, 50000, program_seed(805, seed))
        for cpr in (1, 4):
            P = gpu.Program(prog, conflicts_per_round=cpr, conflict_budget=60, time_budget_ms=60_000)
            status, _, _ = P.solve(1, cap=1)
            s = P.stats()
            if status == gpu.UNSAT:
                continue          # a final conflict at the root is counted outside rounds
            c = s["conflicts"] - s["loop_nogoods"]     # loop nogoods are analysed outside rounds
            tot[cpr][0] += c
            tot[cpr][1] += s["conflict_rounds"]
            if cpr == 1:
                assert c == s["conflict_rounds"]
            assert s["conflict_rounds"] <= c <= cpr * s["conflict_rounds"]
    assert tot[4][0] > tot[4][1]


@pytest.mark.parametrize("k", [3, 10, 30])
def test_last_analysis_of_a_round_equals_the_oracle(gpu, k):
    """Resolution learning with several conflicts per round: the round's last
    analysis (run on the same state as the others) against the oracle."""
    from test_gpu_learning import _check_conflict
    prog = random_program(5000, 12000, program_seed(806, k))
    P = gpu.Program(prog, conflicts_per_round=4, learning=gpu.LEARN_RES, conflict_budget=k,
                    time_budget_ms=60_000)
    status, _, _ = P.solve(1, cap=1)
    if status != gpu.UNKNOWN or P.stats()["conflicts"] < k:
        pytest.skip("search ended before the k-th conflict")
    _check_conflict(gpu, P)


def test_bad_conflicts_per_round_is_rejected(gpu):
    with pytest.raises(gpu.AspError):
        gpu.Program(tiny_program(1), conflicts_per_round=5)
