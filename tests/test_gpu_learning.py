"""Resolution-based learning to the first UIP on the GPU (Section 4.2,
Algorithm 3; needs a GB300).  At the k-th conflict of a search (the solve
stops on its conflict budget right after the analysis, before the
backjump), the learned nogood and the backjump target equal those of the
oracle's first-UIP resolution run on the GPU's own state (trail order,
levels, reasons, conflicting nogood).  Whole searches with it give the
oracle's answers."""
import numpy as np
import pytest

import oracle
from synth.programs import batch_programs, coloring_program, program_seed, random_program, tiny_program

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


def _lits(arr):
    return [(int(l) >> 1, bool(int(l) & 1)) for l in arr]


def _oracle_of_state(gpu, P, lc):
    """The oracle's first-UIP analysis of the GPU's last conflict."""
    st = P.state()
    level, reason = st["level"], st["reason"]
    trail = _lits(lc["trail"])
    pos = np.full(P.n_vars, -1, np.int64)
    sign = {}
    for i, (v, f) in enumerate(trail):
        pos[v] = i
        sign[v] = f
    dec = {int(level[v]): v for (v, _) in trail if reason[v] == gpu.R_DECISION}

    def antecedent(v):
        r = int(reason[v])
        if r == gpu.R_DECISION:
            return None
        if r == gpu.R_COMPLETE:
            # a literal set by CompleteAssignment: its antecedent is every
            # decision up to its level
            return [(v, not sign[v])] + [(dec[L], False) for L in range(2, int(level[v]) + 1)]
        return _lits(P.nogood(r))

    delta = _lits(P.nogood(lc["conflict"]))
    d, kappa, uip = oracle.first_uip(delta, pos, level, antecedent)
    return d, kappa, uip, level, delta


def _check_conflict(gpu, P):
    lc = P.last_conflict()
    assert lc is not None
    d, kappa, uip, level, delta = _oracle_of_state(gpu, P, lc)
    learned = _lits(P.nogood(lc["learned"]))
    assert len(learned) == lc["length"]
    assert learned[0] == uip                                   # the first UIP comes first
    assert set(learned) == {l for l in d if level[l[0]] > 1}   # root-level literals left out
    assert len(set(learned)) == len(learned)
    assert lc["target"] == max(kappa, 1)
    assert lc["level"] == max(int(level[v]) for (v, _) in delta)


CASES = [(300, 900, 0), (300, 900, 1), (800, 2000, 2), (2000, 5000, 3), (5000, 12000, 4), (20000, 50000, 5)]


@pytest.mark.parametrize("atoms,rules,seed", CASES)
@pytest.mark.parametrize("k", [1, 2, 3, 5, 9, 17, 40])
@pytest.mark.parametrize("grid", [1, 0])
def test_learned_nogood_equals_the_oracle(gpu, atoms, rules, seed, k, grid):
    prog = random_program(atoms, rules, program_seed(701, seed))
    P = gpu.Program(prog, learning=gpu.LEARN_RES, conflict_budget=k, grid_ctas=grid, time_budget_ms=60_000)
    status, _, _ = P.solve(1, cap=1)
    s = P.stats()
    if status != gpu.UNKNOWN or s["conflicts"] != k:
        pytest.skip("search ended before the k-th conflict")
    _check_conflict(gpu, P)


@pytest.mark.parametrize("mode", [1, 2, 3])
@pytest.mark.parametrize("k", [4, 25])
def test_learned_nogood_in_every_view(gpu, mode, k):
    prog = random_program(3000, 7500, program_seed(702, k))
    P = gpu.Program(prog, learning=gpu.LEARN_RES, view_mode=mode, conflict_budget=k, time_budget_ms=60_000)
    status, _, _ = P.solve(1, cap=1)
    if status != gpu.UNKNOWN or P.stats()["conflicts"] != k:
        pytest.skip("search ended before the k-th conflict")
    _check_conflict(gpu, P)


@pytest.mark.parametrize("k", [3, 12, 30])
def test_learned_nogood_with_frontier_and_activity(gpu, k):
    prog = random_program(4000, 10000, program_seed(703, k))
    P = gpu.Program(prog, learning=gpu.LEARN_RES, frontier=True, heuristic=1, conflict_budget=k,
                    time_budget_ms=60_000)
    status, _, _ = P.solve(1, cap=1)
    if status != gpu.UNKNOWN or P.stats()["conflicts"] != k:
        pytest.skip("search ended before the k-th conflict")
    _check_conflict(gpu, P)


def test_some_parity_case_runs(gpu):
    """At least most of the parity cases reach their conflict (the skips
    above must not hide the comparison)."""
    reached = 0
    for (atoms, rules, seed) in CASES:
        P = gpu.Program(random_program(atoms, rules, program_seed(701, seed)), learning=gpu.LEARN_RES,
                        conflict_budget=9, time_budget_ms=60_000)
        status, _, _ = P.solve(1, cap=1)
        reached += status == gpu.UNKNOWN and P.stats()["conflicts"] == 9
    assert reached >= len(CASES) // 2


@pytest.mark.parametrize("index", [3, 77, 151, 402, 555, 918])
@pytest.mark.parametrize("grid", [1, 0])
def test_tiny_full_enumeration(gpu, index, grid):
    prog = tiny_program(index)
    want = _sets(oracle.brute_force(prog))
    status, models, n = gpu.Program(prog, learning=gpu.LEARN_RES, grid_ctas=grid).solve(0, cap=1 << 12)
    assert _sets(models) == want and n == len(want)
    assert status == (gpu.SAT if want else gpu.UNSAT)


@pytest.mark.parametrize("seed", range(8))
def test_search_answers(gpu, seed):
    prog = random_program(600 + 150 * seed, 1400 + 300 * seed, program_seed(704, seed))
    ost, _, _ = oracle.cdnl(prog, max_models=1, time_budget_s=30)
    assert ost in (oracle.SAT, oracle.UNSAT)
    P = gpu.Program(prog, learning=gpu.LEARN_RES, time_budget_ms=60_000)
    st, models, _ = P.solve(1, cap=1)
    assert st == (gpu.SAT if ost == oracle.SAT else gpu.UNSAT)
    for m in models:
        assert oracle.is_answer_set(prog, m)
    s = P.stats()
    if s["conflicts"] > s["loop_nogoods"]:
        assert s["learned"] > 0


def test_colouring_enumeration(gpu):
    """All 360 answer sets of the n = 40 colouring program, against the oracle."""
    prog = coloring_program(40, 4.5, seed_index=7)
    ost, om, _ = oracle.cdnl(prog, time_budget_s=120)
    assert ost in (oracle.SAT, oracle.UNSAT)
    st, models, cnt = gpu.Program(prog, learning=gpu.LEARN_RES, time_budget_ms=120_000).solve(0, cap=1 << 14)
    assert _sets(models) == _sets(om) and cnt == len(om)


def test_batch(gpu):
    progs = batch_programs(12, rules_per_atom=2, lo=50, hi=1500, config_id=705)
    P = [gpu.Program(p, learning=gpu.LEARN_RES, time_budget_ms=20_000) for p in progs]
    st, nm, models = gpu.solve_batch(P, max_models_each=1, cap_each=1)
    for i, p in enumerate(progs):
        ost, _, _ = oracle.cdnl(p, max_models=1, time_budget_s=30)
        assert ost in (oracle.SAT, oracle.UNSAT)
        assert st[i] == (gpu.SAT if ost == oracle.SAT else gpu.UNSAT), i
        for m in models[i]:
            assert oracle.is_answer_set(p, m)


def test_batch_conflict_parity(gpu):
    """In a batch (one CTA per program) the analysis runs in the program's
    CTA: the k-th conflict of each program against the oracle."""
    progs = batch_programs(6, rules_per_atom=3, lo=400, hi=3000, config_id=706)
    P = [gpu.Program(p, learning=gpu.LEARN_RES, conflict_budget=6, time_budget_ms=20_000) for p in progs]
    st, _, _ = gpu.solve_batch(P, max_models_each=1, cap_each=1)
    checked = 0
    for i in range(len(progs)):
        if st[i] == gpu.UNKNOWN and P[i].stats()["conflicts"] == 6:
            _check_conflict(gpu, P[i])
            checked += 1
    assert checked >= 1


def test_unknown_learning_is_rejected(gpu):
    with pytest.raises(gpu.AspError):
        gpu.Program(tiny_program(1), learning=7)
