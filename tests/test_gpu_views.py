"""The three shared-memory view layouts of the sweep (2-bit with literals by
variable, 2-bit and byte views over a copy of the store whose literals name
view entries) give the same propagation fixpoints, answer sets and
dependency bitmaps (needs a GB300)."""
import numpy as np
import pytest

import oracle
from synth.programs import batch_programs, program_seed, random_program, tiny_program

from test_gpu_solver import _gpu_to_oracle_perm, _mask, _sets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1909_01786_gb300 import aspgpu
    aspgpu.lib()
    return aspgpu


MODES = [1, 2, 3]     # PLAIN, PACKED, BYTES


@pytest.mark.parametrize("mode", MODES)
def test_requested_view_is_used_when_it_fits(gpu, mode):
    prog = random_program(3000, 9000, program_seed(601, 0))
    P = gpu.Program(prog, view_mode=mode)
    st = P.stats()
    assert st["view_mode"] == mode and st["batch_view_mode"] == mode


def test_automatic_view_prefers_bytes(gpu):
    P = gpu.Program(random_program(3000, 9000, program_seed(601, 1)))
    assert P.stats()["view_mode"] == gpu.VIEW_BYTES


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("grid", [1, 5, 0])
@pytest.mark.parametrize("seed", range(6))
def test_propagation_fixpoint_in_every_view(gpu, mode, grid, seed):
    prog = random_program(200 + 37 * seed, 700 + 113 * seed, program_seed(602, seed))
    P = gpu.Program(prog, view_mode=mode, grid_ctas=grid)
    perm = _gpu_to_oracle_perm(prog)
    rng = np.random.default_rng(1000 + seed)
    for _ in range(3):
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


@pytest.mark.parametrize("mode", MODES)
def test_large_store_root_closure_in_every_view(gpu, mode):
    from synth.programs import large_random_program
    prog = large_random_program(0)
    P = gpu.Program(prog, view_mode=mode)
    assert P.stats()["view_mode"] == mode
    perm = _gpu_to_oracle_perm(prog)
    conflict, clo = P.propagate(np.zeros(P.n_vars, np.int8))
    oconf, oclo, _, _ = oracle.up_closure(prog, np.zeros(P.n_vars, np.int8))
    assert conflict == oconf
    if not oconf:
        assert (clo == oclo[perm]).all()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("index", [3, 77, 151, 402, 555, 918])
def test_tiny_full_enumeration_in_every_view(gpu, mode, index):
    prog = tiny_program(index)
    want = _sets(oracle.brute_force(prog))
    status, models, n = gpu.Program(prog, view_mode=mode).solve(0, cap=1 << 12)
    assert _sets(models) == want and n == len(want)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("seed", range(3))
def test_search_answers_in_every_view(gpu, mode, seed):
    prog = random_program(800, 1600, program_seed(603, seed))
    ost, _, _ = oracle.cdnl(prog, max_models=1, time_budget_s=30)
    assert ost in (oracle.SAT, oracle.UNSAT)
    st, models, _ = gpu.Program(prog, view_mode=mode, time_budget_ms=30_000).solve(1, cap=1)
    assert st == (gpu.SAT if ost == oracle.SAT else gpu.UNSAT)
    for m in models:
        assert oracle.is_answer_set(prog, m)


@pytest.mark.parametrize("mode", MODES)
def test_dependency_bitmaps_in_every_view(gpu, mode):
    """Claims made through view entries record the right variables: every
    propagated variable's bitmap is the OR over its reason (Section 4.2)."""
    prog = random_program(1500, 3600, program_seed(604, 0))
    P = gpu.Program(prog, view_mode=mode, conflict_budget=500, time_budget_ms=20_000)
    P.solve(1, cap=1)
    st = P.state(deps_words=64)
    lvl, rea, deps = st["level"], st["reason"], st["deps"]
    W = deps.shape[1]
    for v in st["trail"]:
        L = int(lvl[v])
        if L <= 1 or rea[v] in (gpu.R_DECISION, gpu.R_COMPLETE):
            continue
        nw = min(W, (L + 63) // 64)
        want = np.zeros(nw, np.uint64)
        for lit in P.nogood(int(rea[v])):
            u = lit >> 1
            if u == v or lvl[u] <= 1:
                continue
            want |= deps[u, :nw] & _mask(min(W, (int(lvl[u]) + 63) // 64), nw)
        assert (deps[v, :nw] == want).all(), v


@pytest.mark.parametrize("mode", MODES)
def test_batch_in_every_view(gpu, mode):
    progs = batch_programs(10, rules_per_atom=2, lo=50, hi=1500, config_id=605)
    P = [gpu.Program(p, view_mode=mode, time_budget_ms=20_000) for p in progs]
    st, nm, models = gpu.solve_batch(P, max_models_each=1, cap_each=1)
    for i, p in enumerate(progs):
        ost, _, _ = oracle.cdnl(p, max_models=1, time_budget_s=30)
        assert ost in (oracle.SAT, oracle.UNSAT)
        assert st[i] == (gpu.SAT if ost == oracle.SAT else gpu.UNSAT), i
        for m in models[i]:
            assert oracle.is_answer_set(p, m)


@pytest.mark.parametrize("fr", [1, 2, 3])
@pytest.mark.parametrize("mode", [1, 2, 3])
@pytest.mark.parametrize("grid", [1, 5, 0])
@pytest.mark.parametrize("seed", range(5))
def test_frontier_propagation_reaches_the_same_fixpoint(gpu, fr, mode, grid, seed):
    """Rounds that check only the nogoods (fr = 1) or the bucket units (fr =
    2) of the last round's assignments (full sweeps after (re)starts) reach
    the unique UP closure."""
    prog = random_program(300 + 53 * seed, 900 + 151 * seed, program_seed(608, seed))
    P = gpu.Program(prog, view_mode=mode, grid_ctas=grid, frontier=fr)
    perm = _gpu_to_oracle_perm(prog)
    rng = np.random.default_rng(3000 + seed)
    for _ in range(3):
        partial = np.zeros(P.n_vars, np.int8)
        k = int(rng.integers(1, 25))
        pick = rng.choice(prog.n_atoms, size=k, replace=False)
        partial[pick] = rng.choice([-1, 1], size=k)
        conflict, clo = P.propagate(partial)
        opart = np.zeros(P.n_vars, np.int8)
        opart[perm] = partial
        oconf, oclo, _, _ = oracle.up_closure(prog, opart)
        assert conflict == oconf
        if not oconf:
            assert (clo == oclo[perm]).all()


@pytest.mark.parametrize("fr", [1, 2, 3])
@pytest.mark.parametrize("index", [3, 77, 151, 402, 555, 918])
def test_frontier_tiny_full_enumeration(gpu, fr, index):
    prog = tiny_program(index)
    want = _sets(oracle.brute_force(prog))
    status, models, n = gpu.Program(prog, frontier=fr).solve(0, cap=1 << 12)
    assert _sets(models) == want and n == len(want)


@pytest.mark.parametrize("fr", [1, 2, 3])
@pytest.mark.parametrize("seed", range(4))
def test_frontier_search_answers_and_bitmaps(gpu, fr, seed):
    prog = random_program(700, 1400, program_seed(609, seed))
    ost, _, _ = oracle.cdnl(prog, max_models=1, time_budget_s=30)
    assert ost in (oracle.SAT, oracle.UNSAT)
    P = gpu.Program(prog, frontier=fr, time_budget_ms=30_000)
    st, models, _ = P.solve(1, cap=1)
    assert st == (gpu.SAT if ost == oracle.SAT else gpu.UNSAT)
    for m in models:
        assert oracle.is_answer_set(prog, m)
    s = P.state(deps_words=64)
    lvl, rea, deps = s["level"], s["reason"], s["deps"]
    W = deps.shape[1]
    for v in s["trail"]:
        L = int(lvl[v])
        if L <= 1 or rea[v] in (gpu.R_DECISION, gpu.R_COMPLETE):
            continue
        nw = min(W, (L + 63) // 64)
        want = np.zeros(nw, np.uint64)
        for lit in P.nogood(int(rea[v])):
            u = lit >> 1
            if u == v or lvl[u] <= 1:
                continue
            want |= deps[u, :nw] & _mask(min(W, (int(lvl[u]) + 63) // 64), nw)
        assert (deps[v, :nw] == want).all(), v


@pytest.mark.parametrize("fr", [1, 2, 3])
def test_frontier_batch(gpu, fr):
    progs = batch_programs(10, rules_per_atom=2, lo=50, hi=1500, config_id=610)
    P = [gpu.Program(p, frontier=fr, time_budget_ms=20_000) for p in progs]
    st, nm, models = gpu.solve_batch(P, max_models_each=1, cap_each=1)
    for i, p in enumerate(progs):
        ost, _, _ = oracle.cdnl(p, max_models=1, time_budget_s=30)
        assert ost in (oracle.SAT, oracle.UNSAT)
        assert st[i] == (gpu.SAT if ost == oracle.SAT else gpu.UNSAT), i
        for m in models[i]:
            assert oracle.is_answer_set(p, m)
