"""Batched solving (asp_solve_batch: one launch, one CTA per program from a
work queue) against the CPU oracle (needs a GB300)."""
import numpy as np
import pytest

import oracle
from synth.programs import batch_programs, program_seed, random_program, tiny_program

pytestmark = pytest.mark.gpu


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


def test_batch_full_enumeration_of_tiny_programs(gpu):
    progs = [tiny_program(i) for i in range(0, 400, 13)]
    P = [gpu.Program(p) for p in progs]
    st, nm, models = gpu.solve_batch(P, max_models_each=0, cap_each=4096)
    for i, p in enumerate(progs):
        want = _sets(oracle.brute_force(p))
        assert _sets(models[i]) == want and nm[i] == len(want), i
        assert st[i] == (gpu.SAT if want else gpu.UNSAT)


def test_batch_mixed_sizes_match_oracle(gpu):
    sizes = [(40, 160), (80, 240), (150, 300), (600, 1200), (2500, 5000), (60, 240), (900, 1800), (30, 120)]
    progs = [random_program(na, nr, program_seed(401, i)) for i, (na, nr) in enumerate(sizes)]
    P = [gpu.Program(p, time_budget_ms=30_000) for p in progs]
    st, nm, models = gpu.solve_batch(P, max_models_each=2, cap_each=2)
    for i, p in enumerate(progs):
        ost, om, _ = oracle.cdnl(p, max_models=2, time_budget_s=30)
        assert ost in (oracle.SAT, oracle.UNSAT)
        assert st[i] == (gpu.SAT if ost == oracle.SAT else gpu.UNSAT), i
        assert nm[i] == len(om), i
        for m in models[i]:
            assert oracle.is_answer_set(p, m)


def test_batch_program_larger_than_the_shared_memory_view(gpu):
    """A program whose assignment does not fit a CTA's shared memory is read
    from global memory instead; results are unchanged."""
    big = random_program(60_000, 120_000, program_seed(402, 0))
    small = random_program(50, 100, program_seed(402, 1))
    P = [gpu.Program(big, time_budget_ms=60_000), gpu.Program(small)]
    st, nm, models = gpu.solve_batch(P, max_models_each=1, cap_each=1)
    for i, p in enumerate([big, small]):
        ost, _, _ = oracle.cdnl(p, max_models=1, time_budget_s=60)
        assert ost in (oracle.SAT, oracle.UNSAT)
        assert st[i] == (gpu.SAT if ost == oracle.SAT else gpu.UNSAT)
        for m in models[i]:
            assert oracle.is_answer_set(p, m)


def test_batch_equals_single_program_solves(gpu):
    """Same programs, one at a time on the whole grid vs batched: the same
    SAT/UNSAT answers and valid models."""
    progs = batch_programs(12, rules_per_atom=2, lo=100, hi=3000, config_id=403)
    single = []
    for p in progs:
        s, m, n = gpu.Program(p, time_budget_ms=20_000).solve(1, cap=1)
        single.append(s)
    P = [gpu.Program(p, time_budget_ms=20_000) for p in progs]
    st, nm, models = gpu.solve_batch(P, max_models_each=1, cap_each=1)
    for i, p in enumerate(progs):
        assert st[i] == single[i], i
        assert st[i] in (gpu.SAT, gpu.UNSAT)
        for m in models[i]:
            assert oracle.is_answer_set(p, m)


@pytest.mark.parametrize("config", [0, 1])
def test_batch_plan_configurations_and_replays(gpu, config):
    """A prepared batch (descriptors uploaded, launch captured in a CUDA
    graph) solved twice with either kernel configuration: full enumeration
    equals brute force both times."""
    progs = [tiny_program(i) for i in range(5, 400, 17)]
    P = [gpu.Program(p) for p in progs]
    plan = gpu.BatchPlan(P, max_models_each=0, cap_each=4096, config=config)
    assert plan.info()["config"] == config
    assert plan.info()["block_threads"] == (256 if config == 0 else 128)
    for _ in range(2):
        st, nm, models = plan.run()
        for i, p in enumerate(progs):
            want = _sets(oracle.brute_force(p))
            assert _sets(models[i]) == want and nm[i] == len(want), i
            assert st[i] == (gpu.SAT if want else gpu.UNSAT)
    plan.close()


def test_autotuned_batch_matches_the_oracle(gpu):
    progs = batch_programs(40, rules_per_atom=2, lo=50, hi=2000, config_id=404)
    P = [gpu.Program(p, time_budget_ms=20_000) for p in progs]
    plan = gpu.BatchPlan(P, max_models_each=1, cap_each=1)
    info = plan.info()
    assert info["config"] in (0, 1)
    # four schedules tried (two kernel configurations, full sweeps or the
    # unit frontier); the chosen one has the lowest time per program
    trials = info["trial_ns_per_program"]
    times = trials["full"] + trials["units"]
    assert all(t > 0 for t in times)
    assert trials[info["frontier"]][info["config"]] == min(times)
    st, nm, models = plan.run()
    for i, p in enumerate(progs):
        ost, _, _ = oracle.cdnl(p, max_models=1, time_budget_s=30)
        assert ost in (oracle.SAT, oracle.UNSAT)
        assert st[i] == (gpu.SAT if ost == oracle.SAT else gpu.UNSAT), i
        for m in models[i]:
            assert oracle.is_answer_set(p, m)
    plan.close()
