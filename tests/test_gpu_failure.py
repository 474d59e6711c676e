"""Failure detection without a GPU fault (needs a GB300).

- The persistent kernel's grid barrier gives up after a bounded wait: with a
  one-second limit and one CTA that does not arrive (it waits, bounded, on a
  flag nothing sets), the solve returns ASP_E_DEVICE within seconds, and the
  next solves on the same context give the oracle's answer.
- A device allocation that fails (injected on the host) gives ASP_E_OOM and
  leaves nothing allocated; the next load succeeds.
- A learned-nogood store too small for the search gives ASP_E_DEVICE."""
import time

import pytest

import oracle
from synth.programs import program_seed, random_program, tiny_program

pytestmark = pytest.mark.gpu

ASP_E_OOM, ASP_E_DEVICE = -3, -6


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1909_01786_gb300 import aspgpu
    aspgpu.lib()
    return aspgpu


def _oracle_status(prog):
    st, _, _ = oracle.cdnl(prog, max_models=1, time_budget_s=60)
    assert st in (oracle.SAT, oracle.UNSAT)
    return st


@pytest.mark.parametrize("stall_cta", [1, 77])
def test_barrier_timeout_is_reported_and_the_context_survives(gpu, stall_cta):
    import torch
    # large enough for a grid of one CTA per SM (the grid grows with the
    # store), 2 rules per atom so that the oracle decides it quickly
    prog = random_program(12000, 24000, program_seed(901, stall_cta))
    want = _oracle_status(prog)
    P = gpu.Program(prog, time_budget_ms=30_000)
    if stall_cta >= torch.cuda.get_device_properties(0).multi_processor_count:
        pytest.skip("fewer CTAs in the grid")
    L = gpu.lib()
    assert L.asp_debug_barrier(P.handle, stall_cta, 1000) == 0
    t0 = time.perf_counter()
    with pytest.raises(gpu.AspError) as e:
        P.solve(1, cap=1)
    dt = time.perf_counter() - t0
    assert e.value.code == ASP_E_DEVICE
    assert dt < 15.0, dt
    torch.cuda.synchronize()                     # the context still answers
    assert L.asp_debug_barrier(P.handle, -1, 0) == 0
    st, models, _ = P.solve(1, cap=1)
    assert st == (gpu.SAT if want == oracle.SAT else gpu.UNSAT)
    for m in models:
        assert oracle.is_answer_set(prog, m)
    # a program loaded afterwards solves as usual too
    tiny = tiny_program(5)
    want_sets = {bytes(m) for m in oracle.brute_force(tiny)}
    _, tm, n = gpu.Program(tiny).solve(0, cap=64)
    assert {bytes(m) for m in tm} == want_sets and n == len(want_sets)


def test_barrier_limit_restored_by_default(gpu):
    prog = random_program(300, 700, program_seed(901, 9))
    P = gpu.Program(prog)
    L = gpu.lib()
    assert L.asp_debug_barrier(P.handle, 10_000_000, 1000) == -1   # not a CTA of the grid
    assert L.asp_debug_barrier(P.handle, -1, 0) == 0
    st, _, _ = P.solve(1, cap=1)
    assert st in (gpu.SAT, gpu.UNSAT)


def test_failed_allocation_gives_out_of_memory(gpu):
    prog = random_program(300, 600, program_seed(902, 0))
    L = gpu.lib()
    failures = 0
    try:
        for nth in range(1, 64):
            assert L.asp_debug_fail_alloc(nth) == 0
            try:
                P = gpu.Program(prog, torch_memory=False)   # cudaMalloc / cudaFree
            except gpu.AspError as e:
                assert e.code == ASP_E_OOM, (nth, e.code)
                assert b"allocation" in L.asp_last_error()
                failures += 1
                continue
            P.close()
            break
    finally:
        L.asp_debug_fail_alloc(0)
    assert failures >= 10, failures                # every allocation of the load was tried
    st, _, _ = gpu.Program(prog, torch_memory=False).solve(1, cap=1)  # nothing left armed
    assert st in (gpu.SAT, gpu.UNSAT, gpu.UNKNOWN)


def test_learned_store_overflow_is_reported(gpu):
    prog = random_program(2000, 6000, program_seed(903, 0))      # 3 rules per atom: conflicts come early
    P = gpu.Program(prog, learned_capacity=64, conflict_budget=1000)
    with pytest.raises(gpu.AspError) as e:
        P.solve(1, cap=1)
    assert e.value.code == ASP_E_DEVICE
    # the same program with room to learn still solves
    Q = gpu.Program(prog, conflict_budget=1000)
    st, _, _ = Q.solve(1, cap=1)
    assert st in (gpu.SAT, gpu.UNSAT, gpu.UNKNOWN)
