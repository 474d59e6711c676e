"""The workloads at their stated sizes against the oracle (needs a GB300).

- Tiny programs (20 atoms, 40 rules, 3 constraints), all 1000 seeds: every
  answer set, one program at a time and batched, equal as sets to the
  oracle's brute force over 2^20 interpretations (stored in
  tests/golden/tiny_answer_sets.json by a script that calls only the oracle).
- 3-colouring of G(n, 4.5/(n-1)), seeds 0..9, up to 1000 answer sets: each
  model decodes to a proper colouring (checked against the graph, not by a
  solver) and passes the oracle's reduct check; the count is min(1000, the
  number of answer sets), compared with the oracle's count when the
  enumeration ends below 1000.  The oracle decides these graphs up to a few
  hundred vertices; at n = 2000 neither it nor this solver finds a colouring
  within minutes (the average degree 4.5 lies just below the 3-colouring
  threshold), so n = 2000 runs with a time budget and any model it returns is
  checked.
- Batches of 4096 random programs (atoms log-uniform in [200, 20000]): with 4
  rules per atom, and the decidable sub-family with 2 rules per atom.  The
  oracle runs on every host core; wherever both decide, SAT/UNSAT agree, and
  every model passes the reduct check.
- The large random program (100k atoms, 400k rules), seeds 0..4, with a time
  budget: any model passes the reduct check."""
import multiprocessing as mp
import json
import os

import numpy as np
import pytest

import oracle
from synth.programs import batch_programs, coloring_graph, coloring_program, large_random_program, tiny_program

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


def _masks(models, n):
    w = np.int64(1) << np.arange(n, dtype=np.int64)
    return sorted(int((np.asarray(m[:n], np.int64) * w).sum()) for m in models)


def _golden():
    data = json.load(open(os.path.join(GOLDEN, "tiny_answer_sets.json")))
    return {r["index"]: r["answer_sets"] for r in data["programs"]}


# ------------------------------------------------------------ tiny programs

@pytest.mark.parametrize("fr", [0, 2, 3])
def test_tiny_programs_all_1000_seeds(gpu, fr):
    golden = _golden()
    assert sorted(golden) == list(range(1000))
    models_total = 0
    for i in range(1000):
        prog = tiny_program(i)
        P = gpu.Program(prog, frontier=fr)
        status, models, n = P.solve(0, cap=256)
        want = golden[i]
        assert _masks(models, prog.n_atoms) == want and n == len(want), i
        assert status == (gpu.SAT if want else gpu.UNSAT), i
        models_total += n
        P.close()
    print(f"tiny programs: 1000 seeds, {models_total} answer sets, all equal to brute force")


@pytest.mark.parametrize("fr", [0, 2])
def test_tiny_programs_all_1000_seeds_batched(gpu, fr):
    golden = _golden()
    progs = [tiny_program(i) for i in range(1000)]
    P = [gpu.Program(p, frontier=fr) for p in progs]
    st, nm, models = gpu.solve_batch(P, max_models_each=0, cap_each=64)
    for i, p in enumerate(progs):
        want = golden[i]
        assert _masks(models[i], p.n_atoms) == want and nm[i] == len(want), i
        assert st[i] == (gpu.SAT if want else gpu.UNSAT), i


# ------------------------------------------------------------ 3-colouring

def _check_colourings(prog, edges, n, models):
    seen = set()
    for m in models:
        col = np.asarray(m[:3 * n], bool).reshape(n, 3)
        assert (col.sum(1) == 1).all(), "a vertex without exactly one colour"
        colour = col.argmax(1)
        assert (colour[edges[:, 0]] != colour[edges[:, 1]]).all(), "an edge with equal colours"
        neg = np.asarray(m[3 * n:6 * n], bool).reshape(n, 3)
        assert (neg == ~col).all()
        assert oracle.is_answer_set(prog, m)
        seen.add(np.asarray(m, bool).tobytes())
    assert len(seen) == len(models)


@pytest.mark.parametrize("n", [100, 200])
@pytest.mark.parametrize("seed", range(10))
def test_colouring_up_to_1000_answer_sets(gpu, n, seed):
    edges = coloring_graph(n, 4.5, seed)
    prog = coloring_program(n, 4.5, seed_index=seed, edges=edges)
    P = gpu.Program(prog, time_budget_ms=60_000, learning=gpu.LEARN_RES)
    st, models, cnt = P.solve(1000, cap=1000)
    assert st in (gpu.SAT, gpu.UNSAT), "no answer within the time budget"
    assert len(models) == min(cnt, 1000)
    _check_colourings(prog, edges, n, models)
    if cnt < 1000:
        # the enumeration ended: exactly cnt answer sets exist
        assert st == (gpu.SAT if cnt else gpu.UNSAT)
        ost, om, _ = oracle.cdnl(prog, max_models=1001, time_budget_s=120)
        assert ost in (oracle.SAT, oracle.UNSAT)
        assert len(om) == cnt
    else:
        assert cnt == 1000 and st == gpu.SAT


@pytest.mark.parametrize("seed", range(10))
def test_colouring_n2000_within_a_time_budget(gpu, seed):
    edges = coloring_graph(2000, 4.5, seed)
    prog = coloring_program(2000, 4.5, seed_index=seed, edges=edges)
    P = gpu.Program(prog, time_budget_ms=5_000, learning=gpu.LEARN_RES, restart_conflicts=64)
    st, models, cnt = P.solve(1000, cap=1000)
    s = P.stats()
    print(f"colouring n=2000 seed {seed}: status {st}, {cnt} models, {s['conflicts']} conflicts, "
          f"{s['decisions']} decisions in {s['ns_total'] / 1e9:.1f} s")
    _check_colourings(prog, edges, 2000, models)


# ------------------------------------------------------------ batches

def _oracle_status(args):
    prog, budget_s = args
    st, models, _ = oracle.cdnl(prog, max_models=1, time_budget_s=budget_s)
    return st


def _oracle_on_all_cores(progs, budget_s):
    ctx = mp.get_context("spawn")
    with ctx.Pool(os.cpu_count() or 1) as pool:
        return np.array(pool.map(_oracle_status, [(p, budget_s) for p in progs], chunksize=8))


@pytest.mark.parametrize("rules_per_atom,conflicts,oracle_s", [(4, 100, 0.2), (2, 2000, 2.0)])
def test_batch_4096_statuses_equal_the_oracle(gpu, rules_per_atom, conflicts, oracle_s):
    progs = batch_programs(4096, rules_per_atom=rules_per_atom, config_id=4)
    want = _oracle_on_all_cores(progs, oracle_s)
    P = [gpu.Program(p, conflict_budget=conflicts, time_budget_ms=int(1000 * oracle_s) + 3000, deps_levels=1024,
                     learned_capacity=1 << 20) for p in progs]
    st, nm, models = gpu.solve_batch(P, max_models_each=1, cap_each=1)
    decided = (st == gpu.SAT) | (st == gpu.UNSAT)
    odecided = (want == oracle.SAT) | (want == oracle.UNSAT)
    both = decided & odecided
    assert (st[both] == want[both]).all(), np.nonzero(st[both] != want[both])[0][:10]
    for i in np.nonzero(st == gpu.SAT)[0]:
        assert oracle.is_answer_set(progs[i], models[i][0]), i
    print(f"4096 programs, {rules_per_atom} rules per atom: GPU decided {int(decided.sum())} "
          f"({int((st == gpu.SAT).sum())} SAT), oracle decided {int(odecided.sum())}, "
          f"both {int(both.sum())}, 0 mismatches")
    if rules_per_atom == 2:
        assert decided.sum() >= 0.85 * 4096


# ------------------------------------------------------------ large program

@pytest.mark.parametrize("seed", range(5))
def test_large_program_seeds(gpu, seed):
    prog = large_random_program(seed)
    P = gpu.Program(prog, time_budget_ms=5_000)
    st, models, cnt = P.solve(1, cap=1)
    s = P.stats()
    print(f"100k/400k seed {seed}: status {st}, {s['conflicts']} conflicts, {s['decisions']} decisions, "
          f"max level {s['max_level']}")
    assert st in (gpu.SAT, gpu.UNSAT, gpu.UNKNOWN)
    for m in models:
        assert oracle.is_answer_set(prog, m)
