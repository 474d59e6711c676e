"""3-colouring of G(n, average degree 4.5), up to 1000 answer sets (needs a
GB300).  Every answer set must decode to a proper 3-colouring of the graph
(a check independent of the solver and of the oracle's CDNL) and pass the
oracle's reduct check; the count is min(1000, number of answer sets).  At
n = 2000 this family is beyond this solver within minutes (no answer set in
240 s), so the enumeration is checked on graphs of 60-150 vertices."""
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


@pytest.mark.parametrize("n,seed_index", [(60, 0), (90, 1), (150, 2)])
def test_enumerates_proper_colourings(gpu, n, seed_index):
    edges = coloring_graph(n, 4.5, seed_index)
    prog = coloring_program(n, 4.5, seed_index=seed_index, edges=edges)
    st, models, cnt = gpu.Program(prog, time_budget_ms=60_000).solve(1000, cap=1000)
    assert st in (gpu.SAT, gpu.UNSAT)
    if st == gpu.UNSAT:
        # the search space was exhausted: fewer than 1000 answer sets exist,
        # and the oracle (when it finishes) counts the same number
        assert cnt < 1000
        ost, om, _ = oracle.cdnl(prog, max_models=cnt + 1, time_budget_s=120)
        if ost in (oracle.SAT, oracle.UNSAT) and len(om) <= cnt:
            assert len(om) == cnt
    else:
        assert cnt == 1000
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
