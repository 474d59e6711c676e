"""Learned decision heuristic (needs a GB300): MLP numerics against a CPU
forward pass, one training step against a CPU gradient step, decision
traces, and unchanged answers when the heuristic steers the search."""
import numpy as np
import pytest

import oracle
from synth.programs import program_seed, random_program, tiny_program

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1909_01786_gb300 import aspgpu, heuristic
    aspgpu.lib()
    return aspgpu, heuristic


def _bf16(w):
    """Round float32 to bf16 (nearest even) and back, as the device does."""
    u = np.asarray(w, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def test_mlp_scores_match_cpu_forward_within_fp32_bound(gpu):
    aspgpu, H = gpu
    rng = np.random.default_rng(0)
    w = H.init_weights(3)
    w[-1] = 0.25
    X = rng.normal(0, 2, (5000, 16)).astype(np.float32)
    got = aspgpu.mlp_score(w, X).astype(np.float64)
    wb = _bf16(w)
    want = H.forward_np(wb, X)
    # fp32 accumulation of 16 + 64 terms: bound by the magnitudes summed
    W1, b1, w2, b2 = (a.astype(np.float64) for a in H.split(wb))
    mag = np.abs(X) @ np.abs(W1).T + np.abs(b1)
    bound = 1e-5 * (np.maximum(mag, 1.0) @ np.abs(w2) + abs(b2[0]) + 1.0)
    assert np.all(np.abs(got - want) <= bound)


def test_one_training_step_matches_cpu_gradient_step(gpu):
    aspgpu, H = gpu
    rng = np.random.default_rng(1)
    n = 1000                                   # one minibatch, one update
    X = rng.normal(0, 1, (n, 16)).astype(np.float32)
    y = (rng.random(n) < 0.4).astype(np.float32)
    w0 = H.init_weights(4)
    lr = 0.1
    got = aspgpu.train_mlp(X, y, w0, epochs=1, learning_rate=lr)
    # CPU reference: mean binary cross-entropy gradient, w -= lr * g
    W1, b1, w2, b2 = (a.astype(np.float64) for a in H.split(w0))
    A = X @ W1.T + b1
    h = np.maximum(A, 0)
    p = 1 / (1 + np.exp(-(h @ w2 + b2[0])))
    d = (p - y) / n
    gw2 = h.T @ d
    gb2 = d.sum()
    dh = (d[:, None] * w2[None, :]) * (A > 0)
    gW1 = dh.T @ X
    gb1 = dh.sum(0)
    g = np.concatenate([gW1.reshape(-1), gb1, gw2, [gb2]])
    want = w0.astype(np.float64) - lr * g
    assert np.allclose(got, want, rtol=1e-4, atol=1e-6)


def test_training_learns_a_separable_rule(gpu):
    aspgpu, H = gpu
    rng = np.random.default_rng(2)
    X = rng.normal(0, 1, (20000, 16)).astype(np.float32)
    y = (X[:, 3] - 0.5 * X[:, 7] > 0).astype(np.float32)
    w = aspgpu.train_mlp(X, y, H.init_weights(5), epochs=40, learning_rate=0.2)
    acc = np.mean((H.forward_np(w, X) > 0) == (y > 0.5))
    assert acc > 0.95


def test_decision_traces_are_labelled_by_the_answer_set(gpu):
    aspgpu, H = gpu
    prog = random_program(3000, 5000, program_seed(501, 1))       # satisfiable
    P = aspgpu.Program(prog, trace_capacity=4000)
    st, models, n = P.solve(1, cap=1)
    assert st == aspgpu.SAT
    X, y, js = P.trace(4000, with_rules=True)
    assert X.shape[0] > 0 and np.isfinite(X).all()
    assert (X[:, 7] == 1.0).all()              # the constant feature
    assert set(np.unique(y)) <= {0, 1}         # all labelled: a model was found
    # label = the sampled rule's body holds in the model, recomputed on the CPU
    headed = np.nonzero(prog.head >= 0)[0]
    order = headed[np.argsort(prog.head[headed], kind="stable")]   # solver rule j -> input rule
    rules = list(prog.rules())
    M = models[0].astype(bool)
    for j, lab in zip(js, y):
        h, pos, neg = rules[order[j]]
        body = all(M[a] for a in pos) and not any(M[a] for a in neg)
        assert lab == int(body)


@pytest.mark.parametrize("index", list(range(0, 200, 23)))
def test_learned_heuristic_leaves_answer_sets_unchanged(gpu, index):
    aspgpu, H = gpu
    prog = tiny_program(index)
    w = H.init_weights(index)
    want = {frozenset(np.nonzero(m)[0].tolist()) for m in oracle.brute_force(prog)}
    _, models, n = aspgpu.Program(prog, heuristic=2, mlp_weights=w).solve(0, cap=4096)
    assert {frozenset(np.nonzero(m)[0].tolist()) for m in models} == want and n == len(want)


@pytest.mark.parametrize("seed", range(4))
def test_learned_heuristic_sat_agreement(gpu, seed):
    aspgpu, H = gpu
    prog = random_program(600, 1200, program_seed(502, seed))
    ost, _, _ = oracle.cdnl(prog, max_models=1, time_budget_s=30)
    assert ost in (oracle.SAT, oracle.UNSAT)
    st, models, _ = aspgpu.Program(prog, heuristic=2, mlp_weights=H.init_weights(seed),
                                   time_budget_ms=30_000).solve(1, cap=1)
    assert st == (aspgpu.SAT if ost == oracle.SAT else aspgpu.UNSAT)
    for m in models:
        assert oracle.is_answer_set(prog, m)


@pytest.mark.parametrize("index", list(range(3, 200, 29)))
def test_static_learned_order_leaves_answer_sets_unchanged(gpu, index):
    aspgpu, H = gpu
    prog = tiny_program(index)
    want = {frozenset(np.nonzero(m)[0].tolist()) for m in oracle.brute_force(prog)}
    _, models, n = aspgpu.Program(prog, heuristic=3, mlp_weights=H.init_weights(index)).solve(0, cap=4096)
    assert {frozenset(np.nonzero(m)[0].tolist()) for m in models} == want and n == len(want)


@pytest.mark.parametrize("seed", range(3))
def test_static_learned_order_sat_agreement(gpu, seed):
    aspgpu, H = gpu
    prog = random_program(600, 1200, program_seed(503, seed))
    ost, _, _ = oracle.cdnl(prog, max_models=1, time_budget_s=30)
    assert ost in (oracle.SAT, oracle.UNSAT)
    st, models, _ = aspgpu.Program(prog, heuristic=3, mlp_weights=H.init_weights(seed),
                                   time_budget_ms=30_000).solve(1, cap=1)
    assert st == (aspgpu.SAT if ost == oracle.SAT else aspgpu.UNSAT)
    for m in models:
        assert oracle.is_answer_set(prog, m)


def test_static_features_hold_the_search_state_at_its_start(gpu):
    aspgpu, H = gpu
    X = np.random.default_rng(3).normal(0, 1, (50, 16)).astype(np.float32)
    Z = H.static_features(X)
    assert (Z[:, :8] == X[:, :8]).all() and (Z[:, 9] == X[:, 2]).all()
    assert (Z[:, [8, 10, 12, 13, 14, 15]] == 0).all() and np.allclose(Z[:, 11], 1 / 64)
