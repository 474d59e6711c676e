"""The oracle's compact completion (no GPU).

For a rule with an empty positive body the unit nogood {Ft_r} fixes t_r at
the root, so {Tb_r, Ft_r} can never hold and Tt_r always holds; the compact
variant leaves that nogood out and drops Tt_r from {Fb_r, Tt_r, Tn_r}
(likewise n_r for an empty negative body).  Pins:
- closed-form counts: per rule with k distinct body atoms,
  6 + k - [B+ empty] - [B- empty] nogoods and 11 + 3k - 3([B+ empty] +
  [B- empty]) literals; constraints and atom nogoods as in the full
  completion;
- the unit-propagation closure of any partial assignment is the full
  completion's (the nogoods removed are satisfied, the literals removed are
  true, once the units have fired);
- on every interpretation of small programs extended by the definitions of
  b, t and n, a nogood is violated under the compact completion iff one is
  under the full one."""
import itertools

import numpy as np
import pytest

import oracle
from synth.programs import from_rules, program_seed, random_program, tiny_program


def _nogoods(prog, compact):
    nv, off, lits = oracle.completion(prog, compact=compact)
    return nv, [tuple(int(l) for l in lits[off[i]:off[i + 1]]) for i in range(off.shape[0] - 1)]


def _expected_counts(prog, compact):
    n_ng = n_lit = 0
    cnt = np.zeros(prog.n_atoms, np.int64)
    for r in range(prog.head.shape[0]):
        P = set(prog.pos[prog.pos_off[r]:prog.pos_off[r + 1]].tolist())
        N = set(prog.neg[prog.neg_off[r]:prog.neg_off[r + 1]].tolist())
        if prog.head[r] < 0:
            n_ng += 1
            n_lit += len(P) + len(N)
            continue
        cnt[prog.head[r]] += 1
        k = len(P) + len(N)
        e = (int(not P) + int(not N)) if compact else 0
        n_ng += 6 + k - e
        n_lit += 11 + 3 * k - 3 * e
    n_ng += prog.n_atoms
    n_lit += int((1 + cnt).sum())
    return n_ng, n_lit


@pytest.mark.parametrize("compact", [False, True])
@pytest.mark.parametrize("seed", range(8))
def test_closed_form_counts(compact, seed):
    prog = random_program(50 + 10 * seed, 150 + 20 * seed, program_seed(610, seed))
    _, ngs = _nogoods(prog, compact)
    assert (len(ngs), sum(len(n) for n in ngs)) == _expected_counts(prog, compact)


def test_counts_on_facts_and_empty_bodies():
    # a. b :- not a. c :- a.  (a fact, an empty B+, an empty B-)
    prog = from_rules(3, [(0, [], []), (1, [], [0]), (2, [0], [])])
    full = _expected_counts(prog, False)
    comp = _expected_counts(prog, True)
    assert comp == (full[0] - 4, full[1] - 12)
    _, ngs = _nogoods(prog, True)
    assert (len(ngs), sum(len(n) for n in ngs)) == comp
    b0 = 3 + 0                                  # b of the fact a.
    assert (-(b0 + 1),) in ngs                  # {Fb} alone: the fact's body always holds


@pytest.mark.parametrize("seed", range(12))
def test_closure_equals_the_full_completion(seed):
    prog = random_program(40 + 5 * seed, 120 + 15 * seed, program_seed(611, seed))
    nv, _ = _nogoods(prog, False)
    rng = np.random.default_rng(seed)
    for trial in range(6):
        partial = np.zeros(nv, np.int8)
        k = int(rng.integers(0, 8))
        pick = rng.choice(prog.n_atoms, size=k, replace=False)
        partial[pick] = rng.choice([-1, 1], size=k)
        c1, clo1, _, _ = oracle.up_closure(prog, partial)
        c2, clo2, _, _ = oracle.up_closure(prog, partial, compact=True)
        assert c1 == c2
        if not c1:
            assert (clo1 == clo2).all()


def _extended(prog, M):
    """Interpretation M over the atoms, with b_j, t_j, n_j of the oracle's
    j-th headed rule (input order) set by their definitions."""
    X = list(M)
    for r in range(prog.head.shape[0]):
        if prog.head[r] < 0:
            continue
        P = prog.pos[prog.pos_off[r]:prog.pos_off[r + 1]]
        N = prog.neg[prog.neg_off[r]:prog.neg_off[r + 1]]
        t = all(M[a] for a in P)
        n = not any(M[a] for a in N)
        X += [t and n, t, n]
    return X


def _violated(ngs, X):
    return any(all(X[abs(l) - 1] == (l > 0) for l in ng) for ng in ngs)


@pytest.mark.parametrize("index", [0, 3, 11, 40])
def test_violation_agrees_on_every_interpretation(index):
    prog = tiny_program(index, n_atoms=10, n_rules=18, n_constraints=2)
    _, full = _nogoods(prog, False)
    _, comp = _nogoods(prog, True)
    for bits in itertools.product([False, True], repeat=prog.n_atoms):
        X = _extended(prog, bits)
        assert _violated(full, X) == _violated(comp, X)
