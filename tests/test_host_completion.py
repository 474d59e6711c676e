"""The library's host-side completion (A1: the nogood store built from a
program, Section 2) and its static decision scores (Section 4, Decision),
checked without a GPU through asp_debug_completion / asp_debug_rule_scores.

- The nogoods equal, as a multiset, the oracle's own completion (an
  independent encoder) mapped to the library's variables, for the full and
  the compact completion, on hand programs with duplicate body atoms,
  self-loops, facts, atoms without rules, repeated and empty constraints, on
  tiny programs, random programs, long support nogoods and colourings.
- Counts follow the closed forms (6 + k nogoods and 11 + 3k literals per
  rule with k body atoms), and the store's order is by length, then long,
  unit and empty nogoods.
- The rule order is the headed rules sorted by head atom, ties in input
  order; the occurrence score is the number of the head atom's literals in
  the completion and the Jeroslow-Wang score the sum of 2^(16 - |delta|) over
  the nogoods holding F b_j or F head(j), both recomputed here from the
  oracle's completion."""
import ctypes as C
from collections import Counter

import numpy as np
import pytest

import oracle
from paper_1909_01786_gb300 import aspgpu
from synth.programs import coloring_program, from_rules, program_seed, random_program, tiny_program

from test_gpu_full_size import _oracle_to_library


def _nogood_multiset(off, lits):
    return Counter(tuple(sorted(lits[off[i]:off[i + 1]].tolist())) for i in range(off.shape[0] - 1))


def _oracle_in_library_encoding(prog, compact=False):
    nv, off, lits = oracle.completion(prog, compact=compact)
    o2g = _oracle_to_library(prog, nv)
    enc = (2 * o2g[np.abs(lits).astype(np.int64) - 1] + (lits < 0)).astype(np.int64)
    return nv, off, enc


HAND = {
    "even loop": (2, [(0, [], [1]), (1, [], [0])]),
    "odd loop": (1, [(0, [], [0])]),
    "positive loop and constraint": (2, [(0, [1], []), (1, [0], []), (-1, [], [0])]),
    "facts and an atom without rules": (4, [(0, [], []), (1, [0], []), (2, [0, 1], [3])]),
    "duplicate body atoms": (3, [(0, [1, 1, 2], [2, 2]), (1, [], [0, 0]), (-1, [0, 0], [1, 1])]),
    "self-loops": (2, [(0, [0], []), (1, [1], [0]), (1, [], [1])]),
    "two empty constraints": (2, [(0, [], [1]), (-1, [], []), (-1, [], [])]),
    "constraint with p and not p": (2, [(0, [], [1]), (-1, [0], [0])]),
    "many rules for one atom (long support nogood)": (3, [(0, [1], [2])] * 9 + [(0, [2], [1])] * 9 + [(1, [], [2])]),
}


def _cases():
    for name, (n, rules) in HAND.items():
        yield name, from_rules(n, rules)
    for i in range(40):
        yield f"tiny {i}", tiny_program(i)
    for i, (n, r) in enumerate([(50, 120), (300, 1200), (2000, 8000)]):
        yield f"random {n}/{r}", random_program(n, r, program_seed(707, i))
    yield "random, 20 rules per atom", random_program(30, 600, program_seed(707, 9))
    yield "3-colouring n=60", coloring_program(60, 4.5, seed_index=1)


CASES = list(_cases())


@pytest.mark.parametrize("compact", [False, True])
@pytest.mark.parametrize("name,prog", CASES, ids=[c[0] for c in CASES])
def test_nogoods_equal_the_oracle_completion(name, prog, compact):
    nv, off, lits = aspgpu.completion(prog, compact=compact)
    onv, ooff, oenc = _oracle_in_library_encoding(prog, compact)
    assert nv == onv
    assert _nogood_multiset(off, lits) == _nogood_multiset(ooff, oenc)


@pytest.mark.parametrize("name,prog", CASES, ids=[c[0] for c in CASES])
def test_counts_and_order(name, prog):
    nv, off, lits = aspgpu.completion(prog)
    headed = prog.head >= 0
    assert nv == prog.n_atoms + 3 * int(headed.sum())
    # per headed rule with k distinct body atoms: 6 + k nogoods, 11 + 3k
    # literals; per atom one support nogood of 1 + |rules(atom)| literals;
    # per constraint one nogood of its distinct literals
    want_n = want_l = 0
    for r in range(prog.head.shape[0]):
        pos = set(prog.pos[prog.pos_off[r]:prog.pos_off[r + 1]].tolist())
        neg = set(prog.neg[prog.neg_off[r]:prog.neg_off[r + 1]].tolist())
        if headed[r]:
            k = len(pos) + len(neg)
            want_n += 6 + k
            want_l += 11 + 3 * k
        else:
            want_n += 1
            want_l += len(pos) + len(neg)
    want_n += prog.n_atoms
    want_l += prog.n_atoms + int(headed.sum())
    assert off.shape[0] - 1 == want_n and lits.shape[0] == want_l
    lens = np.diff(off)
    # order: lengths 2..15 non-decreasing, then longer, then units, then empty
    rank = np.where(lens == 0, 3, np.where(lens == 1, 2, np.where(lens > 15, 1, 0)))
    assert (np.diff(rank) >= 0).all()
    bucket = lens[rank == 0]
    assert (np.diff(bucket) >= 0).all()
    assert ((lits >> 1) < nv).all() and (lits >= 0).all()


@pytest.mark.parametrize("name,prog", CASES, ids=[c[0] for c in CASES])
def test_rule_order_and_static_scores(name, prog):
    idx, occ, jw = aspgpu.rule_scores(prog)
    headed = np.nonzero(prog.head >= 0)[0]
    order = headed[np.argsort(prog.head[headed], kind="stable")]
    assert np.array_equal(idx, order)
    nv, off, enc = _oracle_in_library_encoding(prog)
    var = enc >> 1
    heads = prog.head[order].astype(np.int64)
    occ_want = np.bincount(var[var < prog.n_atoms], minlength=prog.n_atoms)[heads]
    assert np.array_equal(occ.astype(np.int64), occ_want)
    # Jeroslow-Wang: sum of 2^(16 - |delta|) over the nogoods holding the
    # false literal of a variable
    lens = np.diff(off)
    weight = np.where(lens <= 16, 2.0 ** (16 - np.minimum(lens, 16)), 0.0).astype(np.int64)
    per_lit = np.repeat(weight, lens)
    neg_lit = (enc & 1) == 1
    jw_f = np.bincount(var[neg_lit], weights=per_lit[neg_lit], minlength=nv).astype(np.int64)
    b = prog.n_atoms + 3 * np.arange(order.shape[0])
    jw_want = np.minimum(jw_f[b] + jw_f[heads], 2 ** 31 - 1)
    assert np.array_equal(jw.astype(np.int64), jw_want)


def test_argument_errors_and_capacity():
    L = aspgpu.lib()
    prog = tiny_program(0)
    keep, ptrs = aspgpu._program_arrays(prog)
    nv, nn, nl = C.c_int64(), C.c_int64(), C.c_int64()
    counts = [C.byref(nv), C.byref(nn), C.byref(nl)]
    n_rules = int(prog.head.shape[0])
    assert L.asp_debug_completion(prog.n_atoms, n_rules, *ptrs, 0, *counts, None, None, 0) == 0
    off = np.zeros(nn.value + 1, np.int64)
    short = np.zeros(nl.value - 1, np.int32)
    assert L.asp_debug_completion(prog.n_atoms, n_rules, *ptrs, 0, *counts, off.ctypes.data, short.ctypes.data,
                                  short.shape[0]) == -5
    assert b"n_literals" in L.asp_last_error()
    assert L.asp_debug_completion(prog.n_atoms, n_rules, *ptrs, 0, None, None, None, None, None, 0) == -1
    bad = from_rules(2, [(5, [], [])])             # head atom 5 of a 2-atom program
    _, bptrs = aspgpu._program_arrays(bad)
    assert L.asp_debug_completion(2, 1, *bptrs, 0, *counts, None, None, 0) == -2
    assert b"range" in L.asp_last_error()
    nh = C.c_int32()
    assert L.asp_debug_rule_scores(prog.n_atoms, n_rules, *ptrs, 0, C.byref(nh), None, None, None, 0) == 0
    one = np.zeros(1, np.int32)
    assert L.asp_debug_rule_scores(prog.n_atoms, n_rules, *ptrs, 0, C.byref(nh), one.ctypes.data, None, None,
                                   1) == -5


def _raw(n_atoms, head, pos_off, pos, neg_off, neg):
    """asp_debug_completion on raw arrays (count-only call)."""
    L = aspgpu.lib()
    arrs = [np.ascontiguousarray(head, np.int32), np.ascontiguousarray(pos_off, np.int64),
            np.ascontiguousarray(pos, np.int32), np.ascontiguousarray(neg_off, np.int64),
            np.ascontiguousarray(neg, np.int32)]
    nv, nn, nl = C.c_int64(), C.c_int64(), C.c_int64()
    rc = L.asp_debug_completion(int(n_atoms), int(arrs[0].shape[0]), *[a.ctypes.data if a.size else None for a in arrs],
                                0, C.byref(nv), C.byref(nn), C.byref(nl), None, None, 0)
    return rc, L.asp_last_error().decode()


def test_program_validator_rejects_malformed_arrays():
    """The argument checks asp_load_ground runs before any device work
    (invalid or truncated program arrays give ASP_E_ARG / ASP_E_RANGE with a
    message, never a crash)."""
    ok = _raw(3, [0, -1], [0, 1, 2], [1, 2], [0, 0, 1], [0])
    assert ok[0] == 0
    cases = [
        ((3, [0, 5], [0, 1, 2], [1, 2], [0, 0, 1], [0]), -2, "head"),               # head out of range
        ((3, [0, -2], [0, 1, 2], [1, 2], [0, 0, 1], [0]), -2, "head"),              # head below -1
        ((3, [0, -1], [0, 1, 2], [1, 7], [0, 0, 1], [0]), -2, "body"),              # body atom out of range
        ((3, [0, -1], [0, 1, 2], [1, 2], [0, 0, 1], [-1]), -2, "body"),             # negative body atom
        ((3, [0, -1], [1, 1, 2], [1, 2], [0, 0, 1], [0]), -1, "start at 0"),        # offsets not from 0
        ((3, [0, -1], [0, 2, 1], [1, 2], [0, 0, 1], [0]), -1, "monotone"),          # offsets decreasing
        ((-1, [0, -1], [0, 1, 2], [1, 2], [0, 0, 1], [0]), -1, "negative"),         # negative atom count
    ]
    for args, code, word in cases:
        rc, msg = _raw(*args)
        assert rc == code, (args, rc, msg)
        assert word in msg, (word, msg)
    # a positive body referenced by offsets but not given
    L = aspgpu.lib()
    head = np.array([0], np.int32)
    off1 = np.array([0, 1], np.int64)
    off0 = np.array([0, 0], np.int64)
    nv, nn, nl = C.c_int64(), C.c_int64(), C.c_int64()
    rc = L.asp_debug_completion(2, 1, head.ctypes.data, off1.ctypes.data, None, off0.ctypes.data, None, 0,
                                C.byref(nv), C.byref(nn), C.byref(nl), None, None, 0)
    assert rc == -1 and "null" in L.asp_last_error().decode()
