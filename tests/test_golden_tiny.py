"""The stored answer sets of the 1000 tiny programs (no GPU).

The file is written by tests/golden/make_tiny_answer_sets.py from the
oracle's brute force alone.  Here: each stored program digest matches the
generator's program today, and a sample of entries equals a fresh brute
force (including programs with and without answer sets)."""
import json
import os
import sys

import numpy as np

import oracle
from synth.programs import tiny_program

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
from make_tiny_answer_sets import program_digest  # noqa: E402

DATA = json.load(open(os.path.join(HERE, "golden", "tiny_answer_sets.json")))


def test_every_program_digest_matches_the_generator():
    rows = DATA["programs"]
    assert [r["index"] for r in rows] == list(range(1000))
    for r in rows:
        assert program_digest(tiny_program(r["index"])) == r["digest"], r["index"]


def test_sample_equals_a_fresh_brute_force():
    rows = {r["index"]: r for r in DATA["programs"]}
    sat = [i for i in rows if rows[i]["answer_sets"]][:3]
    unsat = [i for i in rows if not rows[i]["answer_sets"]][:2]
    for i in sat + unsat:
        prog = tiny_program(i)
        models = oracle.brute_force(prog)
        w = np.int64(1) << np.arange(prog.n_atoms, dtype=np.int64)
        masks = sorted(int((m.astype(np.int64) * w).sum()) for m in models)
        assert masks == rows[i]["answer_sets"], i


def test_answer_sets_form_an_antichain_and_pass_the_reduct_check():
    """Answer sets of a normal program are pairwise incomparable (no one is a
    proper subset of another), and each passes the reduct check."""
    for r in DATA["programs"][:300]:
        sets = r["answer_sets"]
        for a in sets:
            for b in sets:
                assert a == b or (a & b) != a
        if sets:
            prog = tiny_program(r["index"])
            for a in sets:
                M = np.array([(a >> k) & 1 for k in range(prog.n_atoms)], np.uint8)
                assert oracle.is_answer_set(prog, M)
