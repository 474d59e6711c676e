"""Write tiny_answer_sets.json: every answer set of the 1000 tiny random
programs (20 atoms, 40 rules, 3 constraints; synth.programs.tiny_program,
indices 0..999), found by the oracle's brute force over all 2^20
interpretations (oracle.brute_force: M is an answer set iff M is the least
model of the reduct of the program w.r.t. M and violates no constraint --
Section 1 of the paper, "Answer Set Programming").

Each program is stored with a digest of its rule arrays, so a change of the
generator shows up as a mismatch instead of a wrong expectation.  Only the
oracle computes the stored values.

    python tests/golden/make_tiny_answer_sets.py [--workers N]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "tiny_answer_sets.json")
COUNT = 1000


def program_digest(prog) -> str:
    h = hashlib.sha256()
    for a in (prog.head, prog.pos_off, prog.pos, prog.neg_off, prog.neg):
        h.update(a.astype("<i8").tobytes())
    return h.hexdigest()[:16]


def _one(index):
    import numpy as np
    import oracle
    from synth.programs import tiny_program
    prog = tiny_program(index)
    models = oracle.brute_force(prog)
    masks = sorted(int(np.sum(m.astype(np.int64) << np.arange(prog.n_atoms, dtype=np.int64))) for m in models)
    return index, program_digest(prog), masks


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(a.workers) as pool:
        rows = sorted(pool.map(_one, range(COUNT)))
    out = {
        "about": "All answer sets of tiny_program(i), i = 0..999 (20 atoms, 40 rules, 3 two-literal "
                 "constraints), by the oracle's brute force over 2^20 interpretations with the reduct "
                 "least-model check (Section 1 of arXiv 1909.01786). Each answer set is a bitmask: bit a "
                 "is atom a. digest = sha256 of the program's rule arrays (first 16 hex digits).",
        "writer": "tests/golden/make_tiny_answer_sets.py (calls only oracle/)",
        "programs": [{"index": i, "digest": d, "answer_sets": m} for i, d, m in rows],
    }
    with open(OUT, "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")
    n_sets = sum(len(r[2]) for r in rows)
    print(f"wrote {OUT}: {COUNT} programs, {n_sets} answer sets, "
          f"{sum(1 for r in rows if r[2])} with at least one")


if __name__ == "__main__":
    main()
