"""Cross-check of the oracle's two answer-set computations (test
infrastructure): O2, the simple CDNL solver, against O1, brute force over
all 2^20 interpretations, on seeded 20-atom programs (40 rules, 3
constraints, the tiny-program family; --rules and --constraints give denser
programs of the same generator, with more conflicts per search).  Sets of
answer sets, counts and SAT/UNSAT must agree on every program.

    python -m oracle.crosscheck --count 10000 --workers 16
    python -m oracle.crosscheck --count 10000 --rules 60 --constraints 4

Prints one JSON line: programs checked, disagreements (with their indices),
answer-set total, UNSAT programs, seconds.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time


def _one(job):
    index, n_rules, n_constraints = job
    import oracle
    from synth.programs import tiny_program
    prog = tiny_program(index, n_rules=n_rules, n_constraints=n_constraints)
    bf = {bytes(m) for m in oracle.brute_force(prog)}
    status, models, _ = oracle.cdnl(prog)
    got = [bytes(m) for m in models]
    ok = set(got) == bf and len(got) == len(bf) and status == (oracle.SAT if bf else oracle.UNSAT)
    return index, ok, len(bf)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=10000)
    ap.add_argument("--first", type=int, default=0)
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--rules", type=int, default=40)
    ap.add_argument("--constraints", type=int, default=3)
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import oracle
    oracle.build()
    t0 = time.time()
    bad, n_sets, unsat, done = [], 0, 0, 0
    with mp.get_context("spawn").Pool(a.workers) as pool:
        for index, ok, k in pool.imap_unordered(_one, [(i, a.rules, a.constraints) for i in
                                                            range(a.first, a.first + a.count)], chunksize=8):
            done += 1
            n_sets += k
            unsat += k == 0
            if not ok:
                bad.append(index)
    print(json.dumps({"family": f"tiny programs: 20 atoms, {a.rules} rules, {a.constraints} constraints",
                      "first_index": a.first, "programs": done, "disagreements": len(bad),
                      "disagreeing_indices": bad[:50], "answer_sets": n_sets, "unsat_programs": unsat,
                      "seconds": round(time.time() - t0, 1)}))
    return 0 if not bad else 1


if __name__ == "__main__":
    sys.exit(main())
