"""Host-side helpers of bench.py (no GPU): the DRAM traffic of the roofline is
taken from the committed ncu capture only while the kernel sources hash to
the captured value and the workload is the captured one; the work ratios and
the compact summary read the line they are given."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_needs_the_captured_sources_and_workload():
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    sha, atoms, rules = t["solver_src_sha"], t["atoms"], t["rules"]
    got = bench._traffic(sha, 1e9, atoms, rules)
    assert got == t["dram_bytes_per_literal_check"] * 1e9
    assert bench._traffic(sha, 2e9, atoms, rules) == 2 * got
    assert bench._traffic("0" * 16, 1e9, atoms, rules) is None
    assert bench._traffic(sha, 1e9, atoms + 1, rules) is None
    # the capture's own figures are consistent
    per_check = (t["dram_bytes_read"] + t["dram_bytes_write"]) / t["literal_checks_in_captured_launch"]
    assert abs(per_check - t["dram_bytes_per_literal_check"]) < 1e-12


def test_source_hash_covers_the_solve_kernel_sources():
    h = bench._src_sha()
    assert len(h) == 16 and int(h, 16) >= 0


def _line():
    return {
        "value": 4.5e11, "roofline": {"frac": 0.39},
        "search": {"decisions_per_s": 2000.0, "propagations_per_s": 8.0e6, "conflicts_per_s": 270.0},
        "cpu_baseline": {"decisions_per_s": 250.0, "propagations_per_s": 2.0e6, "conflicts_per_s": 0.0},
        "big_store": {"sweep": {"frac_of_hbm": 0.86}, "solver": {"frac_of_hbm": 0.6}},
        "frontier_compare": {"full": {"decisions_per_s": 2000.0, "literal_checks_per_round": 7.7e6},
                             "nogoods": {"decisions_per_s": 1400.0, "literal_checks_per_round": 2.7e4}},
    }


def test_work_ratios_divide_the_same_rates():
    out = _line()
    r = bench._work_ratios(out)
    assert r["decisions_per_s"] == 8.0 and r["propagations_per_s"] == 4.0
    assert r["conflicts_per_s"] is None                  # no oracle rate to divide by
    assert bench._work_ratios({"search": out["search"]}) is None


def test_summary_reads_every_leg_and_tolerates_missing_ones():
    out = _line()
    out["work_vs_oracle"] = bench._work_ratios(out)
    s = bench._summary(out)
    assert s["checks_per_s"] == 4.5e11 and s["frac_hbm"] == 0.39
    assert s["big_store_sweep_frac"] == 0.86 and s["big_store_solver_frac"] == 0.6
    assert s["literal_checks_per_round"] == {"scanned_full_sweeps": 7.7e6, "necessary_occurrence_lists": 2.7e4}
    assert s["frontier_decisions_per_s"] == {"full": 2000.0, "nogoods": 1400.0}
    assert s["batched_solved"] == [None, None, None] and s["learned_speedup"] == [None, None]
    json.dumps(s)
