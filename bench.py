"""Benchmark: nogood-literal checks per second of the device-resident solver.

Workload: the large random ground program (100k atoms, 400k rules, body size
uniform 1..4, each body literal negated with probability 1/2, seed 0) --
searched for a first answer set with a conflict budget per step, because this
program family is beyond complete search in minutes (for the CPU oracle and
for this solver alike).  One step = one asp_solve of that program: initial
propagation, propagate-and-check sweeps, decisions, fwd-learning, backjumps,
completion and stability steps as they occur, until the budget or an answer.

value: literal checks (literals read and classified by the sweeps) per second
       over the K timed steps, inputs resident in HBM, L2 flushed between steps.
e2e:   the same metric through the C ABI with host buffers: asp_load_ground
       (completion built on the host, nogood store copied in) + asp_solve
       (model copied out) + asp_free per step.

Multi-GPU: the search does not shard; N ranks run N independent replicas
(whole-job value = all ranks' checks / the slowest rank's time).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "nogood-literal checks/s"
UNIT = "checks/s"
def workload(a):
    return (f"large random program: {a.atoms // 1000}k atoms, {a.rules // 1000}k rules, body 1-4, "
            "negation 0.5, seed 0; first answer set, conflict budget per step")


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--atoms", type=int, default=100_000)
    ap.add_argument("--rules", type=int, default=400_000)
    ap.add_argument("--conflicts", type=int, default=200, help="conflict budget per step")
    ap.add_argument("--view", type=int, default=0, help="sweep view layout: 0 auto, 1 plain, 2 packed, 3 bytes")
    ap.add_argument("--frontier", action="store_true", help="frontier rounds (full sweeps after backjumps)")
    ap.add_argument("--save-weights", default="", help="write the trained heuristic weights to this JSON file")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="oracle sample length")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch", type=int, default=256,
                    help="programs of the batched workload (config-4 family); 0 = skip")
    ap.add_argument("--batch-conflicts", type=int, default=2000, help="per-program conflict budget (batched leg)")
    ap.add_argument("--learned-conflicts", type=int, default=100,
                    help="per-program conflict budget of the learned-heuristic and search-option legs")
    ap.add_argument("--learned", type=int, default=256,
                    help="held-out programs for the learned-heuristic comparison; 0 = skip")
    ap.add_argument("--learned-train", type=int, default=1024, help="training programs (traces)")
    ap.add_argument("--learned-seeds", type=int, default=1, help="disjoint held-out sets evaluated")
    ap.add_argument("--no-learning-compare", action="store_true",
                    help="skip the fwd-learning vs first-UIP resolution comparison")
    ap.add_argument("--big-atoms", type=int, default=400_000,
                    help="atoms of the store-larger-than-L2 program (4 rules per atom); 0 = skip that leg")
    ap.add_argument("--big-conflicts", type=int, default=40, help="conflict budget of the in-solver leg on it")
    ap.add_argument("--tiny", type=int, default=1000, help="tiny programs enumerated (config-1 family); 0 = skip")
    ap.add_argument("--batch-ms", type=int, default=2000,
                    help="device time budget per program of the batched leg (the oracle gets the same in CPU time)")
    ap.add_argument("--batch-frontier", type=int, default=2,
                    help="propagation rounds of the one-at-a-time comparison and of an explicitly configured "
                         "batch (0 full sweeps, 2 the unit frontier); the autotuned batch chooses its own")
    ap.add_argument("--batch-rules-per-atom", type=int, default=2,
                    help="rules per atom of the batched workload (2: the family decides within the budget)")
    ap.add_argument("--sweep-only", type=int, default=0,
                    help="profiling aid: load the program and run this many standalone sweeps")
    return ap.parse_args()


def _program(a):
    from synth.programs import random_program, program_seed
    return random_program(a.atoms, a.rules, program_seed(2, 0))


def _cpu_baseline(prog, seconds):
    """The oracle's CDNL as it stands on one host core, bounded by CPU time."""
    import oracle
    t = time.perf_counter()
    _, _, st = oracle.cdnl(prog, max_models=1, time_budget_s=seconds)
    dt = time.perf_counter() - t
    return dict(value=st["literal_checks"] / dt, unit=UNIT, cores=1, kind="oracle",
                sample=f"oracle CDNL (first-UIP) on the same program for {seconds:.0f} s of CPU time: "
                       f"{st['conflicts']} conflicts, {st['decisions']} decisions, "
                       f"{st['propagations']} propagations, {st['literal_checks']} literal checks",
                propagations_per_s=st["propagations"] / dt, decisions_per_s=st["decisions"] / dt,
                conflicts_per_s=st["conflicts"] / dt)


class _Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm = sorted(float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit())
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 3 + i and r[3 + i] == "Active"})
        return dict(sm_mhz=sm[len(sm) // 2] if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=reasons, samples=len(sm))


def _plain(o):
    """numpy scalars and arrays in the JSON line"""
    if hasattr(o, "tolist"):
        return o.tolist()
    return str(o)


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def _traffic(kernel_src_sha, checks_per_launch, atoms, rules):
    """DRAM bytes per launch of the solve kernel from the committed ncu
    capture, if it was taken on the current kernel source.  The capture ran a
    shorter launch (smaller conflict budget) of the same workload; its bytes
    per literal check are scaled to this launch's checks."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except OSError:
        return None
    if t.get("solver_src_sha") != kernel_src_sha or (t.get("atoms"), t.get("rules")) != (atoms, rules):
        return None
    return t["dram_bytes_per_literal_check"] * checks_per_launch


def _src_sha():
    h = hashlib.sha256()
    for f in ("solver.cuh", "kernels.cuh", "solve.cu", "sweep.cu", "device.cuh", "store.cpp", "store.h", "api.cpp"):
        h.update(open(os.path.join(ROOT, "paper_1909_01786_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def run_reference(a, rank, world):
    if rank != 0:
        return
    prog = _program(a)
    per_step = max(a.cpu_seconds / max(a.steps, 1), 1.0)
    import oracle
    oracle.cdnl(_program_small(), max_models=1)          # load and build the oracle
    for _ in range(a.warmup):                            # untimed warm-up steps
        oracle.cdnl(prog, max_models=1, time_budget_s=per_step)
    checks = props = 0
    t0 = time.perf_counter()
    for _ in range(a.steps):
        _, _, st = oracle.cdnl(prog, max_models=1, time_budget_s=per_step)
        checks += st["literal_checks"]
        props += st["propagations"]
    dt = time.perf_counter() - t0
    v = checks / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3 / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": {"workload": workload(a) + f"; oracle bounded to {per_step:.1f} s per step"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{a.steps} steps of {per_step:.1f} s CPU time each"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "propagations_per_s": props / dt}), flush=True)


def _program_small():
    from synth.programs import random_program, program_seed
    return random_program(50, 100, program_seed(2, 1))


def aggregate_over_ranks(ms, checks, world, device):
    """Whole-job figures of N independent replicas: the slowest rank's time
    and the checks of all ranks (one all-reduce each; nothing when N = 1)."""
    if world <= 1:
        return float(ms), float(checks)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    c = torch.tensor([float(checks)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def run_ours(a, rank, world, local_rank):
    import torch
    from paper_1909_01786_gb300 import aspgpu

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    prog = _program(a)
    P = aspgpu.Program(prog, conflict_budget=a.conflicts, time_budget_ms=120_000, view_mode=a.view, frontier=a.frontier)
    words = max((prog.n_atoms + 63) // 64, 1)
    d_models = torch.zeros(words, dtype=torch.int64, device=dev)
    d_result = torch.zeros(4, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.int32, device=dev)   # 1 GiB > L2
    stream = torch.cuda.current_stream(dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    def step():
        P.solve_async(1, d_models.data_ptr(), 1, d_result.data_ptr())

    for _ in range(a.warmup):
        flush.fill_(1)
        step()
    torch.cuda.synchronize(dev)

    totals = dict(literal_checks=0, nogood_visits=0, propagations=0, decisions=0, conflicts=0, rounds=0,
                  max_level=0, learned=0, learned_literals=0,
                  ns_total=0, ns_sweep=0, ns_analysis=0, ns_decision=0, ns_stability=0,
                  ns_buckets=0, ns_learned=0, ns_barrier=0, ns_slowest_cta=0, ns_slowest_sweep=0,
                  ns_slowest_long=0, ns_slowest_buckets=0)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    statuses = []
    barrier()
    with _Clocks(local_rank) as clk:
        for i in range(a.steps):
            flush.fill_(i)
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
            torch.cuda.synchronize(dev)
            s = P.stats()
            for k in totals:
                totals[k] = max(totals[k], s[k]) if k == "max_level" else totals[k] + s[k]
            statuses.append(int(d_result[0].item()))
        barrier()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in ev)
    checks = totals["literal_checks"]
    ms, checks_all = aggregate_over_ranks(ms, checks, world, dev)
    value = checks_all / (ms / 1e3)

    # dominant kernel: the persistent solve kernel (one launch per step).
    # Algorithmic bytes: 4 B per literal read and classified plus 4 B per
    # nogood visited (the literal word and the CSR offset a store with
    # offsets would read), over the nogoods the sweeps scanned.
    peaks = _peaks()
    peak = peaks.get("hbm_gbs")
    visits = totals["nogood_visits"]
    alg_bytes = 4.0 * checks + 4.0 * visits
    achieved = alg_bytes / (ms / 1e3) / 1e9
    achieved_4b = 4.0 * checks / (ms / 1e3) / 1e9
    sha = _src_sha()
    traffic = _traffic(sha, checks / max(len(ev), 1), a.atoms, a.rules)
    store_mb = P.stats()['store_bytes'] / 1e6
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if peak else None,
                "traffic": traffic, "kernel": "solve_kernel",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peak else None,
                "bytes_per_launch": alg_bytes / max(len(ev), 1),
                "achieved_4B_per_check": achieved_4b,
                "frac_4B_per_check": (achieved_4b / peak) if peak else None,
                "regime": (f"store of {store_mb:.0f} MB stays in L2 (126 MB): the sweep is bound by L2 and "
                           "shared-memory latency, not HBM; the HBM-bound figure is the big_store leg"
                           if store_mb < 100 else f"store of {store_mb:.0f} MB streams from HBM"),
                "note": "achieved = (4 B x literal checks + 4 B x nogood visits) / kernel time (Sigma(4 len + 4) "
                        "over scanned nogoods); traffic = DRAM bytes per literal check from an ncu capture "
                        "of a 20-conflict launch of this workload x this launch's checks"}

    # sweep kernel alone: one launch loads the shared-memory views once and
    # makes K passes; per-pass time = (t(K+1) - t(1)) / K
    st = P.stats()
    sweep_bytes = 4 * (st["n_literals"] - st["n_unit_nogoods"]) + 4 * (st["n_nogoods"] - st["n_unit_nogoods"])

    def timed(passes, reps=5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        P.sweep(passes)
        e0.record(stream)
        for _ in range(reps):
            P.sweep(passes)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    K = 16
    t1, tk = timed(1), timed(K + 1)
    per_pass = (tk - t1) / K
    sweep = {"ms_per_pass": per_pass, "ms_view_load_and_one_pass": t1, "bytes_per_pass": sweep_bytes,
             "bytes_rule": "Sigma(4 len + 4) over the non-unit nogoods",
             "achieved_gbs": sweep_bytes / (per_pass / 1e3) / 1e9,
             "frac_of_hbm": (sweep_bytes / (per_pass / 1e3) / 1e9) / peak if peak else None,
             "note": (f"store of {st['store_bytes'] / 1e6:.0f} MB "
                      + ("is L2-resident (< 126 MB L2)" if st["store_bytes"] < 126e6 else "streams from DRAM every pass"))}

    # every rank solves its block of the batched workload (all ranks reach
    # the aggregation together, before rank 0's own sections)
    batched = _batched(a, aspgpu, torch, rank, world, dev) if a.batch > 0 else None
    out = None
    if rank == 0:
        e2e = None
        if not a.no_e2e:
            e2e_checks, t_e2e, h2d = 0, 0.0, 0
            n_e2e = max(1, a.steps)
            for _ in range(n_e2e):
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                Q = aspgpu.Program(prog, conflict_budget=a.conflicts, time_budget_ms=120_000, view_mode=a.view, frontier=a.frontier)
                Q.solve(1, cap=1)
                s = Q.stats()
                Q.close()
                t_e2e += time.perf_counter() - t0
                e2e_checks += s["literal_checks"]
                h2d = s["store_bytes"]
            d2h = words * 8 + 32
            e2e = {"value": e2e_checks / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                   "d2h_bytes_per_step": int(d2h), "steps": n_e2e}
        big = _big_store(a, aspgpu, torch, dev, peak) if a.big_atoms > 0 else None
        tiny = _tiny(a, aspgpu, torch) if a.tiny > 0 else None
        learned = _learned(a, aspgpu, torch) if a.learned > 0 else None
        learning = None if a.no_learning_compare else _learning(a, aspgpu, prog)
        frontiers = _frontiers(a, aspgpu, prog)
        options = None if a.no_learning_compare or a.learned <= 0 else _search_options(a, aspgpu, torch)
        cpu = None if a.no_cpu else _cpu_baseline(prog, a.cpu_seconds)
        tsec = ms / 1e3
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": workload(a), "atoms": a.atoms, "rules": a.rules,
                       "conflict_budget_per_step": a.conflicts, "n_vars": st["n_vars"],
                       "n_nogoods": st["n_nogoods"], "n_literals": st["n_literals"],
                       "store_bytes": st["store_bytes"], "l2": "flushed between steps (1 GiB write)",
                       "view": {1: "plain 2-bit", 2: "packed 2-bit", 3: "bytes"}.get(st["view_mode"]),
                       "parallelism": f"replicas x{world}"},
            "e2e": e2e, "gpu_launches": a.steps,
            "roofline": roofline, "sweep_kernel": sweep, "cpu_baseline": cpu, "big_store": big,
            "tiny_programs": tiny, "batched": batched,
            "learned_heuristic": learned, "learning_compare": learning, "search_options": options,
            "frontier_compare": frontiers,
            "clocks": clk.summary(),
            "search": {"statuses": statuses, "decisions_per_s": totals["decisions"] / tsec,
                       "propagations_per_s": totals["propagations"] / tsec,
                       "conflicts_per_s": totals["conflicts"] / tsec, "rounds_per_s": totals["rounds"] / tsec,
                       "max_level": int(totals["max_level"]),
                       "learned_avg_len": totals["learned_literals"] / max(totals["learned"], 1),
                       "device_ns": {k: totals[k] for k in ("ns_total", "ns_sweep", "ns_analysis",
                                                           "ns_decision", "ns_stability", "ns_buckets",
                                                           "ns_learned", "ns_barrier", "ns_slowest_cta",
                                                           "ns_slowest_sweep", "ns_slowest_long",
                                                           "ns_slowest_buckets")}},
            "solver_src_sha": sha,
        }
        out["work_vs_oracle"] = _work_ratios(out)
        out["summary"] = _summary(out)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out, default=_plain), flush=True)


def _learning(a, aspgpu, prog):
    """fwd-learning against resolution to the first UIP (Algorithm 3) on the
    same programs, budgets and heuristic: device time, rates and learned
    nogood length of each (the quantities the paper compares)."""
    from synth.programs import random_program, program_seed
    cases = [(f"{a.atoms // 1000}k atoms, {a.rules // 1000}k rules (the main workload)", prog, a.conflicts),
             ("20k atoms, 50k rules, seed (2 << 32) | 1", random_program(20_000, 50_000, program_seed(2, 1)), 1000)]
    out = []
    for name, pr, budget in cases:
        row = {"workload": name, "conflict_budget": budget}
        for mode, key in ((aspgpu.LEARN_FWD, "fwd"), (aspgpu.LEARN_RES, "res")):
            P = aspgpu.Program(pr, learning=mode, conflict_budget=budget, time_budget_ms=60_000,
                               view_mode=a.view, frontier=a.frontier)
            P.solve(1, cap=1)                      # warm-up solve
            status, _, _ = P.solve(1, cap=1)
            s = P.stats()
            sec = max(s["ns_total"], 1) / 1e9
            row[key] = {"status": int(status), "device_s": sec, "conflicts": s["conflicts"],
                        "decisions_per_s": s["decisions"] / sec, "propagations_per_s": s["propagations"] / sec,
                        "conflicts_per_s": s["conflicts"] / sec, "learned_per_s": s["learned"] / sec,
                        "learned_avg_len": s["learned_literals"] / max(s["learned"], 1),
                        "us_per_analysis": s["ns_analysis"] / max(s["conflicts"], 1) / 1e3,
                        "analysis_share": s["ns_analysis"] / max(s["ns_total"], 1),
                        "max_level": s["max_level"]}
            P.close()
        out.append(row)
    return out


def _frontiers(a, aspgpu, prog):
    """The same search (same program, budget and heuristic) under each
    propagation-round mode: full sweeps, the nogood frontier (occurrence
    lists), and the unit frontier (dirty bucket units).  Device time, rates,
    rounds per decision, and literals and nogoods checked per round."""
    out = {}
    for name, fr, grid in (("full", aspgpu.FRONTIER_FULL, 0), ("nogoods", aspgpu.FRONTIER_NOGOODS, 0),
                           ("units", aspgpu.FRONTIER_UNITS, 0), ("units_chained", aspgpu.FRONTIER_UNITS_CHAINED, 0),
                           ("units_76_ctas", aspgpu.FRONTIER_UNITS, 76), ("units_38_ctas", aspgpu.FRONTIER_UNITS, 38),
                           ("units_chained_76_ctas", aspgpu.FRONTIER_UNITS_CHAINED, 76)):
        P = aspgpu.Program(prog, frontier=fr, conflict_budget=a.conflicts, time_budget_ms=60_000, view_mode=a.view,
                           grid_ctas=grid)
        P.solve(1, cap=1)                          # warm-up solve
        status, _, _ = P.solve(1, cap=1)
        s = P.stats()
        sec = max(s["ns_total"], 1) / 1e9
        rounds = max(s["rounds"], 1)
        out[name] = {"status": int(status), "device_s": sec, "conflicts": s["conflicts"],
                     "decisions_per_s": s["decisions"] / sec, "propagations_per_s": s["propagations"] / sec,
                     "conflicts_per_s": s["conflicts"] / sec, "rounds_per_s": s["rounds"] / sec,
                     "rounds_per_decision": s["rounds"] / max(s["decisions"], 1),
                     "us_per_round": s["ns_total"] / rounds / 1e3,
                     "literal_checks_per_round": s["literal_checks"] / rounds,
                     "nogood_visits_per_round": s["nogood_visits"] / rounds,
                     "literal_checks_per_s": s["literal_checks"] / sec,
                     "us_per_round_split": {k: s[k] / rounds / 1e3 for k in (
                         "ns_slowest_cta", "ns_slowest_sweep", "ns_slowest_long", "ns_slowest_buckets",
                         "ns_buckets", "ns_learned", "ns_barrier")}}
        P.close()
    full = out["full"]["decisions_per_s"]
    for v in out.values():
        v["decisions_per_s_vs_full"] = v["decisions_per_s"] / full if full else None
    return out


def shard_bounds(count, rank, world):
    """Rank `rank`'s contiguous block [lo, hi) of `count` independent programs
    (sizes are drawn i.i.d., so blocks are alike); blocks differ by at most one."""
    base, extra = divmod(count, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def _oracle_first(args):
    prog, budget_s, conflicts = args
    import oracle
    t = time.perf_counter()
    st, _, _ = oracle.cdnl(prog, max_models=1, time_budget_s=budget_s, conflict_budget=conflicts)
    return st, time.perf_counter() - t


def _oracle_pool(progs, budget_s, conflicts=0):
    """The oracle's CDNL, one program per host core (spawned workers)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_first, [(p, budget_s, conflicts) for p in progs], chunksize=4)
    return [r[0] for r in res], [r[1] for r in res], time.perf_counter() - t0, cores


def _oracle_enumerate(prog):
    import oracle
    return len(oracle.brute_force(prog))


def _oracle_pool_enumerate(progs):
    """The oracle's brute force (every answer set), one program per host core."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        n = pool.map(_oracle_enumerate, progs, chunksize=1)
    return sum(n), time.perf_counter() - t0, cores


def _batched(a, aspgpu, torch, rank=0, world=1, device=None):
    """Batched vs plain on the same programs: atom counts log-uniform in
    [200, 20000], rules = k x atoms (k = --batch-rules-per-atom; at 2 the
    family decides within the budget, at 4 almost nothing does), seeds
    (4 << 32) | i; per-program conflict budget.  solved = SAT or UNSAT within
    the budget.  The oracle's CDNL runs beside them on every host core, and
    its statuses are compared wherever both decide.  Under N ranks each rank
    solves its own block of the programs (no exchange of data); the job
    reports all ranks' solved programs over the slowest rank's time."""
    import numpy as np
    from synth.programs import batch_programs
    lo, hi = shard_bounds(a.batch, rank, world)
    rpa = a.batch_rules_per_atom
    progs = batch_programs(hi - lo, rules_per_atom=rpa, config_id=4, first_index=lo) if hi > lo else []
    kw = dict(conflict_budget=a.batch_conflicts, time_budget_ms=a.batch_ms, deps_levels=1024,
              learned_capacity=1 << 20, frontier=a.batch_frontier)
    P = [aspgpu.Program(p, **kw) for p in progs]
    solved_b = solved_p = agree = 0
    tb = tp = t_prepare = 0.0
    info = None
    st = np.zeros(0, np.int32)
    plain_ms = []
    if P:
        # autotuned configuration, launch captured in a CUDA graph; the timed
        # region replays it once
        t0 = time.perf_counter()
        plan = aspgpu.BatchPlan(P, max_models_each=1, cap_each=1, config=aspgpu.BATCH_AUTOTUNE)
        t_prepare = time.perf_counter() - t0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, nm, _ = plan.run()
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        info = plan.info()
        plan.close()
        solved_b = int(((st == 10) | (st == 20)).sum())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i, q in enumerate(P):
            t1 = time.perf_counter()
            s_, _, _ = q.solve(1, cap=1)
            plain_ms.append((time.perf_counter() - t1) * 1e3)
            solved_p += s_ in (10, 20)
            agree += int((s_ in (10, 20)) and (int(st[i]) in (10, 20)) and (s_ == int(st[i])))
        torch.cuda.synchronize()
        tp = time.perf_counter() - t0
        for q in P:
            q.close()
    oracle_part = None
    if rank == 0 and progs:
        ost, osec, owall, cores = _oracle_pool(progs, a.batch_ms / 1e3)
        ost = np.array(ost)
        od = (ost == 10) | (ost == 20)
        gd = (st == 10) | (st == 20)
        both = od & gd
        oracle_part = {"solved": int(od.sum()), "seconds": owall, "cores": cores,
                       "solved_per_s": int(od.sum()) / owall if owall else None,
                       "budget": f"{a.batch_ms / 1e3:g} s of CPU per program", "decided_by_both": int(both.sum()),
                       "status_mismatches": int((ost[both] != st[both]).sum())}
    if world > 1:
        # whole-job figures: MAX of the times, SUM of the counts
        tb, solved_b = aggregate_over_ranks(tb, solved_b, world, device)
        tp, solved_p = aggregate_over_ranks(tp, solved_p, world, device)
        _, agree = aggregate_over_ranks(0.0, agree, world, device)
        solved_b, solved_p, agree = int(solved_b), int(solved_p), int(agree)
    pct = (lambda q: float(np.percentile(plain_ms, q)) if plain_ms else None)
    return {"workload": f"{a.batch} programs, {rpa} rules per atom, atoms log-uniform in [200, 20000], "
                        f"conflict budget {a.batch_conflicts} and {a.batch_ms} ms per program, first answer set, "
                        f"frontier mode {a.batch_frontier} (batched and plain)"
                        + (f"; {world} ranks, one block of programs each" if world > 1 else ""),
            "batched": {"seconds": tb, "solved": solved_b, "solved_per_s": solved_b / tb if tb else None,
                        "prepare_seconds": t_prepare, "autotune": info},
            "plain": {"seconds": tp, "solved": solved_p, "solved_per_s": solved_p / tp if tp else None,
                      "ms_per_program_p50_p90_max": [pct(50), pct(90), max(plain_ms) if plain_ms else None]},
            "oracle_all_cores": oracle_part,
            "both_solved_and_agree": agree,
            "speedup_solved_per_s": (solved_b / tb) / (solved_p / tp) if solved_p and tb and tp else None}


def _big_store(a, aspgpu, torch, dev, peak):
    """The store larger than L2: a random program of --big-atoms atoms and 4
    rules per atom (seed (2 << 32) | 7).  The standalone sweep per pass
    (HBM-bound: the store streams every pass) and the solve kernel with a
    small conflict budget, both with algorithmic bytes Sigma(4 len + 4)."""
    from synth.programs import random_program, program_seed
    prog = random_program(a.big_atoms, 4 * a.big_atoms, program_seed(2, 7))
    P = aspgpu.Program(prog, conflict_budget=a.big_conflicts, time_budget_ms=60_000)
    st = P.stats()
    stream = torch.cuda.current_stream(dev)
    nonunit = st["n_nogoods"] - st["n_unit_nogoods"]
    sweep_bytes = 4 * (st["n_literals"] - st["n_unit_nogoods"]) + 4 * nonunit

    def timed(passes, reps=5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        P.sweep(passes)
        e0.record(stream)
        for _ in range(reps):
            P.sweep(passes)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    K = 16
    t1, tk = timed(1), timed(K + 1)
    per_pass = (tk - t1) / K
    sw_gbs = sweep_bytes / (per_pass / 1e3) / 1e9
    P.solve(1, cap=1)                                    # warm-up solve
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    status, _, _ = P.solve(1, cap=1)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    s = P.stats()
    dev_ms = s["ns_total"] / 1e6
    alg = 4.0 * s["literal_checks"] + 4.0 * s["nogood_visits"]
    out = {"workload": f"random program, {a.big_atoms // 1000}k atoms, {4 * a.big_atoms // 1000}k rules, "
                       f"body 1-4, negation 0.5; store {st['store_bytes'] / 1e6:.0f} MB (> 126 MB L2)",
           "store_bytes": st["store_bytes"], "nogoods": st["n_nogoods"], "literals": st["n_literals"],
           "sweep": {"ms_per_pass": per_pass, "ms_one_pass_launch": t1, "ms_17_pass_launch": tk,
                     "view_mode": {1: "plain 2-bit", 2: "packed 2-bit", 3: "bytes"}.get(st["view_mode"]),
                     "bytes_per_pass": sweep_bytes, "achieved_gbs": sw_gbs,
                     "frac_of_hbm": sw_gbs / peak if peak else None,
                     "note": "standalone sweep_kernel, (t(17 passes) - t(1 pass)) / 16, CUDA events"},
           "solver": {"status": int(status), "conflict_budget": a.big_conflicts, "device_ms": dev_ms,
                      "event_ms": ms, "literal_checks": s["literal_checks"], "nogood_visits": s["nogood_visits"],
                      "achieved_gbs": alg / (dev_ms / 1e3) / 1e9,
                      "frac_of_hbm": alg / (dev_ms / 1e3) / 1e9 / peak if peak else None,
                      "frac_4B_per_check": 4.0 * s["literal_checks"] / (dev_ms / 1e3) / 1e9 / peak if peak else None,
                      "rounds_per_s": s["rounds"] / (dev_ms / 1e3),
                      "decisions_per_s": s["decisions"] / (dev_ms / 1e3)}}
    P.close()
    return out


def _tiny(a, aspgpu, torch):
    """Tiny programs (20 atoms, 40 rules, 3 constraints; seeds 0..N-1): all
    answer sets of every program, batched (one launch) and one at a time;
    the oracle's brute force over 2^20 interpretations on a sample."""
    import oracle
    from synth.programs import tiny_program
    progs = [tiny_program(i) for i in range(a.tiny)]
    P = [aspgpu.Program(p) for p in progs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, nm, _ = aspgpu.solve_batch(P, max_models_each=0, cap_each=64)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    t0 = time.perf_counter()
    n_plain = 0
    for q in P:
        _, _, n = q.solve(0, cap=64)
        n_plain += n
    torch.cuda.synchronize()
    tp = time.perf_counter() - t0
    for q in P:
        q.close()
    sample = progs[:8]
    t0 = time.perf_counter()
    n_bf = sum(len(oracle.brute_force(p)) for p in sample)
    tbf = time.perf_counter() - t0
    pool_sample = progs[:64]
    n_pool, t_pool, cores = _oracle_pool_enumerate(pool_sample)
    return {"workload": f"{a.tiny} tiny programs (20 atoms, 40 rules, 3 constraints), every answer set",
            "answer_sets": int(nm.sum()), "answer_sets_plain": int(n_plain),
            "batched": {"seconds": tb, "instances_per_s": a.tiny / tb},
            "plain": {"seconds": tp, "instances_per_s": a.tiny / tp},
            "cpu_baseline": {"kind": "oracle brute force over 2^20 interpretations", "cores": 1,
                             "sample": f"first {len(sample)} programs ({n_bf} answer sets)",
                             "instances_per_s": len(sample) / tbf},
            "oracle_all_cores": {"kind": "oracle brute force, one program per host core", "cores": cores,
                                 "sample": f"first {len(pool_sample)} programs ({n_pool} answer sets)",
                                 "instances_per_s": len(pool_sample) / t_pool}}


def _work_ratios(out):
    """Rates of the same search work against the oracle on one core (the
    literal-check ratio compares different work: the sweeps re-read the whole
    store, the oracle reads occurrence lists)."""
    s, c = out.get("search"), out.get("cpu_baseline")
    if not s or not c:
        return None
    return {k: s[k] / c[k] if c.get(k) else None for k in ("decisions_per_s", "propagations_per_s", "conflicts_per_s")}


def _summary(out):
    """The headline figures of every leg, compact (the end of the line)."""
    def g(d, *ks):
        for k in ks:
            if not isinstance(d, dict):
                return None
            d = d.get(k)
        return round(d, 4) if isinstance(d, float) else d
    return {
        "checks_per_s": g(out, "value"), "frac_hbm": g(out, "roofline", "frac"),
        "decisions_per_s": g(out, "search", "decisions_per_s"),
        "propagations_per_s": g(out, "search", "propagations_per_s"),
        "work_vs_oracle": out.get("work_vs_oracle"),
        "big_store_sweep_frac": g(out, "big_store", "sweep", "frac_of_hbm"),
        "big_store_solver_frac": g(out, "big_store", "solver", "frac_of_hbm"),
        "tiny_instances_per_s": [g(out, "tiny_programs", "batched", "instances_per_s"),
                                 g(out, "tiny_programs", "plain", "instances_per_s"),
                                 g(out, "tiny_programs", "oracle_all_cores", "instances_per_s")],
        "batched_solved": [g(out, "batched", "batched", "solved"), g(out, "batched", "plain", "solved"),
                           g(out, "batched", "oracle_all_cores", "solved")],
        "batched_speedup": g(out, "batched", "speedup_solved_per_s"),
        "batched_oracle_mismatches": g(out, "batched", "oracle_all_cores", "status_mismatches"),
        "learned_solved": [g(out, "learned_heuristic", "plain", "solved"),
                           g(out, "learned_heuristic", "learned", "solved"),
                           g(out, "learned_heuristic", "learned_static", "solved"),
                           g(out, "learned_heuristic", "oracle_all_cores", "solved")],
        "learned_speedup": [g(out, "learned_heuristic", "speedup_solved_per_s"),
                            g(out, "learned_heuristic", "speedup_static_solved_per_s")],
        "frontier_decisions_per_s": {k: g(out, "frontier_compare", k, "decisions_per_s")
                                     for k in (out.get("frontier_compare") or {})},
        # literals read per round: every bucket literal (full sweeps, the
        # headline's count) against those of the nogoods holding a variable
        # assigned in the previous round (the occurrence-list frontier)
        "literal_checks_per_round": {"scanned_full_sweeps": g(out, "frontier_compare", "full",
                                                              "literal_checks_per_round"),
                                     "necessary_occurrence_lists": g(out, "frontier_compare", "nogoods",
                                                                     "literal_checks_per_round")},
    }


def _a11_programs(count, first_index):
    """Half random programs (4 rules per atom, atoms log-uniform in
    [200, 2000]), half 3-colourings of G(n, 4.5/(n-1)) with n in [40, 400]."""
    from synth.programs import batch_programs, coloring_program, batch_sizes
    half = count // 2
    progs = batch_programs(half, rules_per_atom=4, config_id=5, first_index=first_index, lo=200, hi=2000)
    _, ns = batch_sizes(count - half, lo=40, hi=400, config_id=6, first_index=first_index)
    progs += [coloring_program(int(n), 4.5, seed_index=first_index + i) for i, n in enumerate(ns)]
    return progs


def _learned(a, aspgpu, torch):
    """Learned vs plain decision heuristic on held-out programs, both batched,
    same per-program conflict budget; training on traces of the plain
    heuristic on disjoint seeds."""
    from paper_1909_01786_gb300 import heuristic as H
    budget = a.learned_conflicts
    t0 = time.perf_counter()
    X, y = H.collect_traces(_a11_programs(a.learned_train, 10**6), conflict_budget=budget)
    w, tstats = H.fit(X, y)
    ws, sstats = H.fit(X, y, static=True)
    t_train = time.perf_counter() - t0
    if a.save_weights:
        H.save(w, a.save_weights, **tstats)
    import numpy as np
    import oracle
    names = ("plain", "learned", "learned_static")
    per_seed = []
    mism = checked = bad = 0
    for seed in range(a.learned_seeds):
        evalp = _a11_programs(a.learned, 2 * 10**6 + seed * 10**5)
        out = {}
        for name, kw in zip(names, (dict(heuristic=0), dict(heuristic=2, mlp_weights=w),
                                    dict(heuristic=3, mlp_weights=ws))):
            P = [aspgpu.Program(p, conflict_budget=budget, time_budget_ms=20_000, deps_levels=1024,
                                learned_capacity=1 << 20, **kw) for p in evalp]
            torch.cuda.synchronize()
            t = time.perf_counter()
            st, nm, models = aspgpu.solve_batch(P, max_models_each=1, cap_each=1)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
            dec = sum(q.stats()["decisions"] for q in P)
            con = sum(q.stats()["conflicts"] for q in P)
            solved = int(((st == 10) | (st == 20)).sum())
            out[name] = {"seconds": dt, "solved": solved, "solved_per_s": solved / dt,
                         "decisions": int(dec), "conflicts": int(con), "statuses": st.copy(), "models": models}
            for q in P:
                q.close()
        # zero mismatches: where both decided they agree; models are answer sets
        sp = out["plain"]["statuses"]
        for name in ("learned", "learned_static"):
            sl = out[name]["statuses"]
            both = ((sp == 10) | (sp == 20)) & ((sl == 10) | (sl == 20))
            mism += int((sp[both] != sl[both]).sum())
        for name in names:
            for i, m in enumerate(out[name]["models"]):
                if len(m):
                    checked += 1
                    bad += not oracle.is_answer_set(evalp[i], m[0])
            del out[name]["statuses"], out[name]["models"]
        per_seed.append(out)
    ratio = lambda name: [o[name]["solved_per_s"] / o["plain"]["solved_per_s"] if o["plain"]["solved"] else None
                          for o in per_seed]
    first = per_seed[0]
    # the oracle's CDNL on every host core, same held-out programs and
    # conflict budget (first seed set)
    ost, _, owall, cores = _oracle_pool(_a11_programs(a.learned, 2 * 10**6), 20.0, conflicts=budget)
    ost = np.array(ost)
    osolved = int(((ost == 10) | (ost == 20)).sum())
    oracle_part = {"solved": osolved, "seconds": owall, "cores": cores, "solved_per_s": osolved / owall,
                   "budget": f"{budget} conflicts (and 20 s) per program"}
    r_l, r_s = ratio("learned"), ratio("learned_static")
    spread = lambda r: [min(x for x in r if x is not None), max(x for x in r if x is not None)] \
        if any(x is not None for x in r) else None
    return {"workload": f"{a.learned_seeds} x {a.learned} held-out programs (half random, 4 rules per atom, "
                        f"200-2000 atoms; half 3-colourings, 40-400 vertices), conflict budget {budget}, batched",
            "training": {"programs": a.learned_train, "seconds": t_train, **tstats},
            **first, "per_seed": per_seed if a.learned_seeds > 1 else None, "oracle_all_cores": oracle_part,
            "status_mismatches": mism, "models_checked": checked, "invalid_models": bad,
            "speedup_solved_per_s": r_l[0], "speedup_static_solved_per_s": r_s[0],
            "speedup_spread": {"learned": spread(r_l), "learned_static": spread(r_s)},
            "static_training": sstats}


def _search_options(a, aspgpu, torch):
    """Solved programs within the same per-program conflict budget, batched,
    under each learning / backjump / restart option, on the held-out set of
    the learned-heuristic comparison."""
    import oracle
    evalp = _a11_programs(a.learned, 2 * 10**6)
    budget = a.learned_conflicts
    modes = (("fwd, backjump h-1 (default)", dict()),
             ("fwd, asserting backjump", dict(backjump=aspgpu.BACKJUMP_ASSERTING)),
             ("fwd, Luby restarts x16", dict(restart_conflicts=16)),
             ("fwd, 4 conflicts per round", dict(conflicts_per_round=4)),
             ("res (first UIP)", dict(learning=aspgpu.LEARN_RES)),
             ("res, Luby restarts x16", dict(learning=aspgpu.LEARN_RES, restart_conflicts=16)))
    out, ref = {}, None
    checked = bad = mism = 0
    for name, kw in modes:
        P = [aspgpu.Program(p, conflict_budget=budget, time_budget_ms=20_000, deps_levels=1024,
                            learned_capacity=1 << 20, **kw) for p in evalp]
        torch.cuda.synchronize()
        t = time.perf_counter()
        st, nm, models = aspgpu.solve_batch(P, max_models_each=1, cap_each=1)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        decided = (st == 10) | (st == 20)
        if ref is None:
            ref = st.copy()
        else:
            both = decided & ((ref == 10) | (ref == 20))
            mism += int((st[both] != ref[both]).sum())
        for i, m in enumerate(models):
            if len(m):
                checked += 1
                bad += not oracle.is_answer_set(evalp[i], m[0])
        out[name] = {"seconds": dt, "solved": int(decided.sum()), "solved_per_s": int(decided.sum()) / dt,
                     "conflicts": int(sum(q.stats()["conflicts"] for q in P)),
                     "restarts": int(sum(q.stats()["restarts"] for q in P))}
        for q in P:
            q.close()
    return {"workload": f"{a.learned} held-out programs of the learned-heuristic comparison, conflict "
                        f"budget {budget}, batched", "modes": out, "status_mismatches": mism,
            "models_checked": checked, "invalid_models": bad}


def run_sweeps(a):
    """Standalone propagate-and-check sweeps over the store (root assignment
    after initial propagation), for kernel profiling."""
    import numpy as np
    import torch
    from paper_1909_01786_gb300 import aspgpu
    prog = _program(a)
    P = aspgpu.Program(prog, view_mode=a.view)
    P.propagate(np.zeros(P.n_vars, np.int8))
    for _ in range(3):
        P.sweep(a.sweep_only)
    torch.cuda.synchronize()
    st = P.stats()
    print(json.dumps({"sweeps": a.sweep_only, "store_bytes": st["store_bytes"], "view_mode": st["view_mode"]}))


def main():
    a = _args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(a.gpus)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if "WORLD_SIZE" not in os.environ:
        world = 1 if a.gpus <= 1 else a.gpus
        if world > 1:
            print(json.dumps({"error": "run N>1 under torch.distributed.run"}))
            return
    if a.sweep_only:
        run_sweeps(a)
    elif a.impl == "reference":
        run_reference(a, rank, world)
    else:
        run_ours(a, rank, world, local_rank)


if __name__ == "__main__":
    main()
