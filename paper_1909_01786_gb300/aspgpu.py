"""ctypes binding of libaspgpu (include/aspgpu.h): argument marshalling only.

Every step of the search runs in the library's CUDA kernels.  There is no
fallback: if the compiled library or a CUDA device is missing, calls raise.
PyTorch, when present, provides device memory (its caching allocator) and
streams.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

ASP_OK, ASP_E_CAPACITY = 0, -5
MLP_FEATURES, MLP_PARAMS = 16, 1153
HEUR_OCCURRENCE, HEUR_ACTIVITY, HEUR_LEARNED, HEUR_LEARNED_STATIC, HEUR_JW, HEUR_VSIDS = 0, 1, 2, 3, 4, 5
SAT, UNSAT, UNKNOWN = 10, 20, 0
VIEW_AUTO, VIEW_PLAIN, VIEW_PACKED, VIEW_BYTES = 0, 1, 2, 3
LEARN_FWD, LEARN_RES = 0, 1
FRONTIER_FULL, FRONTIER_NOGOODS, FRONTIER_UNITS, FRONTIER_UNITS_CHAINED = 0, 1, 2, 3
BACKJUMP_H_MINUS_1, BACKJUMP_ASSERTING = 0, 1
R_DECISION, R_COMPLETE, R_INPUT = 0xFFFFFFFF, 0xFFFFFFFE, 0xFFFFFFFD

_lib = None
_lock = threading.Lock()


class AspError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"aspgpu error {code}: {msg}")
        self.code = code


class Options(C.Structure):
    _fields_ = [("heuristic", C.c_int32), ("deps_levels", C.c_int32),
                ("conflict_budget", C.c_int64), ("time_budget_ms", C.c_int64),
                ("learned_capacity", C.c_int64), ("grid_ctas", C.c_int32),
                ("block_threads", C.c_int32), ("cuda_stream", C.c_void_p),
                ("dev_alloc", C.c_void_p), ("dev_free", C.c_void_p), ("alloc_ctx", C.c_void_p),
                ("mlp_weights", C.c_void_p), ("trace_capacity", C.c_int64),
                ("view_mode", C.c_int32), ("frontier", C.c_int32), ("learning", C.c_int32),
                ("backjump", C.c_int32), ("restart_conflicts", C.c_int32),
                ("conflicts_per_round", C.c_int32), ("compact", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in (
        "n_vars", "n_atoms", "n_rules_with_head", "n_nogoods", "n_literals",
        "n_unit_nogoods", "n_long_nogoods", "store_bytes", "rounds", "literal_checks",
        "propagations", "conflicts", "decisions", "completions", "learned",
        "learned_literals", "loop_nogoods", "models", "max_level", "ns_total",
        "ns_sweep", "ns_analysis", "ns_decision", "ns_stability", "ns_buckets", "ns_learned",
        "ns_barrier", "view_mode", "batch_view_mode", "ns_slowest_cta", "ns_slowest_sweep",
        "restarts", "conflict_rounds", "nogood_visits", "ns_slowest_long", "ns_slowest_buckets")]


EXPORTS = ["asp_default_options", "asp_load_ground", "asp_solve", "asp_solve_async", "asp_solve_batch",
           "asp_stats", "asp_free", "asp_last_error", "asp_debug_propagate", "asp_sweep",
           "asp_debug_state", "asp_debug_last_conflict", "asp_debug_nogood", "asp_debug_learned",
           "asp_build_info", "asp_debug_barrier", "asp_debug_fail_alloc", "asp_propagate_noalloc", "asp_trace", "asp_train_mlp",
           "asp_mlp_score", "asp_batch_create", "asp_batch_run", "asp_batch_info", "asp_batch_free",
           "asp_debug_completion", "asp_debug_rule_scores"]


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libaspgpu.so (building it in-tree if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            _build.build()
        if not os.path.exists(path):
            raise AspError(-7, f"{path} not built")
        L = C.CDLL(path)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        L.asp_default_options.argtypes = [vp]
        L.asp_default_options.restype = None
        L.asp_load_ground.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, vp]
        L.asp_load_ground.restype = C.c_int
        L.asp_solve.argtypes = [vp, i64, vp, i64, vp, vp]
        L.asp_solve.restype = C.c_int
        L.asp_solve_async.argtypes = [vp, i64, vp, i64, vp]
        L.asp_solve_async.restype = C.c_int
        L.asp_solve_batch.argtypes = [i32, vp, i64, vp, vp, vp, vp]
        L.asp_solve_batch.restype = C.c_int
        L.asp_batch_create.argtypes = [i32, vp, i64, vp, i32, vp]
        L.asp_batch_create.restype = C.c_int
        L.asp_batch_run.argtypes = [vp, vp, vp, vp]
        L.asp_batch_run.restype = C.c_int
        L.asp_batch_info.argtypes = [vp, vp, vp, vp, vp, vp]
        L.asp_batch_info.restype = C.c_int
        L.asp_batch_free.argtypes = [vp]
        L.asp_batch_free.restype = None
        L.asp_stats.argtypes = [vp, vp]
        L.asp_stats.restype = C.c_int
        L.asp_free.argtypes = [vp]
        L.asp_free.restype = None
        L.asp_last_error.argtypes = []
        L.asp_last_error.restype = C.c_char_p
        L.asp_debug_propagate.argtypes = [vp, vp, vp, vp]
        L.asp_debug_propagate.restype = C.c_int
        L.asp_sweep.argtypes = [vp, C.c_int32]
        L.asp_sweep.restype = C.c_int
        L.asp_debug_state.argtypes = [vp, vp, vp, vp, vp, vp, i32]
        L.asp_debug_state.restype = C.c_int
        L.asp_debug_last_conflict.argtypes = [vp, vp, vp, i64]
        L.asp_debug_last_conflict.restype = C.c_int
        L.asp_debug_nogood.argtypes = [vp, C.c_uint32, vp, i64]
        L.asp_debug_nogood.restype = i64
        L.asp_debug_learned.argtypes = [vp, vp, i64]
        L.asp_debug_learned.restype = i64
        L.asp_build_info.argtypes = [vp, vp]
        L.asp_build_info.restype = C.c_int
        L.asp_debug_barrier.argtypes = [vp, i32, i32]
        L.asp_debug_barrier.restype = C.c_int
        L.asp_debug_fail_alloc.argtypes = [i64]
        L.asp_debug_fail_alloc.restype = C.c_int
        L.asp_propagate_noalloc.argtypes = [vp, vp, vp, vp]
        L.asp_propagate_noalloc.restype = C.c_int
        L.asp_trace.argtypes = [vp, vp, vp, vp, i64]
        L.asp_trace.restype = i64
        L.asp_train_mlp.argtypes = [vp, vp, i64, i32, C.c_float, vp]
        L.asp_train_mlp.restype = C.c_int
        L.asp_mlp_score.argtypes = [vp, vp, i64, vp]
        L.asp_mlp_score.restype = C.c_int
        L.asp_debug_completion.argtypes = [i32, i32, vp, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp, i64]
        L.asp_debug_completion.restype = C.c_int
        L.asp_debug_rule_scores.argtypes = [i32, i32, vp, vp, vp, vp, vp, i32, vp, vp, vp, vp, i64]
        L.asp_debug_rule_scores.restype = C.c_int
        _lib = L
        return L


def _check(rc, ok=(ASP_OK,)):
    if rc not in ok:
        raise AspError(rc, lib().asp_last_error().decode())
    return rc


_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class _TorchAllocator:
    """Device memory from PyTorch's caching allocator on the given stream."""

    def __init__(self, torch, device, stream):
        self.torch, self.device, self.stream = torch, device, stream

        def alloc(n, ctx):
            return self.torch.cuda.caching_allocator_alloc(int(n), device=self.device, stream=self.stream)

        def free(p, n, ctx):
            self.torch.cuda.caching_allocator_delete(p)

        self.c_alloc, self.c_free = _ALLOC(alloc), _FREE(free)


def words_to_models(words: np.ndarray, n_atoms: int) -> np.ndarray:
    """uint64 model rows -> uint8 [rows, n_atoms]."""
    if words.shape[0] == 0:
        return np.zeros((0, n_atoms), dtype=np.uint8)
    b = np.unpackbits(words.astype("<u8").view(np.uint8).reshape(words.shape[0], -1), axis=1, bitorder="little")
    return b[:, :n_atoms].copy()


class Program:
    """A ground program loaded on the GPU (asp_load_ground)."""

    def __init__(self, prog, *, heuristic=0, deps_levels=0, conflict_budget=0, time_budget_ms=120_000,
                 learned_capacity=0, grid_ctas=0, block_threads=0, stream=None, torch_memory=True,
                 mlp_weights=None, trace_capacity=0, view_mode=0, frontier=False, learning=LEARN_FWD,
                 backjump=BACKJUMP_H_MINUS_1, restart_conflicts=0, conflicts_per_round=1, compact=False):
        L = lib()
        self.n_atoms = int(prog.n_atoms)
        self._keep = []
        opt = Options()
        L.asp_default_options(C.byref(opt))
        if mlp_weights is not None:
            w = np.ascontiguousarray(mlp_weights, dtype=np.float32)
            assert w.shape == (MLP_PARAMS,)
            self._keep.append(w)
            opt.mlp_weights = w.ctypes.data
        opt.trace_capacity = int(trace_capacity)
        opt.view_mode = int(view_mode)
        opt.frontier = int(frontier)         # False/True = full / nogood frontier; FRONTIER_UNITS
        opt.learning = int(learning)
        opt.backjump = int(backjump)
        opt.restart_conflicts = int(restart_conflicts)
        opt.conflicts_per_round = int(conflicts_per_round)
        opt.compact = 1 if compact else 0
        opt.heuristic, opt.deps_levels = heuristic, deps_levels
        opt.conflict_budget, opt.time_budget_ms = conflict_budget, time_budget_ms
        opt.learned_capacity, opt.grid_ctas, opt.block_threads = learned_capacity, grid_ctas, block_threads
        self._alloc = None
        if torch_memory:
            try:
                import torch
            except ImportError:
                torch = None
            if torch is not None and torch.cuda.is_available():
                dev = torch.cuda.current_device()
                s = stream if stream is not None else torch.cuda.current_stream(dev)
                self._alloc = _TorchAllocator(torch, dev, s)
                opt.cuda_stream = s.cuda_stream
                opt.dev_alloc = C.cast(self._alloc.c_alloc, C.c_void_p).value
                opt.dev_free = C.cast(self._alloc.c_free, C.c_void_p).value
                self.stream = s
        arrs = [np.ascontiguousarray(prog.head, np.int32), np.ascontiguousarray(prog.pos_off, np.int64),
                np.ascontiguousarray(prog.pos, np.int32), np.ascontiguousarray(prog.neg_off, np.int64),
                np.ascontiguousarray(prog.neg, np.int32)]
        h = C.c_void_p()
        _check(L.asp_load_ground(self.n_atoms, int(prog.head.shape[0]),
                                 *[a.ctypes.data if a.size else None for a in arrs],
                                 C.byref(opt), C.byref(h)))
        self.handle = h
        self.words = (self.n_atoms + 63) // 64
        st = self.stats()
        self.n_vars = st["n_vars"]

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().asp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, max_models: int = 0, cap: int | None = None, raw: bool = False):
        """Returns (status, models uint8 [n, n_atoms], n_found)."""
        if cap is None:
            cap = max_models if max_models > 0 else 4096
        buf = np.zeros((max(cap, 1), max(self.words, 1)), dtype=np.uint64)
        n = C.c_int64()
        st = C.c_int32()
        rc = lib().asp_solve(self.handle, int(max_models), buf.ctypes.data, int(cap), C.byref(n), C.byref(st))
        _check(rc, ok=(ASP_OK, ASP_E_CAPACITY))
        rows = buf[:min(n.value, cap)]
        return st.value, (rows if raw else words_to_models(rows, self.n_atoms)), n.value

    def solve_async(self, max_models: int, d_models_ptr: int, cap: int, d_result_ptr: int):
        _check(lib().asp_solve_async(self.handle, int(max_models), d_models_ptr or None, int(cap), d_result_ptr))

    def propagate(self, partial: np.ndarray):
        """Unit propagation of a partial assignment over all variables."""
        p = np.ascontiguousarray(partial, dtype=np.int8)
        assert p.shape[0] == self.n_vars
        out = np.zeros(self.n_vars, dtype=np.int8)
        conf = C.c_int32()
        _check(lib().asp_debug_propagate(self.handle, p.ctypes.data, out.ctypes.data, C.byref(conf)))
        return bool(conf.value), out

    def propagate_noalloc(self, d_partial: int, d_closure: int, d_conflict: int) -> int:
        """asp_propagate_noalloc on device buffers (int8 / int8 / int32
        pointers); enqueued on the program's stream.  Returns the ABI code."""
        return lib().asp_propagate_noalloc(self.handle, d_partial, d_closure, d_conflict)

    def learned_ids(self) -> np.ndarray:
        """Ids of the nogoods the last solve learned, in order (asp_debug_learned)."""
        n = lib().asp_debug_learned(self.handle, None, 0)
        if n < 0:
            raise AspError(n, lib().asp_last_error().decode())
        ids = np.zeros(max(n, 1), np.uint32)
        n2 = lib().asp_debug_learned(self.handle, ids.ctypes.data, int(n))
        if n2 < 0:
            raise AspError(n2, lib().asp_last_error().decode())
        return ids[:min(n, n2)].copy()

    def trace(self, cap: int = 1 << 16, with_rules: bool = False):
        """Decision trace of the last solve: (features [n, 16], labels [n])
        and, with_rules, the rule index of each row."""
        f = np.zeros((max(cap, 1), MLP_FEATURES), np.float32)
        y = np.zeros(max(cap, 1), np.int32)
        r = np.zeros(max(cap, 1), np.int32)
        n = lib().asp_trace(self.handle, f.ctypes.data, y.ctypes.data, r.ctypes.data, int(cap))
        if n < 0:
            raise AspError(n, lib().asp_last_error().decode())
        if with_rules:
            return f[:n].copy(), y[:n].copy(), r[:n].copy()
        return f[:n].copy(), y[:n].copy()

    def sweep(self, passes: int = 1):
        _check(lib().asp_sweep(self.handle, int(passes)))

    def stats(self) -> dict:
        s = Stats()
        _check(lib().asp_stats(self.handle, C.byref(s)))
        return {n: getattr(s, n) for n, _ in Stats._fields_}

    def state(self, deps_words: int = 0) -> dict:
        nv = self.n_vars
        trail = np.zeros(max(nv, 1), np.int32)
        level = np.zeros(max(nv, 1), np.int32)
        reason = np.zeros(max(nv, 1), np.uint32)
        deps = np.zeros((max(nv, 1), max(deps_words, 1)), np.uint64)
        nt = C.c_int64()
        _check(lib().asp_debug_state(self.handle, trail.ctypes.data, C.byref(nt), level.ctypes.data,
                                     reason.ctypes.data, deps.ctypes.data if deps_words else None,
                                     int(deps_words)))
        return dict(trail=trail[:nt.value], level=level[:nv], reason=reason[:nv],
                    deps=deps[:nv] if deps_words else None)

    def last_conflict(self) -> dict | None:
        """The last conflict analysis of the last solve (asp_debug_last_conflict):
        conflicting nogood id, trail as literals up to the conflict, learned
        nogood id and length, backjump target, level resolved at; None if no
        conflict was analysed."""
        info = np.zeros(6, np.int64)
        trail = np.zeros(max(self.n_vars, 1), np.int32)
        _check(lib().asp_debug_last_conflict(self.handle, info.ctypes.data, trail.ctypes.data, int(self.n_vars)))
        nt = int(min(info[1], self.n_vars))
        if info[3] == 0:
            if info[4] == 0:
                return None
            # the analysis stopped on an inconsistent state
            return dict(conflict=int(info[0]), trail=trail[:nt].copy(), failed_check=int(info[4]),
                        involving=int(info[2]), level=int(info[5]))
        return dict(conflict=int(info[0]), trail=trail[:nt].copy(), learned=int(info[2]),
                    length=int(info[3]), target=int(info[4]), level=int(info[5]))

    def nogood(self, nid: int):
        buf = np.zeros(4096, np.int32)
        n = lib().asp_debug_nogood(self.handle, int(nid), buf.ctypes.data, 4096)
        if n < 0:
            raise AspError(n, lib().asp_last_error().decode())
        if n > 4096:
            buf = np.zeros(n, np.int32)
            lib().asp_debug_nogood(self.handle, int(nid), buf.ctypes.data, n)
        return buf[:n].copy()


def _program_arrays(prog):
    arrs = [np.ascontiguousarray(prog.head, np.int32), np.ascontiguousarray(prog.pos_off, np.int64),
            np.ascontiguousarray(prog.pos, np.int32), np.ascontiguousarray(prog.neg_off, np.int64),
            np.ascontiguousarray(prog.neg, np.int32)]
    return arrs, [a.ctypes.data if a.size else None for a in arrs]


def completion(prog, compact: bool = False):
    """The library's completion nogoods, built on the host only
    (asp_debug_completion): (n_vars, off int64[n + 1], lits int32) with
    literals (var << 1 | sign), sign 1 = F, in the library's variables."""
    L = lib()
    keep, ptrs = _program_arrays(prog)
    nv, nn, nl = C.c_int64(), C.c_int64(), C.c_int64()
    args = [int(prog.n_atoms), int(prog.head.shape[0]), *ptrs, 1 if compact else 0,
            C.byref(nv), C.byref(nn), C.byref(nl)]
    _check(L.asp_debug_completion(*args, None, None, 0))
    off = np.zeros(nn.value + 1, np.int64)
    lits = np.zeros(max(nl.value, 1), np.int32)
    _check(L.asp_debug_completion(*args, off.ctypes.data, lits.ctypes.data, int(lits.shape[0])))
    return nv.value, off, lits[:nl.value]


def rule_scores(prog, compact: bool = False):
    """Library rule order and static decision scores, on the host only
    (asp_debug_rule_scores): (rule_index, score_occ, score_jw), one entry per
    headed rule in the library's order."""
    L = lib()
    keep, ptrs = _program_arrays(prog)
    nh = C.c_int32()
    args = [int(prog.n_atoms), int(prog.head.shape[0]), *ptrs, 1 if compact else 0, C.byref(nh)]
    _check(L.asp_debug_rule_scores(*args, None, None, None, 0))
    n = nh.value
    idx = np.zeros(max(n, 1), np.int32)
    occ = np.zeros(max(n, 1), np.uint32)
    jw = np.zeros(max(n, 1), np.uint32)
    _check(L.asp_debug_rule_scores(*args, idx.ctypes.data, occ.ctypes.data, jw.ctypes.data, int(idx.shape[0])))
    return idx[:n], occ[:n], jw[:n]


def build_info() -> dict:
    """asp_build_info: compute capability and PTX version of the solve kernel."""
    b, p = C.c_int32(), C.c_int32()
    _check(lib().asp_build_info(C.byref(b), C.byref(p)))
    return {"binary_version": b.value, "ptx_version": p.value}


def solve_batch(programs, max_models_each: int = 1, cap_each: int = 1):
    """asp_solve_batch over loaded Programs: (statuses, n_models, models list)."""
    n = len(programs)
    handles = (C.c_void_p * n)(*[p.handle.value for p in programs])
    st = np.zeros(n, np.int32)
    nm = np.zeros(n, np.int64)
    bufs = [np.zeros((max(cap_each, 1), max(p.words, 1)), np.uint64) for p in programs]
    ptrs = (C.c_void_p * n)(*[b.ctypes.data for b in bufs])
    caps = np.full(n, cap_each, np.int64)
    _check(lib().asp_solve_batch(n, handles, int(max_models_each), st.ctypes.data, nm.ctypes.data, ptrs,
                                 caps.ctypes.data))
    models = [words_to_models(b[:min(int(k), cap_each)], p.n_atoms) for b, k, p in zip(bufs, nm, programs)]
    return st, nm, models


BATCH_AUTOTUNE = -1


class BatchPlan:
    """asp_batch_create: programs prepared for repeated batched solving
    (descriptors uploaded, configuration chosen, launch captured in a CUDA
    graph); run() replays it."""

    def __init__(self, programs, max_models_each: int = 1, cap_each: int = 1, config: int = BATCH_AUTOTUNE):
        self.programs = list(programs)
        n = len(self.programs)
        self.cap_each = cap_each
        handles = (C.c_void_p * n)(*[p.handle.value for p in self.programs])
        caps = np.full(n, cap_each, np.int64)
        h = C.c_void_p()
        _check(lib().asp_batch_create(n, handles, int(max_models_each), caps.ctypes.data, int(config), C.byref(h)))
        self.handle = h
        self._bufs = [np.zeros((max(cap_each, 1), max(p.words, 1)), np.uint64) for p in self.programs]
        self._ptrs = (C.c_void_p * n)(*[b.ctypes.data for b in self._bufs])

    def run(self):
        n = len(self.programs)
        st = np.zeros(n, np.int32)
        nm = np.zeros(n, np.int64)
        _check(lib().asp_batch_run(self.handle, st.ctypes.data, nm.ctypes.data, self._ptrs))
        models = [words_to_models(b[:min(int(k), self.cap_each)], p.n_atoms)
                  for b, k, p in zip(self._bufs, nm, self.programs)]
        return st, nm, models

    def info(self):
        cfg, bt, grid, fr = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        trial = (C.c_double * 4)()
        _check(lib().asp_batch_info(self.handle, C.byref(cfg), C.byref(bt), C.byref(grid), C.byref(fr), trial))
        return {"config": cfg.value, "block_threads": bt.value, "grid": grid.value,
                "frontier": {FRONTIER_FULL: "full", FRONTIER_UNITS: "units"}.get(fr.value, fr.value),
                "trial_ns_per_program": {"full": [trial[0], trial[1]], "units": [trial[2], trial[3]]}}

    def close(self):
        if self.handle:
            lib().asp_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def train_mlp(features: np.ndarray, labels: np.ndarray, weights: np.ndarray, epochs: int = 50,
              learning_rate: float = 0.05) -> np.ndarray:
    """asp_train_mlp: returns the trained weights (float32 [MLP_PARAMS])."""
    X = np.ascontiguousarray(features, dtype=np.float32)
    y = np.ascontiguousarray(labels, dtype=np.float32)
    w = np.ascontiguousarray(weights, dtype=np.float32).copy()
    _check(lib().asp_train_mlp(X.ctypes.data, y.ctypes.data, int(X.shape[0]), int(epochs),
                               float(learning_rate), w.ctypes.data))
    return w


def mlp_score(weights: np.ndarray, features: np.ndarray) -> np.ndarray:
    """asp_mlp_score: device scores of feature rows (bf16 weights, fp32 sums)."""
    w = np.ascontiguousarray(weights, dtype=np.float32)
    X = np.ascontiguousarray(features, dtype=np.float32)
    out = np.zeros(X.shape[0], np.float32)
    _check(lib().asp_mlp_score(w.ctypes.data, X.ctypes.data, int(X.shape[0]), out.ctypes.data))
    return out
