"""CPU oracle for answer-set computation (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package.  The solver library never does:
the oracle is an independent, plain restatement of the paper's definitions
(arXiv 1909.01786, Sections 1-2 and Algorithm 3), used to check the GPU path.

``build()`` compiles ``asp_oracle.c`` with gcc into ``oracle/_build``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "asp_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libasporacle.so")
_lib = None
_lock = threading.Lock()

SAT, UNSAT, UNKNOWN = 10, 20, 0


def build(force: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Prog(C.Structure):
    _fields_ = [("na", C.c_int32), ("nr", C.c_int32),
                ("head", C.c_void_p), ("pos_off", C.c_void_p), ("pos", C.c_void_p),
                ("neg_off", C.c_void_p), ("neg", C.c_void_p)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER(_Prog)
            lib.oracle_is_answer_set.argtypes = [P, C.c_void_p]
            lib.oracle_is_answer_set.restype = C.c_int
            lib.oracle_least_model_of_reduct.argtypes = [P, C.c_void_p, C.c_void_p]
            lib.oracle_least_model_of_reduct.restype = None
            lib.oracle_brute_force.argtypes = [P, C.c_void_p, C.c_int64]
            lib.oracle_brute_force.restype = C.c_int64
            lib.oracle_completion.argtypes = [P, C.c_int] + [C.c_void_p] * 5
            lib.oracle_completion.restype = C.c_int
            lib.oracle_up_closure.argtypes = [P, C.c_int] + [C.c_void_p] * 5
            lib.oracle_up_closure.restype = C.c_int
            lib.oracle_cdnl.argtypes = [P, C.c_int64, C.c_int64, C.c_double, C.c_void_p, C.c_int64,
                                        C.c_void_p, C.c_void_p]
            lib.oracle_cdnl.restype = C.c_int
            _lib = lib
    return _lib


class _Bound:
    """Keeps the numpy arrays of a program alive while C sees them."""

    def __init__(self, prog):
        self.arrs = [np.ascontiguousarray(prog.head, dtype=np.int32),
                     np.ascontiguousarray(prog.pos_off, dtype=np.int64),
                     np.ascontiguousarray(prog.pos, dtype=np.int32),
                     np.ascontiguousarray(prog.neg_off, dtype=np.int64),
                     np.ascontiguousarray(prog.neg, dtype=np.int32)]
        a = self.arrs
        self.s = _Prog(int(prog.n_atoms), int(prog.head.shape[0]),
                       a[0].ctypes.data, a[1].ctypes.data, a[2].ctypes.data,
                       a[3].ctypes.data, a[4].ctypes.data)
        self.ref = C.byref(self.s)


def _ptr(a):
    return a.ctypes.data if a is not None else None


def is_answer_set(prog, M) -> bool:
    """M (bool/uint8 per atom): M = LM(reduct) and no constraint violated."""
    b = _Bound(prog)
    m = np.ascontiguousarray(M, dtype=np.uint8)
    return bool(_load().oracle_is_answer_set(b.ref, _ptr(m)))


def least_model_of_reduct(prog, M) -> np.ndarray:
    b = _Bound(prog)
    m = np.ascontiguousarray(M, dtype=np.uint8)
    out = np.zeros(prog.n_atoms, dtype=np.uint8)
    _load().oracle_least_model_of_reduct(b.ref, _ptr(m), _ptr(out))
    return out


def brute_force(prog, cap: int = 1 << 16):
    """All answer sets by subset enumeration (n_atoms <= 26); rows of uint8."""
    b = _Bound(prog)
    buf = np.zeros((cap, max(prog.n_atoms, 1)), dtype=np.uint8)
    n = _load().oracle_brute_force(b.ref, _ptr(buf), cap)
    if n < 0:
        raise ValueError("brute force needs at most 26 atoms")
    if n > cap:
        raise ValueError("more answer sets than cap")
    return buf[:n, :prog.n_atoms].copy()


def completion(prog, compact: bool = False):
    """The oracle's completion nogoods: (n_vars, off int64[n+1], lits int32)
    with literal +(v+1) = Tv, -(v+1) = Fv and the oracle's interleaved
    variable layout b_j, t_j, n_j = na+3j, na+3j+1, na+3j+2.  compact: for a
    rule with an empty positive (negative) body, {Tb_j, Ft_j} ({Tb_j, Fn_j})
    is left out and Tt_j (Tn_j) is left out of {Fb_j, Tt_j, Tn_j}."""
    b = _Bound(prog)
    lib = _load()
    nn, nl, nv = C.c_int64(), C.c_int64(), C.c_int64()
    c = 1 if compact else 0
    lib.oracle_completion(b.ref, c, C.byref(nn), C.byref(nl), C.byref(nv), None, None)
    off = np.zeros(nn.value + 1, dtype=np.int64)
    lits = np.zeros(max(nl.value, 1), dtype=np.int32)
    lib.oracle_completion(b.ref, c, C.byref(nn), C.byref(nl), C.byref(nv), _ptr(off), _ptr(lits))
    return nv.value, off, lits[:nl.value]


def up_closure(prog, partial, compact: bool = False):
    """Unit-propagation closure of a partial assignment over the oracle's
    variables (1 / -1 / 0) under its completion (compact: the compact
    variant).  Returns (conflict, closure, order, reasons)."""
    b = _Bound(prog)
    p = np.ascontiguousarray(partial, dtype=np.int8)
    nv = p.shape[0]
    clo = np.zeros(nv, dtype=np.int8)
    order = np.zeros(max(nv, 1), dtype=np.int32)
    reasons = np.zeros(max(nv, 1), dtype=np.int64)
    nd = C.c_int64()
    conflict = _load().oracle_up_closure(b.ref, 1 if compact else 0, _ptr(p), _ptr(clo), _ptr(order), _ptr(reasons),
                                         C.byref(nd))
    return bool(conflict), clo, order[:nd.value].copy(), reasons[:nd.value].copy()


def cdnl(prog, max_models: int = 0, conflict_budget: int = 0, time_budget_s: float = 0.0,
         cap: int = 1 << 14):
    """Simple CDNL solver.  Returns (status, models uint8 rows, stats dict)."""
    b = _Bound(prog)
    width = max(prog.n_atoms, 1)
    cap = int(min(cap, max_models)) if max_models > 0 else int(cap)
    cap = max(cap, 1)
    buf = np.zeros((cap, width), dtype=np.uint8)
    nm = C.c_int64()
    st = np.zeros(5, dtype=np.int64)
    status = _load().oracle_cdnl(b.ref, int(max_models), int(conflict_budget), float(time_budget_s),
                                 _ptr(buf), cap, C.byref(nm), _ptr(st))
    n = min(nm.value, cap)
    stats = dict(decisions=int(st[0]), conflicts=int(st[1]), propagations=int(st[2]),
                 learned=int(st[3]), literal_checks=int(st[4]), n_models=int(nm.value))
    return status, buf[:n, :prog.n_atoms].copy(), stats


def first_uip(delta, position, level, antecedent):
    """Resolution-based conflict analysis to the first UIP (Section 4.2,
    Algorithm 3), in plain Python over a given solver state.

    delta         the violated nogood: literals (var, is_false), all holding
    position[v]   trail position of assigned variable v (assignment order)
    level[v]      decision level of v (1 = the root)
    antecedent(v) the nogood that assigned v: literals (var, is_false) that
                  hold, plus the complement of v's own literal; None for a
                  decision

    Loop of Algorithm 3: sigma = the literal of delta assigned last; kappa =
    the highest level among the other literals of delta (0 if there are
    none); if kappa = dl(sigma), delta becomes the resolvent
    (delta minus sigma) united with (antecedent(sigma) minus the complement
    of sigma); otherwise (delta, kappa) is the result.  Returns
    (learned literals as a set, kappa, sigma = the first UIP).
    """
    d = set(delta)
    while True:
        sigma = max(d, key=lambda l: position[l[0]])
        kappa = max([level[v] for (v, f) in d if (v, f) != sigma] + [0])
        if kappa != level[sigma[0]]:
            return d, kappa, sigma
        eps = antecedent(sigma[0])
        if eps is None:
            raise ValueError("a decision shares its level with another literal of the nogood")
        comp = (sigma[0], not sigma[1])
        eps = set(eps)
        if comp not in eps:
            raise ValueError("the antecedent does not contain the complement of the literal")
        d = (d - {sigma}) | (eps - {comp})
