"""Seeded synthetic ground normal programs.

This module only draws random programs; it contains none of the solver's
arithmetic, so both the CPU oracle and the GPU path may consume it.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-style:

    draw(key, k) = mix64(key + (k + 1) * GAMMA)      (all arithmetic mod 2**64)

is the k-th output of a SplitMix64 generator whose state starts at ``key``.
A program with seed ``S`` gives rule ``r`` its own stream whose key is
``draw(S, r)``; the rule consumes that stream's outputs in a fixed order, so
drawing every rule of every program in lock-step (vectorised over rules)
yields exactly the same program as drawing rule after rule.

``uniform(n)`` takes the next output ``x`` and rejects it while
``x >= 2**64 - (2**64 mod n)`` (no modulo bias), then returns ``x mod n``.

Program format (the boundary's input format): ``n_atoms`` atoms numbered
``0..n_atoms-1``; rule ``r`` has ``head[r]`` (``-1`` for an integrity
constraint), positive body ``pos[pos_off[r]:pos_off[r+1]]`` and negative body
``neg[neg_off[r]:neg_off[r+1]]``.  This is the rule form
``p0 <- p1..pm, not pm+1..not pn`` of the paper's Section 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)
_U64 = np.uint64


@dataclass
class Program:
    n_atoms: int
    head: np.ndarray      # int32 [n_rules], -1 = integrity constraint
    pos_off: np.ndarray   # int64 [n_rules + 1]
    pos: np.ndarray       # int32
    neg_off: np.ndarray   # int64 [n_rules + 1]
    neg: np.ndarray       # int32

    @property
    def n_rules(self) -> int:
        return int(self.head.shape[0])

    def rules(self):
        """Yield (head, [pos atoms], [neg atoms]) per rule (small programs)."""
        for r in range(self.n_rules):
            yield (int(self.head[r]),
                   [int(a) for a in self.pos[self.pos_off[r]:self.pos_off[r + 1]]],
                   [int(a) for a in self.neg[self.neg_off[r]:self.neg_off[r + 1]]])


def from_rules(n_atoms: int, rules) -> Program:
    """Build a Program from a list of (head, pos_list, neg_list)."""
    head = np.array([r[0] for r in rules], dtype=np.int32)
    pl = [list(r[1]) for r in rules]
    nl = [list(r[2]) for r in rules]
    pos_off = np.zeros(len(rules) + 1, dtype=np.int64)
    neg_off = np.zeros(len(rules) + 1, dtype=np.int64)
    pos_off[1:] = np.cumsum([len(x) for x in pl]) if rules else []
    neg_off[1:] = np.cumsum([len(x) for x in nl]) if rules else []
    pos = np.array([a for x in pl for a in x], dtype=np.int32)
    neg = np.array([a for x in nl for a in x], dtype=np.int32)
    return Program(n_atoms, head, pos_off, pos, neg_off, neg)


# ---------------------------------------------------------------- SplitMix64

def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea & Flood 2014)."""
    with np.errstate(over="ignore"):
        z = np.asarray(z, dtype=_U64).copy()
        z ^= z >> _U64(30)
        z *= _C1
        z ^= z >> _U64(27)
        z *= _C2
        z ^= z >> _U64(31)
    return z


def draw(key, k) -> np.ndarray:
    """k-th output of the SplitMix64 generator whose state starts at key."""
    with np.errstate(over="ignore"):
        key = np.asarray(key, dtype=_U64)
        k = np.asarray(k, dtype=_U64)
        return mix64(key + (k + _U64(1)) * GAMMA)


def to_unit_double(x: np.ndarray) -> np.ndarray:
    """Top 53 bits of x as a double in [0, 1)."""
    return (np.asarray(x, dtype=_U64) >> _U64(11)).astype(np.float64) * (2.0 ** -53)


class Streams:
    """One SplitMix64 stream per lane, advanced in lock-step."""

    def __init__(self, keys: np.ndarray):
        self.keys = np.asarray(keys, dtype=_U64)
        self.ctr = np.zeros(self.keys.shape[0], dtype=_U64)

    def raw(self, lanes: np.ndarray) -> np.ndarray:
        x = draw(self.keys[lanes], self.ctr[lanes])
        self.ctr[lanes] += _U64(1)
        return x

    def uniform(self, n, lanes: np.ndarray | None = None) -> np.ndarray:
        """Unbiased integer in [0, n) per lane (n scalar or per-lane array)."""
        if lanes is None:
            lanes = np.arange(self.keys.shape[0])
        lanes = np.asarray(lanes, dtype=np.int64)
        n = np.broadcast_to(np.asarray(n, dtype=_U64), lanes.shape).copy()
        with np.errstate(over="ignore"):
            rem = (_U64(0) - n) % n            # 2**64 mod n
            lim = _U64(0) - rem                # 2**64 - rem (unused when rem == 0)
        out = np.empty(lanes.shape[0], dtype=_U64)
        pend = np.arange(lanes.shape[0])
        while pend.size:
            x = self.raw(lanes[pend])
            ok = (rem[pend] == 0) | (x < lim[pend])
            out[pend[ok]] = x[ok] % n[pend[ok]]
            pend = pend[~ok]
        return out.astype(np.int64)


def program_seed(config_id: int, index: int) -> int:
    return ((config_id & 0xFFFFFFFF) << 32) | (index & 0xFFFFFFFF)


# ---------------------------------------------------------------- generators

def _assemble(n_atoms, head, body, sign, k):
    """Rules with up to 4 body slots -> Program (slot order kept)."""
    nr = head.shape[0]
    slots = np.arange(body.shape[1])[None, :] < k[:, None]
    is_pos = slots & (sign == 0)
    is_neg = slots & (sign == 1)
    pos_cnt = is_pos.sum(1)
    neg_cnt = is_neg.sum(1)
    pos_off = np.zeros(nr + 1, dtype=np.int64)
    neg_off = np.zeros(nr + 1, dtype=np.int64)
    np.cumsum(pos_cnt, out=pos_off[1:])
    np.cumsum(neg_cnt, out=neg_off[1:])
    pos = body[is_pos].astype(np.int32)     # row-major: rule order, then slot order
    neg = body[is_neg].astype(np.int32)
    return Program(int(n_atoms), head.astype(np.int32), pos_off, pos, neg_off, neg)


def _draw_distinct(st: Streams, lanes, n, body, j):
    """Slot j of each lane: uniform atom distinct from slots 0..j-1."""
    pend = np.asarray(lanes, dtype=np.int64)
    nn = np.broadcast_to(np.asarray(n, dtype=np.int64), (body.shape[0],))
    while pend.size:
        a = st.uniform(nn[pend].astype(np.uint64), pend)
        dup = (body[pend, :j] == a[:, None]).any(axis=1) if j else np.zeros(pend.size, bool)
        body[pend[~dup], j] = a[~dup]
        pend = pend[dup]


def _random_rules(seeds: np.ndarray, rule_idx: np.ndarray, n_atoms: np.ndarray):
    """Lock-step draw of 'random family' rules.

    Per rule: head = uniform(n), k = 1 + uniform(4), then for each of the k
    slots an atom uniform over atoms not yet in this body followed by a sign
    bit uniform(2) (1 = negated).
    """
    st = Streams(draw(seeds, rule_idx))
    n_u = n_atoms.astype(np.uint64)
    nr = seeds.shape[0]
    head = st.uniform(n_u)
    k = 1 + st.uniform(4)
    body = np.full((nr, 4), -1, dtype=np.int64)
    sign = np.zeros((nr, 4), dtype=np.int64)
    for j in range(4):
        lanes = np.nonzero(k > j)[0]
        _draw_distinct(st, lanes, n_atoms, body, j)
        sign[lanes, j] = st.uniform(2, lanes)
    return head, body, sign, k


def random_program(n_atoms: int, n_rules: int, seed: int) -> Program:
    """Random ground normal program: heads uniform, body size uniform in 1..4,
    distinct body atoms drawn uniformly, each negated with probability 1/2."""
    if n_atoms < 4:
        raise ValueError("random_program needs at least 4 atoms")
    seeds = np.full(n_rules, seed, dtype=np.uint64)
    ridx = np.arange(n_rules, dtype=np.uint64)
    head, body, sign, k = _random_rules(seeds, ridx, np.full(n_rules, n_atoms, dtype=np.int64))
    return _assemble(n_atoms, head, body, sign, k)


def large_random_program(seed_index: int = 0, n_atoms: int = 100_000, n_rules: int = 400_000):
    """Single large random program (100k atoms, 400k rules by default)."""
    return random_program(n_atoms, n_rules, program_seed(2, seed_index))


def tiny_program(index: int, n_atoms: int = 20, n_rules: int = 40, n_constraints: int = 3) -> Program:
    """Tiny random program: heads uniform, |B+| and |B-| uniform in 0..2 with all
    body atoms distinct (never both p and not p), plus integrity constraints of
    two distinct atoms, each negated with probability 1/2.

    Rule r draws: head, |B+|, |B-|, the B+ atoms, then the B- atoms.
    Constraint c (stream index n_rules + c) draws: atom, sign, atom, sign.
    """
    seed = program_seed(1, index)
    st = Streams(draw(np.full(n_rules, seed, dtype=np.uint64), np.arange(n_rules, dtype=np.uint64)))
    head = st.uniform(n_atoms)
    npos = st.uniform(3)
    nneg = st.uniform(3)
    body = np.full((n_rules, 4), -1, dtype=np.int64)
    for j in range(2):
        _draw_distinct(st, np.nonzero(npos > j)[0], n_atoms, body, j)
    # negative atoms: distinct from the positive ones and from each other
    rules = []
    negs = np.full((n_rules, 2), -1, dtype=np.int64)
    for j in range(2):
        pend = np.nonzero(nneg > j)[0]
        while pend.size:
            a = st.uniform(n_atoms, pend)
            dup = (body[pend] == a[:, None]).any(axis=1)
            dup |= (negs[pend, :j] == a[:, None]).any(axis=1)
            negs[pend[~dup], j] = a[~dup]
            pend = pend[dup]
    for r in range(n_rules):
        rules.append((int(head[r]), [int(x) for x in body[r, :npos[r]]], [int(x) for x in negs[r, :nneg[r]]]))
    cst = Streams(draw(np.full(n_constraints, seed, dtype=np.uint64),
                       np.arange(n_rules, n_rules + n_constraints, dtype=np.uint64)))
    cb = np.full((n_constraints, 4), -1, dtype=np.int64)
    csign = np.zeros((n_constraints, 2), dtype=np.int64)
    allc = np.arange(n_constraints)
    _draw_distinct(cst, allc, n_atoms, cb, 0)
    csign[:, 0] = cst.uniform(2, allc)
    _draw_distinct(cst, allc, n_atoms, cb, 1)
    csign[:, 1] = cst.uniform(2, allc)
    for c in range(n_constraints):
        pos = [int(cb[c, j]) for j in range(2) if csign[c, j] == 0]
        neg = [int(cb[c, j]) for j in range(2) if csign[c, j] == 1]
        rules.append((-1, pos, neg))
    return from_rules(n_atoms, rules)


def coloring_graph(n: int = 2000, avg_degree: float = 4.5, seed_index: int = 0):
    """G(n, p) with p = avg_degree / (n - 1): pair (u, v), u < v, taken in
    lexicographic order with pair index e, is an edge iff
    unit_double(draw(seed, e)) < p."""
    seed = program_seed(3, seed_index)
    p = avg_degree / (n - 1)
    iu, iv = np.triu_indices(n, k=1)
    e = np.arange(iu.shape[0], dtype=np.uint64)
    keep = to_unit_double(draw(np.uint64(seed), e)) < p
    return np.stack([iu[keep], iv[keep]], axis=1).astype(np.int64)


def coloring_atom(n: int, v: int, c: int, negated: bool = False) -> int:
    """col(v,c) = 3v + c; ncol(v,c) = 3n + 3v + c."""
    return (3 * n if negated else 0) + 3 * v + c


def coloring_program(n: int = 2000, avg_degree: float = 4.5, seed_index: int = 0, edges=None) -> Program:
    """Ground 3-colouring: per vertex and colour an even negative loop
    col(v,c) :- not ncol(v,c).  ncol(v,c) :- not col(v,c).
    at-least-one  :- not col(v,0), not col(v,1), not col(v,2).
    at-most-one   :- col(v,c1), col(v,c2).  (c1 < c2)
    per edge and colour  :- col(u,c), col(v,c)."""
    if edges is None:
        edges = coloring_graph(n, avg_degree, seed_index)
    rules = []
    for v in range(n):
        for c in range(3):
            a, na_ = coloring_atom(n, v, c), coloring_atom(n, v, c, True)
            rules.append((a, [], [na_]))
            rules.append((na_, [], [a]))
    for v in range(n):
        rules.append((-1, [], [coloring_atom(n, v, c) for c in range(3)]))
        for c1 in range(3):
            for c2 in range(c1 + 1, 3):
                rules.append((-1, [coloring_atom(n, v, c1), coloring_atom(n, v, c2)], []))
    for (u, v) in edges:
        for c in range(3):
            rules.append((-1, [coloring_atom(n, int(u), c), coloring_atom(n, int(v), c)], []))
    return from_rules(6 * n, rules)


def batch_sizes(count: int, lo: int = 200, hi: int = 20000, config_id: int = 4, first_index: int = 0):
    """Atom counts log-uniform in [lo, hi]: n = round(exp(ln lo + u (ln hi - ln lo)))
    with u = unit_double(draw(seed_i, 2**62))."""
    seeds = np.array([program_seed(config_id, first_index + i) for i in range(count)], dtype=np.uint64)
    u = to_unit_double(draw(seeds, np.full(count, 1 << 62, dtype=np.uint64)))
    n = np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    return seeds, n


def batch_programs(count: int, rules_per_atom: int = 4, config_id: int = 4, first_index: int = 0,
                   lo: int = 200, hi: int = 20000):
    """Batch of random-family programs with log-uniform atom counts and
    rules = rules_per_atom x atoms; all rules of all programs drawn in lock-step."""
    seeds, n = batch_sizes(count, lo, hi, config_id, first_index)
    nrules = n * rules_per_atom
    lane_seed = np.repeat(seeds, nrules)
    starts = np.zeros(count + 1, dtype=np.int64)
    np.cumsum(nrules, out=starts[1:])
    ridx = (np.arange(starts[-1], dtype=np.int64) - np.repeat(starts[:-1], nrules)).astype(np.uint64)
    lane_n = np.repeat(n, nrules)
    head, body, sign, k = _random_rules(lane_seed, ridx, lane_n)
    progs = []
    for i in range(count):
        s, e = starts[i], starts[i + 1]
        progs.append(_assemble(int(n[i]), head[s:e], body[s:e], sign[s:e], k[s:e]))
    return progs
