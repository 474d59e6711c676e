"""The seeded input generators (no GPU): SplitMix64 against a scalar
statement of the published algorithm (state advances by the golden-ratio
increment 0x9E3779B97F4A7C15; output z ^= z >> 30, z *= 0xBF58476D1CE4E5B9,
z ^= z >> 27, z *= 0x94D049BB133111EB, z ^= z >> 31), and determinism and
shape of the program generators."""
import numpy as np

from synth.programs import (batch_programs, coloring_program, draw, program_seed, random_program,
                            tiny_program, to_unit_double)

M64 = (1 << 64) - 1


def _splitmix64_stream(state, n):
    out = []
    for _ in range(n):
        state = (state + 0x9E3779B97F4A7C15) & M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        out.append(z ^ (z >> 31))
    return out


def test_draw_is_splitmix64():
    for key in (0, 1, 1234567, program_seed(2, 0), program_seed(4, 255), M64):
        want = _splitmix64_stream(key, 16)
        got = [int(x) for x in draw(np.full(16, key, np.uint64), np.arange(16, dtype=np.uint64))]
        assert got == want, key


def test_unit_doubles_in_range():
    u = to_unit_double(draw(np.full(1000, 7, np.uint64), np.arange(1000, dtype=np.uint64)))
    assert (u >= 0).all() and (u < 1).all() and 0.4 < u.mean() < 0.6


def _same(p, q):
    return (p.n_atoms == q.n_atoms and all(np.array_equal(getattr(p, f), getattr(q, f))
                                           for f in ("head", "pos_off", "pos", "neg_off", "neg")))


def test_generators_are_deterministic():
    assert _same(tiny_program(5), tiny_program(5))
    assert not _same(tiny_program(5), tiny_program(6))
    assert _same(random_program(300, 900, program_seed(9, 1)), random_program(300, 900, program_seed(9, 1)))
    assert _same(coloring_program(30, 4.5, seed_index=2), coloring_program(30, 4.5, seed_index=2))
    a = batch_programs(3, rules_per_atom=2, lo=50, hi=200, config_id=11)
    b = batch_programs(3, rules_per_atom=2, lo=50, hi=200, config_id=11)
    assert all(_same(x, y) for x, y in zip(a, b))


def test_random_program_shape():
    p = random_program(1000, 4000, program_seed(9, 2))
    assert p.n_atoms == 1000 and p.head.shape == (4000,)
    assert ((p.head >= 0) & (p.head < 1000)).all()
    body = np.diff(p.pos_off) + np.diff(p.neg_off)
    assert body.min() >= 1 and body.max() <= 4
    for r in range(0, 4000, 97):          # distinct atoms within a body
        atoms = list(p.pos[p.pos_off[r]:p.pos_off[r + 1]]) + list(p.neg[p.neg_off[r]:p.neg_off[r + 1]])
        assert len(set(atoms)) == len(atoms)


def test_batch_blocks_equal_the_whole_batch():
    """A contiguous block of a batch (first_index) is the same programs as
    the corresponding slice of the whole batch (used to shard across ranks)."""
    whole = batch_programs(6, rules_per_atom=2, lo=50, hi=300, config_id=12)
    part = batch_programs(3, rules_per_atom=2, lo=50, hi=300, config_id=12, first_index=3)
    assert all(_same(x, y) for x, y in zip(whole[3:], part))


# ------------------------------------------------ workload families

def _proper_colourings(n, edges):
    """Every map V -> {0,1,2} with no edge inside one colour, by enumeration."""
    out = set()
    for code in range(3 ** n):
        col = [(code // 3 ** v) % 3 for v in range(n)]
        if all(col[u] != col[v] for (u, v) in edges):
            out.add(tuple(col))
    return out


def test_colouring_program_answer_sets_are_the_proper_colourings():
    """The 3-colouring encoding's answer sets (oracle CDNL, itself pinned
    against brute force) decode one to one to the proper colourings of the
    graph, enumerated directly."""
    import oracle
    from synth.programs import coloring_atom, coloring_program
    for edges in ([(0, 1), (1, 2), (2, 0)], [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2)],
                  [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)], [(0, 1), (2, 3), (3, 4)]):
        n = 1 + max(max(e) for e in edges)
        prog = coloring_program(n, edges=np.array(edges))
        status, models, _ = oracle.cdnl(prog)
        want = _proper_colourings(n, edges)
        got = set()
        for m in models:
            col = []
            for v in range(n):
                cs = [c for c in range(3) if m[coloring_atom(n, v, c)]]
                assert len(cs) == 1
                for c in range(3):            # ncol(v,c) holds exactly when col(v,c) does not
                    assert m[coloring_atom(n, v, c, True)] == (c not in cs)
                col.append(cs[0])
            got.add(tuple(col))
        assert len(models) == len(got) == len(want) and got == want
        assert status == (oracle.SAT if want else oracle.UNSAT)


def test_colouring_program_shape_and_degree():
    from synth.programs import coloring_graph, coloring_program
    edges = coloring_graph(2000, 4.5, seed_index=0)
    assert (edges[:, 0] < edges[:, 1]).all() and np.unique(edges, axis=0).shape[0] == edges.shape[0]
    assert abs(2 * edges.shape[0] / 2000 - 4.5) < 0.3          # average degree of G(n, 4.5 / (n - 1))
    prog = coloring_program(50, 4.5, seed_index=0)
    e = coloring_graph(50, 4.5, seed_index=0).shape[0]
    assert prog.n_atoms == 300
    assert prog.head.shape[0] == 6 * 50 + 4 * 50 + 3 * e
    assert int((prog.head >= 0).sum()) == 300


def test_batch_sizes_are_log_uniform():
    from synth.programs import batch_sizes
    _, n = batch_sizes(4096)
    assert n.min() >= 200 and n.max() <= 20000
    u = (np.log(n) - np.log(200)) / (np.log(20000) - np.log(200))
    # each quarter of the log range holds about a quarter of the programs
    counts = np.histogram(u, bins=4, range=(0, 1))[0]
    assert (np.abs(counts - 1024) < 120).all(), counts
