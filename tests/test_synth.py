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
