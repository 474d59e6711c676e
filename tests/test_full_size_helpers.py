"""The host-side helpers of the full-size parity tests, checked without a GPU:
the vectorised oracle -> library variable map and the completion membership
index agree with the per-nogood set built by the fwd-learning tests, and the
index rejects nogoods that are not in the completion."""
import numpy as np

import oracle
from synth.programs import program_seed, random_program

from test_gpu_fwd_learning import _oracle_nogoods_in_gpu_vars
from test_gpu_full_size import _Completion, _deps_levels, _oracle_to_library
from test_gpu_solver import _gpu_to_oracle_perm


def test_variable_map_is_the_inverse_of_the_library_to_oracle_permutation():
    for seed in range(3):
        prog = random_program(200, 700, program_seed(706, seed))
        nv, _, _ = oracle.completion(prog)
        o2g = _oracle_to_library(prog, nv)
        g2o = _gpu_to_oracle_perm(prog)
        assert np.array_equal(np.sort(o2g), np.arange(nv))
        assert np.array_equal(o2g[g2o], np.arange(nv))


def test_completion_index_finds_exactly_the_completion():
    for seed in range(3):
        prog = random_program(200, 700, program_seed(706, seed))
        ref = _oracle_nogoods_in_gpu_vars(prog)
        comp = _Completion(prog)
        for ng in ref:
            assert comp.contains([2 * v + int(f) for (v, f) in ng])
        rejected = 0
        for ng in list(ref)[:400]:
            enc = [2 * v + int(f) for (v, f) in ng]
            enc[0] ^= 1                              # one literal's sign flipped
            if frozenset((l >> 1, bool(l & 1)) for l in enc) not in ref:
                assert not comp.contains(enc)
                rejected += 1
        assert rejected > 300


def test_dependency_rows_are_read_up_to_their_level():
    row = np.array([1 << 5, 1 << 0, 0xFFFF], np.uint64)   # the third word is not written below level 129
    assert _deps_levels(row, 100) == {6, 65}
    assert _deps_levels(row, 129) == {6, 65, 129, 130, 131, 132, 133, 134, 135, 136, 137, 138, 139, 140, 141,
                                      142, 143, 144}
