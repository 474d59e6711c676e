"""asp_propagate_noalloc: propagation for callers that cannot allocate device
memory where they need it (real-time loops that must stay out of the
allocator, processes whose device memory a pool or framework hands out up
front).  Its working memory is a static device array inside the library, so
the test checks, through the C ABI, that it gives the same closure as the
allocating entry point asp_debug_propagate on two calls in a row, and that it
refuses a program larger than the array.  Collected last so that a failure here never
hides another test's result."""
import ctypes as C

import numpy as np
import pytest

from synth.programs import program_seed, random_program

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1909_01786_gb300 import aspgpu
    return torch, aspgpu


def _noalloc(torch, aspgpu, P, partial):
    dev = torch.device("cuda")
    d_partial = torch.from_numpy(partial).to(dev)
    d_closure = torch.full((P.n_vars,), 7, dtype=torch.int8, device=dev)
    d_conflict = torch.full((1,), 7, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    L = aspgpu.lib()
    rc = L.asp_propagate_noalloc(P.handle, d_partial.data_ptr(), d_closure.data_ptr(), d_conflict.data_ptr())
    assert rc == 0, L.asp_last_error().decode()
    torch.cuda.synchronize()
    return int(d_conflict.item()), d_closure.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice(env):
    torch, aspgpu = env
    prog = random_program(3000, 9000, program_seed(301, 0))
    P = aspgpu.Program(prog)
    rng = np.random.default_rng(5)
    partial = np.zeros(P.n_vars, np.int8)     # first call: the root closure
    compared = 0
    for call in range(2):                     # the static array is reused
        want_conflict, want = P.propagate(partial)
        got_conflict, got = _noalloc(torch, aspgpu, P, partial)
        assert got_conflict in (0, 1)
        assert bool(got_conflict) == want_conflict
        if not want_conflict:                 # the fixpoint is unique
            assert (got == want).all(), call
            compared += 1
            # second call: extend the closure by a few open atoms
            open_atoms = np.nonzero(want[:prog.n_atoms] == 0)[0]
            pick = rng.choice(open_atoms, size=min(6, open_atoms.shape[0]), replace=False)
            partial = want.copy()
            partial[pick] = rng.choice([-1, 1], size=pick.shape[0])
    assert compared >= 1


def test_noalloc_rejects_programs_beyond_its_array(env):
    torch, aspgpu = env
    prog = random_program(200_000, 300_000, program_seed(301, 1))    # 1.1M variables > 2^20
    P = aspgpu.Program(prog)
    assert P.n_vars > (1 << 20)
    dev = torch.device("cuda")
    buf8 = torch.zeros(P.n_vars, dtype=torch.int8, device=dev)
    out8 = torch.zeros(P.n_vars, dtype=torch.int8, device=dev)
    conf = torch.zeros(1, dtype=torch.int32, device=dev)
    L = aspgpu.lib()
    rc = L.asp_propagate_noalloc(P.handle, buf8.data_ptr(), out8.data_ptr(), conf.data_ptr())
    assert rc == -5
    assert b"2^20" in L.asp_last_error()
