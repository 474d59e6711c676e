"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/aspgpu.h (no compute calls: runs without a GPU)."""
import os
import re

import pytest

from paper_1909_01786_gb300 import aspgpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "aspgpu.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(asp_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("asp_load_ground", "asp_solve", "asp_solve_batch", "asp_free", "asp_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    L = aspgpu.lib()
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert missing == []


def test_binding_covers_every_declared_symbol():
    assert sorted(aspgpu.EXPORTS) == _declared()


def test_library_is_compiled_for_sm_103a_only():
    """The build compiles every translation unit for sm_103a and nothing else
    (the device check of the compiled kernel is the GPU test below)."""
    from paper_1909_01786_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


@pytest.mark.gpu
def test_solve_kernel_reports_compute_capability_10_3():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    info = aspgpu.build_info()
    assert info["binary_version"] == 103, info


def test_no_device_is_a_clean_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from synth.programs import tiny_program
    with pytest.raises(aspgpu.AspError) as e:
        aspgpu.Program(tiny_program(0), torch_memory=False)
    assert e.value.code == -7


def test_bad_arguments_are_rejected_before_any_device_work():
    import ctypes as C
    import numpy as np
    L = aspgpu.lib()
    h = C.c_void_p()
    head = np.array([5], np.int32)          # atom 5 of a 2-atom program
    off = np.array([0, 0], np.int64)
    rc = L.asp_load_ground(2, 1, head.ctypes.data, off.ctypes.data, None, off.ctypes.data, None, None,
                           C.byref(h))
    assert rc in (-2, -7)                    # RANGE, or no device checked first
    rc = L.asp_load_ground(2, 1, head.ctypes.data, off.ctypes.data, None, off.ctypes.data, None, None, None)
    assert rc == -1


def _declared_arity():
    """Parameter count of every asp_* function declared in the header."""
    text = open(os.path.join(ROOT, "include", "aspgpu.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(asp_[a-z_]+)\s*\(([^;{]*?)\)\s*;", text):
        params = m.group(2).strip()
        if params in ("", "void"):
            out[m.group(1)] = 0
            continue
        depth, n = 0, 1
        for ch in params:
            depth += ch == "("
            depth -= ch == ")"
            n += ch == "," and depth == 0
        out[m.group(1)] = n
    return out


def test_binding_argument_counts_match_the_header():
    L = aspgpu.lib()
    arity = _declared_arity()
    assert set(arity) == set(aspgpu.EXPORTS)
    for name, n in arity.items():
        assert len(getattr(L, name).argtypes) == n, (name, n)
