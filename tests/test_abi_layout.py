"""The ctypes structures of the Python binding have the C header's layout:
a small C program compiled against include/aspgpu.h prints sizeof and the
offset of every field, which must equal the ctypes offsets (no GPU)."""
import os
import shutil
import subprocess

import pytest

from paper_1909_01786_gb300 import aspgpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("cname,pystruct", [("asp_options", aspgpu.Options), ("asp_stats_t", aspgpu.Stats)])
def test_struct_layout_matches_header(tmp_path, cname, pystruct):
    fields = [n for n, _ in pystruct._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "aspgpu.h"', 'int main(void) {',
             f'    printf("size %zu\\n", sizeof({cname}));']
    lines += [f'    printf("{f} %zu\\n", offsetof({cname}, {f}));' for f in fields]
    lines += ['    return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                   text=True).stdout.splitlines())
    import ctypes
    assert int(out["size"]) == ctypes.sizeof(pystruct)
    for f in fields:
        assert int(out[f]) == getattr(pystruct, f).offset, f


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_every_option_field_is_bound(tmp_path):
    """No field of asp_options is missing from the binding: the last bound
    field ends where the C struct ends (up to tail padding)."""
    import ctypes
    O = aspgpu.Options
    last = O._fields_[-1][0]
    end = getattr(O, last).offset + getattr(O, last).size
    src = tmp_path / "size.c"
    src.write_text('#include <stdio.h>\n#include "aspgpu.h"\nint main(void){printf("%zu\\n", sizeof(asp_options));return 0;}\n')
    exe = tmp_path / "size"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    size = int(subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout)
    assert size - end < 8 and size == ctypes.sizeof(O)
