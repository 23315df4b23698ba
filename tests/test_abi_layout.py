"""The ctypes mirrors of the C ABI's structs have the header's layout.

A small C program built with the system compiler against include/amto.h
prints sizeof and every field's offsetof; the binding's ctypes.Structure
classes must agree field by field (a field added to the header but not to
the binding, or in another order, shifts every later field).
"""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# header struct name -> binding class name
STRUCTS = {
    "amto_params": "Params",
    "amto_info": "Info",
    "amto_server_params": "ServerParams",
    "amto_request": "Request",
    "amto_result_info": "ResultInfo",
    "amto_server_stats_t": "ServerStats",
    "amto_tune_entry": "TuneEntry",
    "amto_tune_result": "TuneResult",
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    from paper_2011_04240_b300 import amto
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "amto.h"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        cls = getattr(amto, pyname)
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f in cls._fields_:
            lines.append(f'printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    return got


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_struct_layout_matches_header(c_layout, cname):
    from paper_2011_04240_b300 import amto
    cls = getattr(amto, STRUCTS[cname])
    assert ctypes.sizeof(cls) == c_layout[(cname, "sizeof")], cname
    for f in cls._fields_:
        assert getattr(cls, f[0]).offset == c_layout[(cname, f[0])], (cname, f[0])
