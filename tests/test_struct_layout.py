"""The ctypes mirrors of the C ABI's structs in the Python binding have the C layout (CPU).

For every ctypes.Structure the binding declares under a C typedef name, a small C program compiled by
gcc against include/fhash.h and include/fhash_serve.h prints sizeof the struct and offsetof each
field; the binding's ctypes.sizeof and field offsets must be the same, field by field and in the same
order.  A field added, dropped, reordered or retyped on one side only fails here, on the CPU, before a
GPU call could read or write the wrong bytes.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _binding():
    import paper_2507_03836_gb300 as p
    return p


def _structs():
    p = _binding()
    out = []
    for name in dir(p):
        obj = getattr(p, name)
        if isinstance(obj, type) and issubclass(obj, ctypes.Structure) and name.startswith("fhash_"):
            out.append((name, obj))
    return out


def test_binding_structs_match_the_headers(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = _structs()
    assert len(structs) >= 9, [n for n, _ in structs]
    lines = ['#include "fhash.h"', '#include "fhash_serve.h"', "#include <stdio.h>", "#include <stddef.h>",
             "int main(void) {"]
    for name, cls in structs:
        lines.append('    printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for fname, _ in cls._fields_:
            lines.append('    printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, fname, name, fname))
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        key, val = line.split()
        got[key] = int(val)
    for name, cls in structs:
        assert ctypes.sizeof(cls) == got[name], (name, ctypes.sizeof(cls), got[name])
        for fname, _ in cls._fields_:
            assert getattr(cls, fname).offset == got["%s.%s" % (name, fname)], (name, fname)
