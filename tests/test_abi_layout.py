"""The ctypes structs of the binding have the C layout of include/gs.h: a small
C program built with the host compiler prints sizeof and offsetof of every
struct and field the binding declares, and each must equal the ctypes value
(CPU only; no library call)."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _structs():
    from paper_2506_05558_gb300 import gs
    return {name: cls for name, cls in vars(gs).items()
            if name.startswith("gs_") and isinstance(cls, type) and issubclass(cls, C.Structure)}


def test_every_header_struct_is_bound():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    declared = set(re.findall(r"^typedef struct (gs_\w+) \{", src, flags=re.M))
    assert declared == set(_structs())


def test_struct_sizes_and_field_offsets_match_the_header():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = _structs()
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gs.h"', "int main(void) {"]
    for name, cls in sorted(structs.items()):
        lines.append(f'    printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    out_dir = os.path.join(ROOT, "tests", "_build")
    os.makedirs(out_dir, exist_ok=True)
    c_path, exe = os.path.join(out_dir, "layout.c"), os.path.join(out_dir, "layout")
    with open(c_path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), c_path, "-o", exe], check=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([exe], check=True, capture_output=True,
                                                               text=True).stdout.splitlines())
    mismatches = []
    for name, cls in structs.items():
        if int(got[name]) != C.sizeof(cls):
            mismatches.append((name, int(got[name]), C.sizeof(cls)))
        for field, _ in cls._fields_:
            off = getattr(cls, field).offset
            if int(got[f"{name}.{field}"]) != off:
                mismatches.append((f"{name}.{field}", int(got[f"{name}.{field}"]), off))
    assert not mismatches, mismatches
