"""The ctypes structures of the binding against the C declarations of include/discloop.h:
sizeof and every member's offset, from a host C build of the header."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

import paper_1309_2256_gb300._binding as b

HERE = os.path.dirname(os.path.abspath(__file__))
INCLUDE = os.path.join(HERE, "..", "include")

STRUCTS = {
    "dl_solve_params": b.dl_solve_params,
    "dl_solve_stats": b.dl_solve_stats,
    "dl_tsm_params": b.dl_tsm_params,
    "dl_tsm_info": b.dl_tsm_info,
    "dl_batch_params": b.dl_batch_params,
    "dl_batch_info": b.dl_batch_info,
    "dl_nn_train_params": b.dl_nn_train_params,
    "dl_fgcr_params": b.dl_fgcr_params,
    "dl_fgcr_stats": b.dl_fgcr_stats,
}


@pytest.fixture(scope="module")
def c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "discloop.h"', "int main(void) {"]
    for name, st in STRUCTS.items():
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines.append("  return 0;\n}")
    d = tempfile.mkdtemp()
    src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
    with open(src, "w") as f:
        f.write("\n".join(lines))
    subprocess.check_call([cc, "-std=c99", "-I", INCLUDE, "-o", exe, src])
    out = subprocess.check_output([exe]).decode().split("\n")
    table = {}
    for line in out:
        if line.strip():
            name, key, val = line.split()
            table[(name, key)] = int(val)
    return table


@pytest.mark.parametrize("name", sorted(STRUCTS))
def test_struct_matches_header(c_layout, name):
    st = STRUCTS[name]
    assert ctypes.sizeof(st) == c_layout[(name, "sizeof")], name
    for field, _ in st._fields_:
        assert getattr(st, field).offset == c_layout[(name, field)], (name, field)


def test_every_header_struct_is_bound():
    import re
    text = open(os.path.join(INCLUDE, "discloop.h")).read()
    declared = set(re.findall(r"}\s*(dl_\w+)\s*;", text))
    enums = set(re.findall(r"typedef enum\s*{[^}]*}\s*(dl_\w+)\s*;", text, flags=re.S))
    assert declared - enums == set(STRUCTS)
