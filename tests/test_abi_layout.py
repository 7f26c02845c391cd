"""The Python binding's ctypes structures mirror the C structures of include/bltc.h: the same
size and, field by field, the same offset and width, as a C compiler lays them out (gcc on this
machine compiles a probe that prints sizeof and offsetof).  A field added on one side only would
shift every later argument silently; this test fails instead."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

import paper_2003_01836_gb300 as b

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "bltc_params": b.bltc_params,
    "bltc_server_config": b.bltc_server_config,
    "bltc_request_info": b.bltc_request_info,
    "bltc_server_counters": b.bltc_server_counters,
}


def _c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bltc.h"', "int main(void) {"]
    for name, cls in STRUCTS.items():
        lines.append(f'    printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name} {field} %zu %zu\\n", offsetof({name}, {field}), '
                         f'sizeof((({name}*)0)->{field}));')
    lines += ["    return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "probe.c"), os.path.join(d, "probe")
        with open(src, "w") as f:
            f.write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                       check=True, capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        parts = line.split()
        if parts[1] == "sizeof":
            layout[(parts[0], None)] = (int(parts[2]),)
        else:
            layout[(parts[0], parts[1])] = (int(parts[2]), int(parts[3]))
    return layout


def test_ctypes_structures_match_the_header():
    layout = _c_layout()
    for name, cls in STRUCTS.items():
        assert ctypes.sizeof(cls) == layout[(name, None)][0], name
        for field, ctype in cls._fields_:
            off, width = layout[(name, field)]
            assert getattr(cls, field).offset == off, (name, field)
            assert ctypes.sizeof(ctype) == width, (name, field)


def test_tile_fields():
    # bits 0-3: the cap on a batch's source groups; bits 4-11: work items per resident block
    assert b.tile() == 0
    assert b.tile(group_cap=4) == 4
    assert b.tile(items_per_block=32) == 32 << 4
    assert b.tile(group_cap=2, items_per_block=8) == 2 | (8 << 4)
    assert b.params(4, 0.7, 100, tile=b.tile(group_cap=8)).tile == 8
