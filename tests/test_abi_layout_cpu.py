"""The ctypes structures of the Python binding against the C header: a C program compiled
with the host compiler prints sizeof and every field's offsetof for each struct of
include/cmcg.h, and the binding's ctypes layout must agree field by field.  Needs gcc, no GPU,
no built library."""
import ctypes as C
import json
import os
import shutil
import subprocess

import pytest

from paper_1903_12522_gb300 import cmcg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "cmcg_grid": cmcg.Grid,
    "cmcg_bc": cmcg.BC,
    "cmcg_options": cmcg.Options,
    "cmcg_stats": cmcg.Stats,
    "cmcg_info": cmcg.Info,
}


def c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "cmcg.h"', "int main(void) {",
             '    printf("{");']
    first = True
    for cname, py in STRUCTS.items():
        sep = "" if first else ","
        first = False
        lines.append(f'    printf("{sep}\\"{cname}\\": {{\\"size\\": %zu", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'    printf(", \\"{field}\\": %zu", offsetof({cname}, {field}));')
        lines.append('    printf("}");')
    lines += ['    printf("}\\n");', "    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr  # a binding field the header does not have fails here
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return json.loads(out)


def test_ctypes_structs_match_the_header(tmp_path):
    lay = c_layout(tmp_path)
    for cname, py in STRUCTS.items():
        got = lay[cname]
        assert got["size"] == C.sizeof(py), (cname, got["size"], C.sizeof(py))
        for field, _ in py._fields_:
            assert got[field] == getattr(py, field).offset, (cname, field, got[field], getattr(py, field).offset)
