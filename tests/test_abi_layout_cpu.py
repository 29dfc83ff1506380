"""The ctypes structures of the binding against the C header: every field at the same offset and
every structure of the same size, read from a small C program compiled with gcc against
include/knp.h (no GPU and no library needed). A field added to the header but not to the binding
(or the reverse) shifts an offset or the size and fails here."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2403_04491_gb300 import knp as K

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# binding structure -> C type
PAIRS = {
    "MeshDesc": "knp_mesh_desc",
    "P2Info": "knp_p2_info",
    "MeshInfo": "knp_mesh_info",
    "ProblemDesc": "knp_problem_desc",
    "AmgOpts": "knp_amg_opts",
    "AmgSetupRecord": "knp_amg_setup_record",
    "SolveOpts": "knp_solve_opts",
    "SolveStats": "knp_solve_stats",
    "ProblemInfo": "knp_problem_info",
    "StepStats": "knp_step_stats",
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "knp.h"', "int main(void) {"]
    for py, c in PAIRS.items():
        lines.append(f'    printf("{py} size %zu\\n", sizeof({c}));')
        for name, _ in getattr(K, py)._fields_:
            lines.append(f'    printf("{py} {name} %zu\\n", offsetof({c}, {name}));')
    lines += ["    return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        py, name, val = line.split()
        table[py, name] = int(val)
    return table


@pytest.mark.parametrize("py", list(PAIRS))
def test_binding_structure_matches_header(c_layout, py):
    cls = getattr(K, py)
    assert ctypes.sizeof(cls) == c_layout[py, "size"], py
    for name, _ in cls._fields_:
        assert getattr(cls, name).offset == c_layout[py, name], (py, name)
