"""The boundary from plain C: tests/c/abi_mesh.c, compiled as C99 against include/knp.h and
linked to libknp.so, builds a mesh through knp_mesh_create (host-only, no GPU) and prints what the
library returns, which must equal the oracle's topology (P1 and P2); an out-of-range vertex id
must come back as KNP_ERR_INVALID_ARG with a message, and no handle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.topology import build_topology
from synth import make_config

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def abi_mesh(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_2403_04491_gb300.build import build_library
    lib = build_library()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path_factory.mktemp("cabi") / "abi_mesh")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_mesh.c"), "-L", libdir, "-lknp",
                    "-Wl,-rpath," + libdir, "-o", exe], check=True)
    return exe


def test_mesh_intake_from_c(abi_mesh, tmp_path):
    cfg = make_config(1)
    m = cfg.mesh
    pin = np.array([cfg.length, cfg.length])
    path = tmp_path / "mesh.bin"
    with open(path, "wb") as f:
        np.array([m.dim], np.int32).tofile(f)
        np.array([len(m.coords), len(m.elems)], np.int64).tofile(f)
        np.ascontiguousarray(m.coords, np.float64).tofile(f)
        np.ascontiguousarray(m.elems, np.int32).tofile(f)
        np.ascontiguousarray(m.elem_tag, np.int32).tofile(f)
        pin.astype(np.float64).tofile(f)
    out = subprocess.run([abi_mesh, str(path)], capture_output=True, text=True, check=True).stdout.splitlines()
    T = build_topology(m.coords, m.elems, m.elem_tag, pin_point=pin)
    info = [int(x) for x in out[0].split()[1:]]
    assert info == [2, len(m.coords), len(m.elems), T.N_i, T.N_e, len(T.facets), len(T.membrane_vertices),
                    int(m.elem_tag.max()), T.pin_vertex, T.n_dof(3)]
    facets = np.array([[int(x) for x in line.split()[1:]] for line in out if line.startswith("facet")])
    assert np.array_equal(facets[:, :2], T.facets)
    assert np.array_equal(facets[:, 2], T.facet_elem_i) and np.array_equal(facets[:, 3], T.facet_opp_i)
    assert np.array_equal(facets[:, 4], T.facet_cell)
    # P2: the counts of the P2 oracle, and 1^T M_i 1 = |Omega_i| (the P2 basis sums to one)
    from oracle import p2
    T2 = p2.build_topology(m.coords, m.elems, m.elem_tag, pin_point=pin)
    p2line = [int(x) for x in [line for line in out if line.startswith("p2 ")][0].split()[1:]]
    assert p2line == [len(T2.edges), len(T2.node_coords), T2.N_i, T2.N_e, len(T2.membrane_nodes), T2.pin_node,
                      T2.n_dof(3)]
    cnt, vol = [line for line in out if line.startswith("p2mass")][0].split()[1:]
    h = m.length / m.nx
    side = (m.boxes[0, 1] - m.boxes[0, 0]) * h
    assert int(cnt) == int((m.elem_tag > 0).sum()) * 36
    assert abs(float(vol) - side[0] * side[1]) <= 1e-13 * side[0] * side[1]
    err = [line for line in out if line.startswith("error")][0].split(maxsplit=2)
    assert int(err[1]) == 1 and "out of range" in err[2]
