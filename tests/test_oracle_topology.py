"""Pins for oracle/topology.py: the closed-form DOF count of Section 5.1 and the
N column of Table 3, the configs' counts, and the mesh checks."""
import numpy as np
import pytest

from oracle.topology import InvalidMesh, build_topology, model_a_dof_count
from synth import make_config
from synth.configs import model_a
from synth.mesh import structured_mesh

from helpers import paper_values


def test_formula_matches_table3():
    # Table 3 header: N = 17,412 / 67,588 / 266,244 / 1,056,772 for N_x = 64..512, d = 2, p = 1
    t3 = paper_values()["table3_dof_2d_p1"]
    assert [model_a_dof_count(2, nx, 1, 3) for nx in t3["nx"]] == t3["N"]


@pytest.mark.parametrize("d,nx", [(2, 16), (2, 32), (2, 64), (2, 128), (3, 8), (3, 16)])
def test_topology_reproduces_formula(d, nx):
    cfg = model_a(d, nx, 1e-4)
    m = cfg.mesh
    t = build_topology(m.coords, m.elems, m.elem_tag)
    assert t.n_dof(3) == model_a_dof_count(d, nx, 1, 3)
    # every membrane vertex is duplicated: N_i + N_e = n_vertices + n_membrane_vertices
    assert t.N_i + t.N_e == m.coords.shape[0] + len(t.membrane_vertices)
    # closed surface of the cell: (s+1)^d - (s-1)^d vertices for side s = nx/2
    s = nx // 2
    assert len(t.membrane_vertices) == (s + 1) ** d - (s - 1) ** d


def test_config_counts():
    counts = {1: 4612, 4: 274052}
    for i, n in counts.items():
        m = make_config(i).mesh
        t = build_topology(m.coords, m.elems, m.elem_tag)
        assert t.n_dof(3) == n
    m = make_config(1).mesh
    t = build_topology(m.coords, m.elems, m.elem_tag)
    assert len(t.facets) == 64 and t.pin_vertex == 0


def test_pin_is_origin_corner():
    m = make_config(4).mesh
    t = build_topology(m.coords, m.elems, m.elem_tag)
    assert t.pin_vertex == 0 and t.loc_e[0] == 0


def test_rejects_cells_sharing_a_facet():
    coords, elems = structured_mesh(2, 4, 1.0)
    cen = coords[elems].mean(axis=1) * 4
    tag = np.zeros(len(elems), np.int32)
    tag[(cen[:, 0] > 1) & (cen[:, 0] < 2) & (cen[:, 1] > 1) & (cen[:, 1] < 3)] = 1
    tag[(cen[:, 0] > 2) & (cen[:, 0] < 3) & (cen[:, 1] > 1) & (cen[:, 1] < 3)] = 2
    with pytest.raises(InvalidMesh):
        build_topology(coords, elems, tag)


def test_rejects_regions_touching_at_a_vertex():
    coords, elems = structured_mesh(2, 6, 1.0)
    cen = coords[elems].mean(axis=1) * 6
    tag = np.zeros(len(elems), np.int32)
    tag[(cen[:, 0] > 1) & (cen[:, 0] < 3) & (cen[:, 1] > 1) & (cen[:, 1] < 3)] = 1
    tag[(cen[:, 0] > 3) & (cen[:, 0] < 5) & (cen[:, 1] > 3) & (cen[:, 1] < 5)] = 2
    with pytest.raises(InvalidMesh):
        build_topology(coords, elems, tag)
