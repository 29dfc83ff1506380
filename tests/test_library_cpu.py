"""CPU checks of the C-ABI library: it loads, exports every entry point that include/knp.h
declares, and its host-side topology (knp_mesh_create) matches the oracle's. No GPU call."""
import os
import re

import numpy as np
import pytest

from oracle.topology import build_topology
from synth import make_config
from synth.configs import model_a
from synth.mesh import structured_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2403_04491_gb300.build import build_library
    build_library()
    from paper_2403_04491_gb300 import knp
    return knp.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "knp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(knp_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_2403_04491_gb300 import knp
    assert set(declared_functions()) == set(knp.SIGNATURES)


@pytest.mark.parametrize("cfg", [make_config(1), make_config(4), model_a(3, 8, 1e-4), make_config(3).with_nx(32)])
def test_mesh_topology_matches_oracle(lib, cfg):
    from paper_2403_04491_gb300 import Mesh
    m = cfg.mesh
    M = Mesh(m.coords, m.elems, m.elem_tag)
    T = build_topology(m.coords, m.elems, m.elem_tag)
    ni, ne = M.nodes()
    v, e, o, c = M.facets()
    assert M.info["n_dof"] == T.n_dof(3)
    assert np.array_equal(ni, T.nodes_i) and np.array_equal(ne, T.nodes_e)
    assert np.array_equal(v, T.facets) and np.array_equal(e, T.facet_elem_i)
    assert np.array_equal(o, T.facet_opp_i) and np.array_equal(c, T.facet_cell)
    assert M.info["pin_vertex"] == T.pin_vertex
    assert M.info["n_cells"] == int(m.elem_tag.max())


def test_config3_subset_count(lib):
    # the 32^3 version of the 125-cell workload: 192,748 unknowns
    from paper_2403_04491_gb300 import Mesh
    m = make_config(3).with_nx(32).mesh
    assert Mesh(m.coords, m.elems, m.elem_tag).info["n_dof"] == 192748


def _two_cell_mesh(touch):
    coords, elems = structured_mesh(2, 6, 1.0)
    cen = coords[elems].mean(axis=1) * 6
    tag = np.zeros(len(elems), np.int32)
    tag[(cen[:, 0] > 1) & (cen[:, 0] < 3) & (cen[:, 1] > 1) & (cen[:, 1] < 3)] = 1
    if touch == "facet":
        tag[(cen[:, 0] > 3) & (cen[:, 0] < 5) & (cen[:, 1] > 1) & (cen[:, 1] < 3)] = 2
    else:
        tag[(cen[:, 0] > 3) & (cen[:, 0] < 5) & (cen[:, 1] > 3) & (cen[:, 1] < 5)] = 2
    return coords, elems, tag


@pytest.mark.parametrize("touch", ["facet", "vertex"])
def test_invalid_meshes_are_rejected(lib, touch):
    from paper_2403_04491_gb300 import KnpError, Mesh
    coords, elems, tag = _two_cell_mesh(touch)
    with pytest.raises(KnpError) as ei:
        Mesh(coords, elems, tag)
    assert ei.value.code == 2


def test_invalid_arguments_are_rejected(lib):
    from paper_2403_04491_gb300 import KnpError, Mesh
    coords, elems = structured_mesh(2, 2, 1.0)
    bad = elems.copy()
    bad[0, 0] = 999
    with pytest.raises(KnpError) as ei:
        Mesh(coords, bad, np.zeros(len(elems), np.int32))
    assert ei.value.code == 1
    flat = coords.copy()
    flat[:, 1] = 0.0   # every element degenerate
    with pytest.raises(KnpError) as ei:
        Mesh(flat, elems, np.zeros(len(elems), np.int32))
    assert ei.value.code == 2


def test_bench_kernel_source_hash():
    """bench.py locates the finest-level Chebyshev kernel's source text (the DRAM counters it
    reports are tied to that text)."""
    import importlib
    import sys
    sys.path.insert(0, str(ROOT))
    bench = importlib.import_module("bench")
    for kind in ("cheb_fine", "spmv"):
        h = bench.kernel_source_hash(kind)
        assert isinstance(h, str) and len(h) == 16


def test_interface_refined_grid():
    """The interface-refined tensor grid: intervals next to the cell faces are cut into `ratio`
    slabs, the others keep the uniform spacing, the cells keep their snapped extent, and the
    simplices still tile the domain (volumes add up; the topology builds)."""
    from synth.mesh import make_mesh
    nx, L = 16, 1.0
    m = make_mesh(3, nx, L, np.array([[0.3] * 3]), np.array([[0.7] * 3]), refine=(3, 1))
    xs = np.unique(m.coords[:, 0])
    h = np.diff(xs) * nx / L
    assert np.allclose(np.sort(np.unique(np.round(h, 12))), [1 / 3, 1.0])
    lo, hi = m.boxes[0, 0], m.boxes[0, 1]                    # snapped to 5 and 11
    assert (lo[0], hi[0]) == (5, 11)
    # refined intervals: 4, 5 and 10, 11 (next to the planes 5 and 11)
    assert len(xs) == nx + 1 + 4 * 2
    P = m.coords[m.elems]
    vol = np.abs(np.linalg.det(P[:, 1:] - P[:, :1])) / 6
    assert abs(vol.sum() - L ** 3) < 1e-12
    assert abs(vol[m.elem_tag == 1].sum() - ((hi[0] - lo[0]) / nx * L) ** 3) < 1e-12
    t = build_topology(m.coords, m.elems, m.elem_tag)
    assert t.N_i > 0 and len(t.facets) == 6 * 2 * (3 * 2 + 4) ** 2


@pytest.mark.parametrize("where", [(1.0, 1.0), (0.5, 0.02), (0.24, 0.5)])
def test_pin_point(lib, where):
    """The phi_e pin goes on the extracellular vertex nearest to the given point (Remark 4.1 allows
    any extracellular node), in the library as in the oracle; the default is the origin."""
    from paper_2403_04491_gb300 import Mesh
    cfg = make_config(1)
    m = cfg.mesh
    pt = np.asarray(where) * cfg.length
    M = Mesh(m.coords, m.elems, m.elem_tag, pin_point=pt)
    T = build_topology(m.coords, m.elems, m.elem_tag, pin_point=pt)
    assert M.info["pin_vertex"] == T.pin_vertex
    # the nearest extracellular vertex, by brute force
    d = np.sum((m.coords[T.nodes_e] - pt) ** 2, axis=1)
    assert T.pin_vertex == T.nodes_e[np.flatnonzero(d == d.min())[0]]
    assert Mesh(m.coords, m.elems, m.elem_tag).info["pin_vertex"] == build_topology(m.coords, m.elems, m.elem_tag).pin_vertex


def test_mesh_topology_matches_oracle_threaded(lib):
    """A mesh large enough for the threaded facet matching (the 125-cell geometry at 64^3, 1.57M
    tetrahedra): the library's facets, region nodes and pin equal the oracle's."""
    from paper_2403_04491_gb300 import Mesh
    cfg = make_config(3).with_nx(64)
    m = cfg.mesh
    M = Mesh(m.coords, m.elems, m.elem_tag)
    T = build_topology(m.coords, m.elems, m.elem_tag)
    ni, ne = M.nodes()
    v, e, o, c = M.facets()
    assert M.info["n_dof"] == T.n_dof(3)
    assert np.array_equal(ni, T.nodes_i) and np.array_equal(ne, T.nodes_e)
    assert np.array_equal(v, T.facets) and np.array_equal(e, T.facet_elem_i)
    assert np.array_equal(o, T.facet_opp_i) and np.array_equal(c, T.facet_cell)
    assert M.info["pin_vertex"] == T.pin_vertex


def test_threaded_facet_matching_reports_invalid_meshes(lib):
    """The threaded facet matching rejects a mesh with a facet shared by three elements (an
    element duplicated in a large mesh) and two cells touching, as the serial one does."""
    from paper_2403_04491_gb300 import Mesh
    from paper_2403_04491_gb300.knp import KnpError
    m = make_config(2).with_nx(48).mesh
    elems = np.concatenate([m.elems, m.elems[:1]])
    tag = np.concatenate([m.elem_tag, m.elem_tag[:1]])
    with pytest.raises(KnpError, match="more than two"):
        Mesh(m.coords, elems, tag)
    tag2 = m.elem_tag.copy()
    # a second cell right next to the first: retag the extracellular elements sharing a facet with it
    T = build_topology(m.coords, m.elems, m.elem_tag)
    f0 = T.facets[0]
    share = np.flatnonzero(np.isin(m.elems, f0).sum(axis=1) == len(f0))
    tag2[share[m.elem_tag[share] == 0]] = 2
    with pytest.raises(KnpError, match="share a facet"):
        Mesh(m.coords, m.elems, tag2)


@pytest.mark.parametrize("cfg,pin", [(make_config(1), None), (make_config(4).with_nx(64), None),
                                     (model_a(3, 6, 1e-4), None), (make_config(3).with_nx(32), None),
                                     (make_config(8), None), (model_a(2, 8, 1e-4), (0.55e-6, 0.02e-6))],
                         ids=["2d-1cell", "2d-16cells", "3d-1cell", "3d-125cells", "3d-iref", "2d-pin-midpoint"])
def test_p2_nodes_match_oracle(lib, cfg, pin):
    """knp_mesh_p2_*: every P2 table equals the oracle's (oracle/p2.py) exactly."""
    from oracle import p2
    from paper_2403_04491_gb300 import Mesh
    m = cfg.mesh
    M = Mesh(m.coords, m.elems, m.elem_tag, pin_point=pin)
    T = p2.build_topology(m.coords, m.elems, m.elem_tag, pin_point=pin)
    P = M.p2()
    assert P["n_edges"] == len(T.edges) and P["n_nodes"] == len(T.node_coords)
    assert P["n_dof"] == T.n_dof(3)
    for k, ref in (("edges", T.edges), ("elem_nodes", T.elem_nodes), ("facet_nodes", T.facet_nodes),
                   ("nodes_i", T.nodes_i), ("nodes_e", T.nodes_e), ("membrane_nodes", T.membrane_nodes),
                   ("node_cell_i", T.node_cell_i)):
        assert np.array_equal(P[k], ref), k
    assert P["pin_node"] == T.pin_node
    if pin is not None:
        assert T.pin_node >= m.coords.shape[0]      # this pin point sits nearest to an edge midpoint
    # a second query returns the same tables (built once)
    assert np.array_equal(M.p2()["elem_nodes"], P["elem_nodes"])


@pytest.mark.parametrize("cfg", [make_config(1).with_nx(16), model_a(3, 4, 1e-4), make_config(8)],
                         ids=["2d", "3d", "3d-iref"])
def test_p2_region_matrices_match_oracle(lib, cfg):
    """knp_mesh_p2_region_matrices: the library's P2 M_r and A_r (the static values of its P2
    problems) and A_r^{c} for a random nodal c (the per-step kernel's element arithmetic) equal the
    oracle's to rounding."""
    from oracle import problem
    from paper_2403_04491_gb300 import Mesh
    m = cfg.mesh
    M = Mesh(m.coords, m.elems, m.elem_tag)
    pb, _ = problem.from_config(cfg, degree=2)
    from oracle import p2
    rng = np.random.default_rng(4)
    for region, r in ((0, "i"), (1, "e")):
        c = rng.uniform(1.0, 3.0, getattr(pb.topo, "N_" + r))
        Mr, Ar, Acr = M.p2_region_matrices(region, c)
        Ac_ref = p2.weighted_stiffness(pb.geo["cache_" + r], c, pb.geo["en_" + r], len(c))
        for lib_mat, ref in ((Mr, pb.geo["M_" + r]), (Ar, pb.geo["A_" + r]), (Acr, Ac_ref)):
            d = (lib_mat - ref).tocoo()
            assert lib_mat.shape == ref.shape
            assert (abs(d.data).max() if d.nnz else 0.0) <= 1e-13 * abs(ref).max()


@pytest.mark.parametrize("degree", [1, 2])
@pytest.mark.parametrize("cfg", [make_config(1).with_nx(16), make_config(7).with_nx(16), model_a(3, 4, 1e-4),
                                 make_config(4).with_nx(64)], ids=["2d-leak", "2d-kir-source", "3d-hh", "2d-16cells"])
def test_problem_host_build_reaches_the_device(lib, cfg, degree):
    """knp_problem_create without a GPU: the whole host side of the problem build (pattern, static
    values, incidences, membrane tables) runs, and the call stops at its first CUDA call with
    KNP_ERR_CUDA, not at a host check. (On a machine with a GPU this test has nothing to check.)"""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2403_04491_gb300 import KnpError, problem_from_config
    with pytest.raises(KnpError) as ei:
        problem_from_config(cfg, degree=degree)
    msg = str(ei.value)
    assert ei.value.code == 4, msg
    # the first device call of the build is an upload: cudaMalloc (P1) or the P2 tables' copy
    assert "cudaMalloc" in msg or "cudaMemcpyToSymbol" in msg, msg


def test_p2_arguments_are_checked(lib):
    import ctypes as C
    from paper_2403_04491_gb300 import KnpError, Mesh, problem_from_config
    from paper_2403_04491_gb300 import knp
    cfg = make_config(1).with_nx(8)
    m = cfg.mesh
    M = Mesh(m.coords, m.elems, m.elem_tag)
    cnt = C.c_int64()
    assert lib.knp_mesh_p2_region_matrices(M.handle, 2, None, C.byref(cnt), None, None, None, None, None) == 1
    out = np.empty(1)
    assert lib.knp_mesh_p2_region_matrices(M.handle, 0, None, C.byref(cnt), None, None, None, None,
                                           out.ctypes.data_as(knp._DP)) == 1
    assert lib.knp_mesh_p2_get_info(None, None) == 1
    # an unknown degree is refused before any device work
    with pytest.raises(KnpError) as ei:
        problem_from_config(cfg, mesh=M, degree=3)
    assert ei.value.code == 1 and "degree" in str(ei.value)


@pytest.mark.parametrize("dim,nx", [(2, 12), (3, 6)])
def test_jittered_mesh_topology_and_p2_matrices(lib, dim, nx):
    """An unstructured-looking mesh: the structured mesh with its interior vertices moved at
    random by up to a fifth of the spacing (no element inverts). The library's P1 and P2 tables,
    the pin and the P2 region matrices equal the oracle's."""
    from oracle import p2
    from oracle.topology import build_topology
    from paper_2403_04491_gb300 import Mesh
    L = 1e-6
    coords, elems = structured_mesh(dim, nx, L)
    rng = np.random.default_rng(11 + dim)
    interior = np.all((coords > 1e-12 * L) & (coords < L * (1 - 1e-12)), axis=1)
    coords = coords.copy()
    coords[interior] += rng.uniform(-0.2, 0.2, (interior.sum(), dim)) * (L / nx)
    cen = coords[elems].mean(axis=1) / L
    tag = np.all((cen > 0.3) & (cen < 0.7), axis=1).astype(np.int32)
    M = Mesh(coords, elems, tag, pin_point=np.full(dim, 0.5 * L))
    T = build_topology(coords, elems, tag, pin_point=np.full(dim, 0.5 * L))
    ni, ne = M.nodes()
    assert np.array_equal(ni, T.nodes_i) and np.array_equal(ne, T.nodes_e)
    assert M.info["pin_vertex"] == T.pin_vertex
    T2 = p2.build_topology(coords, elems, tag, pin_point=np.full(dim, 0.5 * L))
    P = M.p2()
    for k, ref in (("elem_nodes", T2.elem_nodes), ("facet_nodes", T2.facet_nodes), ("nodes_e", T2.nodes_e),
                   ("membrane_nodes", T2.membrane_nodes)):
        assert np.array_equal(P[k], ref), k
    assert P["pin_node"] == T2.pin_node
    from oracle import system
    pb = system.Problem(topo=T2, coords=coords, elems=elems, R=1, T=1, F=1, Cm=1, z=np.ones(3), D_i=np.ones(3),
                        D_e=np.ones(3), dt=1.0, facet_model=np.zeros(len(T2.facets), np.int32),
                        facet_gleak=np.zeros((len(T2.facets), 3)), fe=p2)
    p2.discretize(pb)
    c = rng.uniform(1, 2, T2.N_i)
    Mi, Ai, Aci = M.p2_region_matrices(0, c)
    Ac_ref = p2.weighted_stiffness(pb.geo["cache_i"], c, pb.geo["en_i"], T2.N_i)
    for a, b in ((Mi, pb.geo["M_i"]), (Ai, pb.geo["A_i"]), (Aci, Ac_ref)):
        d = (a - b).tocoo()
        assert (abs(d.data).max() if d.nnz else 0.0) <= 1e-12 * abs(b).max()
