"""Property tests of the oracle on random inputs (hypothesis): for random 2D meshes (jittered
structured grids), random box cells, random leak conductances and time steps, and P1 or P2
elements, one step of the scheme conserves the charge of every cell and of the extracellular
space (Section 2.2) and reproduces a random manufactured discrete solution; and the library's
host topology (P1 and P2 tables, pins) equals the oracle's on the same random meshes."""
from dataclasses import replace

import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st

from oracle import problem, solve, step, system
from synth import make_config
from synth.configs import MODEL_LEAK
from synth.mesh import StructuredMesh, structured_mesh


def _random_cfg(seed, nx, lo, hi, g, dt, jitter):
    cfg = replace(make_config(1).with_nx(nx), model=MODEL_LEAK, g_leak=g, dt=dt)
    coords, elems = structured_mesh(2, nx, cfg.length)
    rng = np.random.default_rng(seed)
    inner = np.all((coords > 1e-9 * cfg.length) & (coords < cfg.length * (1 - 1e-9)), axis=1)
    coords = coords.copy()
    coords[inner] += rng.uniform(-jitter, jitter, (inner.sum(), 2)) * cfg.length / nx
    # tag by the undisturbed grid boxes so that the cell stays a union of whole boxes
    base, _ = structured_mesh(2, nx, cfg.length)
    cen = base[elems].mean(axis=1) / cfg.length * nx
    tag = np.all((cen > np.array(lo)) & (cen < np.array(hi)), axis=1).astype(np.int32)
    cfg._mesh = StructuredMesh(2, nx, coords, elems, tag, np.array([[lo, hi]]), cfg.length)
    return cfg


def _charges(pb, s):
    g, z = pb.geo, pb.z
    qi = sum(z[k] * (g["M_i"] @ s.c_i[k]) for k in range(pb.n_ions))
    per_cell = np.bincount(pb.topo.node_cell_i, weights=qi)
    qe = sum(z[k] * (g["M_e"] @ s.c_e[k]).sum() for k in range(pb.n_ions))
    scale = sum(abs(z[k]) * (g["M_e"] @ s.c_e[k]).sum() for k in range(pb.n_ions))
    return per_cell, qe, scale


@settings(max_examples=40, deadline=None, derandomize=True)
@given(seed=st.integers(0, 10_000), nx=st.sampled_from([8, 10, 12]), x0=st.integers(1, 3), y0=st.integers(1, 3),
       wx=st.integers(2, 4), wy=st.integers(2, 4), gNa=st.floats(0.0, 2.0), gK=st.floats(0.1, 8.0),
       dt=st.sampled_from([1e-5, 1e-4, 1e-3]), jitter=st.floats(0.0, 0.25), degree=st.sampled_from([1, 2]))
def test_random_problems_conserve_charge_and_solve_exactly(seed, nx, x0, y0, wx, wy, gNa, gK, dt, jitter, degree):
    lo, hi = [x0, y0], [min(x0 + wx, nx - 1), min(y0 + wy, nx - 1)]
    cfg = _random_cfg(seed, nx, lo, hi, (gNa, gK, 0.0), dt, jitter)
    pb, s0 = problem.from_config(cfg, degree=degree)
    c0, e0, scale = _charges(pb, s0)
    s1, _ = step.step(pb, s0)
    c1, e1, _ = _charges(pb, s1)
    assert np.abs(c1 - c0).max() < 1e-12 * scale
    assert abs(e1 - e0) < 1e-12 * scale
    A, f, _ = system.assemble(pb, s0)
    rng = np.random.default_rng(seed)
    u_star = system.pack(pb, s0) * (1 + 0.01 * rng.standard_normal(A.shape[0]))
    u_star[system.pin_dof(pb)] = 0.0
    u = solve.direct(A, A @ u_star)
    assert np.linalg.norm(u - u_star) <= 1e-11 * np.linalg.norm(u_star)


@pytest.fixture(scope="module")
def lib():
    from paper_2403_04491_gb300.build import build_library
    build_library()
    from paper_2403_04491_gb300 import knp
    return knp.load_library()


@settings(max_examples=25, deadline=None, derandomize=True)
@given(seed=st.integers(0, 10_000), nx=st.sampled_from([6, 9, 12]), x0=st.integers(1, 2), y0=st.integers(1, 2),
       wx=st.integers(1, 3), wy=st.integers(1, 3), jitter=st.floats(0.0, 0.25),
       px=st.floats(-0.2, 1.2), py=st.floats(-0.2, 1.2))
def test_library_topology_on_random_meshes(lib, seed, nx, x0, y0, wx, wy, jitter, px, py):
    from oracle import p2
    from oracle.topology import build_topology
    from paper_2403_04491_gb300 import Mesh
    lo, hi = [x0, y0], [min(x0 + wx, nx - 1), min(y0 + wy, nx - 1)]
    cfg = _random_cfg(seed, nx, lo, hi, (0.2, 0.8, 0.0), 1e-4, jitter)
    m = cfg.mesh
    pin = np.array([px, py]) * cfg.length
    M = Mesh(m.coords, m.elems, m.elem_tag, pin_point=pin)
    T = build_topology(m.coords, m.elems, m.elem_tag, pin_point=pin)
    ni, ne = M.nodes()
    v, e, o, c = M.facets()
    assert np.array_equal(ni, T.nodes_i) and np.array_equal(ne, T.nodes_e)
    assert np.array_equal(v, T.facets) and np.array_equal(e, T.facet_elem_i) and np.array_equal(o, T.facet_opp_i)
    assert M.info["pin_vertex"] == T.pin_vertex
    T2 = p2.build_topology(m.coords, m.elems, m.elem_tag, pin_point=pin)
    P = M.p2()
    for k, ref in (("edges", T2.edges), ("elem_nodes", T2.elem_nodes), ("facet_nodes", T2.facet_nodes),
                   ("nodes_i", T2.nodes_i), ("nodes_e", T2.nodes_e), ("membrane_nodes", T2.membrane_nodes),
                   ("node_cell_i", T2.node_cell_i)):
        assert np.array_equal(P[k], ref), k
    assert P["pin_node"] == T2.pin_node
