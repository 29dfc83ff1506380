"""Mesh and time-step convergence of the oracle (the discrete scheme of Sections 3.2-3.3).

Self-convergence on nested meshes: the solution of one IMEX step from a smooth initial state
is computed on structured meshes with N = 16, 32, 64, 128 intervals per side, and successive
solutions are compared at the coarse mesh's vertices (every coarse vertex is a fine vertex).
The geometry is a strip cell x in (L/4, 3L/4) across the whole height, so that the membrane has
no corners (the square cell's corners are re-entrant corners of the extracellular domain, whose
singularities lower the observed orders). P1 elements give second order for the concentrations
and for the potentials up to their constant (the constant itself, fixed by the one-point pin,
converges more slowly);
the backward-Euler-type time step gives first order in dt. No manufactured solution, and so no
second derivation of the equations, is needed."""
from dataclasses import replace

import numpy as np

from oracle import problem, step
from synth import make_config
from synth.mesh import StructuredMesh, structured_mesh


def _strip(nx, dt):
    cfg = replace(make_config(1).with_nx(nx), dt=dt)
    coords, elems = structured_mesh(2, nx, cfg.length)
    cen = coords[elems].mean(axis=1) / cfg.length
    tag = ((cen[:, 0] > 0.25) & (cen[:, 0] < 0.75)).astype(np.int32)
    boxes = np.array([[[nx // 4, 0], [3 * nx // 4, nx]]])
    cfg._mesh = StructuredMesh(2, nx, coords, elems, tag, boxes, cfg.length)
    return cfg


def _run(nx, dt, n_steps):
    """n_steps from [k]_r^0 (1 + 0.1 cos(pi x/L) cos(pi y/L)) (compatible with the no-flux walls)."""
    cfg = _strip(nx, dt)
    pb, s0 = problem.from_config(cfg)
    t = pb.topo
    f = lambda x: np.cos(np.pi * x[:, 0] / cfg.length) * np.cos(np.pi * x[:, 1] / cfg.length)
    s = s0.copy()
    s.c_i = s0.c_i * (1 + 0.1 * f(pb.coords[t.nodes_i]))[None, :]
    s.c_e = s0.c_e * (1 + 0.1 * f(pb.coords[t.nodes_e]))[None, :]
    for _ in range(n_steps):
        s, _ = step.step(pb, s)
    return pb, s


def _at(pbc, pbf, r):
    """Fine-mesh region-node index of each coarse region node (same coordinates)."""
    key = {tuple(np.round(x, 12)): k for k, x in enumerate(pbf.coords[getattr(pbf.topo, "nodes_" + r)])}
    return np.array([key[tuple(np.round(x, 12))] for x in pbc.coords[getattr(pbc.topo, "nodes_" + r)]])


def _orders(errs):
    return [np.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]


def test_second_order_in_space():
    res = {nx: _run(nx, 1e-2, 1) for nx in (16, 32, 64, 128)}
    ec, ep = [], []
    for a, b in ((16, 32), (32, 64), (64, 128)):
        (pbc, sc), (pbf, sf) = res[a], res[b]
        mi, me = _at(pbc, pbf, "i"), _at(pbc, pbf, "e")
        ec.append(np.sqrt(np.mean(np.concatenate([(sc.c_i - sf.c_i[:, mi]).ravel(),
                                                   (sc.c_e - sf.c_e[:, me]).ravel()]) ** 2)))
        # the potentials are defined up to a constant, which the point pin of Remark 4.1 fixes by
        # one pointwise value; compare them without that constant (the mean difference of phi_e)
        di, de = sc.phi_i - sf.phi_i[mi], sc.phi_e - sf.phi_e[me]
        shift = de.mean()
        ep.append(np.sqrt(np.mean(np.concatenate([di - shift, de - shift]) ** 2)))
    oc, op = _orders(ec), _orders(ep)
    print("concentration orders", oc, "potential orders (up to a constant)", op)
    assert all(1.8 <= o <= 2.3 for o in oc), oc
    assert all(1.8 <= o <= 2.3 for o in op), op


def test_first_order_in_time():
    res = {n: _run(32, 8e-3 / n, n)[1] for n in (2, 4, 8, 16)}
    ec, ep = [], []
    for a, b in ((2, 4), (4, 8), (8, 16)):
        sa, sb = res[a], res[b]
        ec.append(np.linalg.norm(np.concatenate([(sa.c_i - sb.c_i).ravel(), (sa.c_e - sb.c_e).ravel()])))
        ep.append(np.linalg.norm(np.concatenate([sa.phi_i - sb.phi_i, sa.phi_e - sb.phi_e])))
    oc, op = _orders(ec), _orders(ep)
    print("concentration orders", oc, "potential orders", op)
    assert all(0.8 <= o <= 1.3 for o in oc + op), (oc, op)
