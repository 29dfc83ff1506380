"""Build an oracle Problem and initial State from a synthetic workload description."""
from __future__ import annotations

import numpy as np

from . import membrane, p2, system
from .topology import build_topology


def facet_inputs(cfg, topo, coords):
    """Per-facet membrane model, leak conductances and stimulus mask, in facet order."""
    n_f = len(topo.facets)
    model = np.full(n_f, cfg.model, np.int32)
    gleak = np.tile(np.asarray(cfg.g_leak, float), (n_f, 1))
    if cfg.gK_sigma:
        xi = cfg.elem_facet_xi()[topo.facet_elem_i, topo.facet_opp_i]
        gleak[:, 1] = cfg.g_leak[1] * np.exp(cfg.gK_sigma * xi)
    centroid_x = coords[topo.facets][:, :, 0].mean(axis=1)
    mask = centroid_x < cfg.stim_xmax
    return model, gleak, mask


def from_config(cfg, dt=None, pin_point=None, degree=1):
    """Oracle Problem and initial State; ``degree`` 1 (P1) or 2 (P2 Lagrange elements, Section 3.3)."""
    m = cfg.mesh
    p = cfg.params
    if degree == 1:
        topo = build_topology(m.coords, m.elems, m.elem_tag, pin_point=pin_point)
        vtopo, node_coords = topo, m.coords
    elif degree == 2:
        topo = p2.build_topology(m.coords, m.elems, m.elem_tag, pin_point=pin_point)
        vtopo, node_coords = topo.base, topo.node_coords
    else:
        raise ValueError("degree must be 1 or 2")
    model, gleak, mask = facet_inputs(cfg, vtopo, m.coords)
    pb = system.Problem(topo=topo, coords=m.coords, elems=m.elems, R=p["R"], T=p["T"], F=p["F"],
                        Cm=p["Cm"], z=np.asarray(p["z"], float), D_i=np.asarray(p["D"], float),
                        D_e=np.asarray(p["D"], float), dt=cfg.dt if dt is None else dt,
                        facet_model=model, facet_gleak=gleak, gbar_Na=p["gbar_Na"],
                        gbar_K=p["gbar_K"], phi_rest=p["phi_rest"], n_ode=25,
                        stim_kind=cfg.stim_kind, stim_gbar=cfg.stim_gbar, stim_t0=cfg.stim_t0,
                        stim_t1=cfg.stim_t1, stim_a=cfg.stim_a, stim_tau=cfg.stim_tau,
                        stim_mask=mask, rho_pump=p["rho_pump"], P_Na=p["P_Na"], P_K=p["P_K"],
                        cKe0=p["c_e0"][1])
    # E_K^0 of the Kir factor: the K reversal potential of the initial concentrations
    pb.E_K0 = float(membrane.reversal_potential(p["R"], p["T"], p["F"], p["z"][1], p["c_i0"][1], p["c_e0"][1]))
    src = cfg.source_e_at(node_coords[topo.nodes_e])
    if src is not None:
        pb.source_e = np.ascontiguousarray(src.T)
        pb.source_t0, pb.source_t1 = cfg.source_t0, cfg.source_t1
    if degree == 1:
        system.discretize(pb)
    else:
        pb.fe = p2
        p2.discretize(pb)
    s0 = system.initial_state(pb, p["c_i0"], p["c_e0"], p["phi_M0"], (p["n0"], p["m0"], p["h0"]))
    return pb, s0
