"""torch.autograd.Function over a KNP-EMI run: probe traces forward, adjoint sweep backward.

Forward runs ``n_steps`` IMEX steps through the C ABI (knp_step), keeping the state every
``checkpoint_every`` steps on the device, and returns phi_e at the probe points after every
step, shape (n_steps, n_probes). Backward recomputes each segment from its checkpoint and
runs knp_adjoint_step for the steps of the segment in reverse, so memory is one checkpoint
per segment plus one segment of states. Inputs with gradients: the per-facet K leak
conductance and the initial intracellular K concentration per intracellular node.
"""
from __future__ import annotations

import numpy as np
import torch

from .knp import Problem


def probe_weights(mesh_coords, elems, tag, nodes_e, N_i, N_e, points):
    """P1 interpolation of phi_e at points inside the extracellular mesh: (index [n_p, d+1]
    into the Eq. 4.3 unknown vector, weight [n_p, d+1]). Each point takes the first extracellular
    element (in element order) that contains it; elements are screened by the distance of their
    centroid, which is at most the largest element diameter from any point of the element."""
    ecell = np.nonzero(tag == 0)[0]
    d = mesh_coords.shape[1]
    loc = np.full(mesh_coords.shape[0], -1, np.int64)
    loc[nodes_e] = np.arange(len(nodes_e))
    cen = np.empty((len(ecell), d))
    diam = 0.0
    chunk = 1 << 22
    for a in range(0, len(ecell), chunk):
        x = mesh_coords[elems[ecell[a:a + chunk]]]                  # [m, d+1, d]
        cen[a:a + chunk] = x.mean(axis=1)
        diam = max(diam, float(np.sqrt(((x[:, 1:, :] - x[:, :1, :]) ** 2).sum(-1)).max()))
        for j in range(1, d + 1):
            for k in range(j + 1, d + 1):
                diam = max(diam, float(np.sqrt(((x[:, k, :] - x[:, j, :]) ** 2).sum(-1)).max()))
    idx = np.empty((len(points), d + 1), np.int64)
    wts = np.empty((len(points), d + 1))
    for p, pt in enumerate(points):
        cand = np.flatnonzero(((cen - pt) ** 2).sum(1) <= (diam * (1 + 1e-12)) ** 2)
        E = elems[ecell[cand]]
        x = mesh_coords[E]
        J = np.linalg.inv((x[:, 1:, :] - x[:, :1, :]).transpose(0, 2, 1))
        lam = np.einsum("nij,nj->ni", J, pt - x[:, 0, :])
        bary = np.concatenate([1 - lam.sum(1, keepdims=True), lam], axis=1)
        k = np.flatnonzero(np.all(bary >= -1e-12, axis=1))
        if len(k) == 0:
            raise ValueError(f"probe {p} is not in the extracellular mesh")
        k = k[0]
        idx[p] = 4 * N_i + 3 * N_e + loc[E[k]]
        wts[p] = bary[k]
    return idx, wts


class Simulation:
    """A problem with its initial state, probes and run length, for KNPFunction."""

    def __init__(self, prob: Problem, probe_idx, probe_w, n_steps: int, checkpoint_every: int = 20,
                 rtol: float = 1e-10, ion_k: int = 1, max_it: int = 1000, phi_e_floor: float = 0.0):
        self.prob = prob
        self.n_steps = n_steps
        self.k = max(1, checkpoint_every)
        self.rtol = rtol
        self.max_it = max_it
        self.phi_e_floor = phi_e_floor   # the phi_e group's floor of the stopping test (0: the library's)
        self.its_forward, self.its_adjoint = [], []   # FGMRES iterations of the last run
        self.ion_k = ion_k
        self.idx = torch.as_tensor(probe_idx, device="cuda")
        self.w = torch.as_tensor(probe_w, device="cuda", dtype=torch.float64)
        s0 = prob.state_get()
        self.s0 = s0
        self.gleak0 = None

    # state as one device vector in the Eq. 4.3 order, gates, time
    def _get(self):
        p = self.prob
        Ni, Ne = p.N_i, p.N_e
        u = torch.empty(4 * (Ni + Ne), dtype=torch.float64, device="cuda")
        c_i, phi_i = u[:3 * Ni], u[3 * Ni:4 * Ni]
        c_e, phi_e = u[4 * Ni:4 * Ni + 3 * Ne], u[4 * Ni + 3 * Ne:]
        p.state_get_device(c_i, phi_i, c_e, phi_e)
        st = p.state_get()   # gates and time (small)
        return u, st["w"].copy(), st["t"]

    def _set(self, u, w, t):
        p = self.prob
        Ni, Ne = p.N_i, p.N_e
        u = u.detach().cpu().numpy()
        p.state_set(u[:3 * Ni].reshape(3, Ni), u[3 * Ni:4 * Ni], u[4 * Ni:4 * Ni + 3 * Ne].reshape(3, Ne),
                    u[4 * Ni + 3 * Ne:], w, t)

    def probes(self, u):
        return (u[self.idx] * self.w).sum(dim=1)


class KNPFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gK_facet, cK_i0, sim: Simulation):
        p = sim.prob
        nf = p.mesh.info["n_facets"]
        gleak = np.array(sim.gleak0 if sim.gleak0 is not None else p._facet_gleak, dtype=np.float64).reshape(nf, -1)
        sim.gleak0 = gleak.copy()
        gleak[:, sim.ion_k] = gK_facet.detach().cpu().numpy()
        p.set_facet_gleak(gleak)
        s0 = sim.s0
        c_i = s0["c_i"].copy()
        c_i[sim.ion_k] = cK_i0.detach().cpu().numpy()
        p.state_set(c_i, s0["phi_i"], s0["c_e"], s0["phi_e"], s0["w"], s0["t"])
        checkpoints = []
        out = []
        sim.its_forward, sim.its_adjoint = [], []
        for n in range(sim.n_steps):
            if n % sim.k == 0:
                checkpoints.append(sim._get())
            st = p.step(1, rtol=sim.rtol, max_it=sim.max_it, phi_e_group=True, phi_e_floor=sim.phi_e_floor)
            sim.its_forward.append(st[0]["iterations"])
            u, _, _ = sim._get()
            out.append(sim.probes(u))
        ctx.sim = sim
        ctx.checkpoints = checkpoints
        return torch.stack(out)

    @staticmethod
    def backward(ctx, grad_out):
        sim = ctx.sim
        p = sim.prob
        Ni = p.N_i
        p.adjoint_begin()
        n_steps = sim.n_steps
        for seg in reversed(range(len(ctx.checkpoints))):
            n0 = seg * sim.k
            n1 = min(n_steps, n0 + sim.k)
            # recompute the segment: states u_{n0}..u_{n1}
            u, w, t = ctx.checkpoints[seg]
            sim._set(u, w, t)
            states = [(u, w, t)]
            for _ in range(n0, n1):
                p.step(1, rtol=sim.rtol, max_it=sim.max_it, phi_e_group=True, phi_e_floor=sim.phi_e_floor)
                states.append(sim._get())
            for n in range(n1, n0, -1):
                u_n = states[n - n0][0]
                dLdu = torch.zeros_like(u_n)
                dLdu.index_add_(0, sim.idx.reshape(-1), (grad_out[n - 1][:, None] * sim.w).reshape(-1))
                sim._set(*states[n - n0 - 1])
                st = p.adjoint_step(u_n, dLdu, rtol=sim.rtol, max_it=sim.max_it, phi_e_floor=sim.phi_e_floor)
                sim.its_adjoint.append(st["iterations"])
        g = p.adjoint_get()
        gK = torch.as_tensor(g["grad_gleak"][:, sim.ion_k])
        cK = torch.as_tensor(g["dLdu0"][sim.ion_k * Ni:(sim.ion_k + 1) * Ni])
        return gK, cK, None
