"""The linearised KNP-EMI system A_{n-1} u_n = f_n and the preconditioner P_0 (Section 4).

Unknown order (Eq. 4.3): [c_i^1 .. c_i^|K|, phi_i, c_e^1 .. c_e^|K|, phi_e], each
block in region node order. Blocks follow the matrices A_r^n and B_rq^n of
Section 4.1 with tau_r^k = dt D_r^k and tau~_r^k = tau_r^k z_k / psi, psi = RT/F.

Readings where the paper is silent or inconsistent:
  * the bulk source enters the right-hand side multiplied by dt (Eq. 3.5 omits it), with
    nodal values, evaluated at t_n (f_r^{k,n} of Section 3.2);
  * Kir-Na/K facets (Section 2.4.2): the rectification factor and the pump flux are nodal, like
    every other membrane coefficient; E_K^0 and [K]_e^0 are the initial (uniform) values;
  * h_r = +-_r (dt I_ch - C_m phi_M^{n-1}) / F: the printed "+C_m phi_M" contradicts a
    re-derivation of h_r in Eq. 3.7 from Eq. 3.2 with the backward difference of Section 3.2;
  * alpha and C are nodal P1 on Gamma; int_Gamma C phi_M v is the exact triple product,
    on both sides of the equation;
  * the stimulus conductance is evaluated at t_{n-1} (explicit I_ch);
  * null space: the phi_e row and column of the extracellular node nearest to the origin
    are replaced by the identity with right-hand side 0 (Remark 4.1);
  * P_0 = blockdiag(M_r + tau_r^k A_r, C_m/F M_{r,Gamma} + sum_k z_k tau~_r^k A_r^{k,0}) with the
    same pin (Eq. 4.4, P_n reused as P_0).
Pinned by tests/test_oracle_system.py (resting steady state, charge conservation,
species mass balance, zero residual of a manufactured solution, LU(P_0)-GMRES
iteration counts of Section 6.3).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import fem, membrane
from .topology import Topology, build_topology

LEAK, HH, KIR = 0, 1, 2


@dataclass
class Problem:
    topo: Topology
    coords: np.ndarray
    elems: np.ndarray
    R: float
    T: float
    F: float
    Cm: float
    z: np.ndarray
    D_i: np.ndarray
    D_e: np.ndarray
    dt: float
    facet_model: np.ndarray            # (n_f,) LEAK or HH
    facet_gleak: np.ndarray            # (n_f, n_ions) S/m^2
    gbar_Na: float = 1200.0
    gbar_K: float = 360.0
    phi_rest: float = -65e-3
    n_ode: int = 25
    stim_kind: int = 0
    stim_gbar: float = 0.0
    stim_t0: float = 0.0
    stim_t1: float = 0.0
    stim_a: float = 2e-3
    stim_tau: float = 10e-3
    stim_mask: np.ndarray = None       # (n_f,) bool
    # Kir-Na/K (Section 2.4.2): pump constants, E_K^0 and [K]_e^0 (t = 0 values)
    rho_pump: float = 1.115e-6
    P_Na: float = 10.0
    P_K: float = 1.5
    E_K0: float = 0.0
    cKe0: float = 4.0
    # bulk source f_r^k(x, t_n) (mol/(m^3 s)): nodal values per region, (n_ions, N_r), switched on
    # for source_t0 < t_n <= source_t1; None = no source
    source_i: np.ndarray = None
    source_e: np.ndarray = None
    source_t0: float = 0.0
    source_t1: float = 0.0
    geo: dict = field(default_factory=dict)
    # the finite-element space's matrix routines: fem (P1) or p2 (P2)
    fe: object = fem

    @property
    def psi(self):
        return self.R * self.T / self.F

    @property
    def n_ions(self):
        return len(self.z)


def discretize(pb: Problem) -> None:
    """Static geometry: M_r, A_r, element caches, facet measures and node maps."""
    t = pb.topo
    g = pb.geo
    g["M_i"], g["A_i"], g["cache_i"] = fem.assemble_bulk(pb.coords, pb.elems[t.elems_i], t.loc_i, t.N_i)
    g["M_e"], g["A_e"], g["cache_e"] = fem.assemble_bulk(pb.coords, pb.elems[t.elems_e], t.loc_e, t.N_e)
    g["en_i"] = t.loc_i[pb.elems[t.elems_i]]
    g["en_e"] = t.loc_e[pb.elems[t.elems_e]]
    g["area"] = fem.facet_measure(pb.coords, t.facets)
    g["fv"] = np.searchsorted(t.membrane_vertices, t.facets)        # facet vertex -> membrane index
    g["fi"] = t.loc_i[t.facets]
    g["fe"] = t.loc_e[t.facets]
    g["mv_i"] = t.loc_i[t.membrane_vertices]
    g["mv_e"] = t.loc_e[t.membrane_vertices]
    g["pin"] = int(t.loc_e[t.pin_vertex])
    n_mv = len(t.membrane_vertices)
    # plain membrane masses
    g["MG_i"] = fem.membrane_mass(g["area"], g["fi"], g["fi"], t.N_i, t.N_i)
    g["MG_e"] = fem.membrane_mass(g["area"], g["fe"], g["fe"], t.N_e, t.N_e)
    g["MG_ie"] = fem.membrane_mass(g["area"], g["fi"], g["fe"], t.N_i, t.N_e)
    g["MG_ei"] = fem.membrane_mass(g["area"], g["fe"], g["fi"], t.N_e, t.N_i)
    g["n_mv"] = n_mv
    if pb.stim_mask is None:
        pb.stim_mask = np.ones(len(t.facets), bool)


def make_problem(coords, elems, tag, params: dict, dt, facet_model, facet_gleak, **kw) -> Problem:
    topo = build_topology(coords, elems, tag)
    pb = Problem(topo=topo, coords=coords, elems=elems, R=params["R"], T=params["T"], F=params["F"],
                 Cm=params["Cm"], z=np.asarray(params["z"], float), D_i=np.asarray(params["D"], float),
                 D_e=np.asarray(params["D"], float), dt=dt, facet_model=facet_model,
                 facet_gleak=facet_gleak, **kw)
    discretize(pb)
    return pb


@dataclass
class State:
    c_i: np.ndarray    # (n_ions, N_i)
    phi_i: np.ndarray  # (N_i,)
    c_e: np.ndarray    # (n_ions, N_e)
    phi_e: np.ndarray  # (N_e,)
    w: np.ndarray      # (3, n_mv) gates (n, m, h) at membrane vertices
    t: float = 0.0

    def copy(self):
        return State(self.c_i.copy(), self.phi_i.copy(), self.c_e.copy(), self.phi_e.copy(),
                     self.w.copy(), self.t)


def initial_state(pb: Problem, c_i0, c_e0, phi_M0, w0) -> State:
    """[k]_r^0 uniform; phi_i^0 = phi_M^0 at every intracellular node, phi_e^0 = 0 (reading: only
    phi_M^0 is prescribed, Section 2.3); gates w_0 at every membrane vertex."""
    t = pb.topo
    K = pb.n_ions
    c_i = np.tile(np.asarray(c_i0, float)[:, None], (1, t.N_i))
    c_e = np.tile(np.asarray(c_e0, float)[:, None], (1, t.N_e))
    w = np.tile(np.asarray(w0, float)[:, None], (1, pb.geo["n_mv"]))
    return State(c_i, np.full(t.N_i, float(phi_M0)), c_e, np.zeros(t.N_e), w, 0.0)


def offsets(pb: Problem):
    Ni, Ne, K = pb.topo.N_i, pb.topo.N_e, pb.n_ions
    off_i = [k * Ni for k in range(K + 1)]
    off_e = [(K + 1) * Ni + k * Ne for k in range(K + 1)]
    return off_i, off_e, (K + 1) * (Ni + Ne)


def pack(pb: Problem, s: State) -> np.ndarray:
    return np.concatenate([s.c_i.ravel(), s.phi_i, s.c_e.ravel(), s.phi_e])


def unpack(pb: Problem, u: np.ndarray, like: State) -> State:
    Ni, Ne, K = pb.topo.N_i, pb.topo.N_e, pb.n_ions
    c_i = u[:K * Ni].reshape(K, Ni)
    phi_i = u[K * Ni:(K + 1) * Ni]
    o = (K + 1) * Ni
    c_e = u[o:o + K * Ne].reshape(K, Ne)
    phi_e = u[o + K * Ne:o + (K + 1) * Ne]
    return State(c_i.copy(), phi_i.copy(), c_e.copy(), phi_e.copy(), like.w.copy(), like.t)


def membrane_fields(pb: Problem, s: State):
    """phi_M^{n-1}, E_k, alpha_r^k, C_r^k at the membrane vertices and the new gates w_n."""
    g = pb.geo
    z = pb.z
    phi_M = s.phi_i[g["mv_i"]] - s.phi_e[g["mv_e"]]
    ci = s.c_i[:, g["mv_i"]]
    ce = s.c_e[:, g["mv_e"]]
    E = membrane.reversal_potential(pb.R, pb.T, pb.F, z[:, None], ci, ce)
    a_i = membrane.alpha_split(pb.D_i, z, ci)
    a_e = membrane.alpha_split(pb.D_e, z, ce)
    C_i = a_i * pb.Cm / (pb.F * z[:, None])
    C_e = a_e * pb.Cm / (pb.F * z[:, None])
    w_new = membrane.rush_larsen(s.w, phi_M, pb.phi_rest, pb.dt, pb.n_ode)
    return dict(phi_M=phi_M, E=E, a_i=a_i, a_e=a_e, C_i=C_i, C_e=C_e, w=w_new, c_i=ci, c_e=ce)


def channel_currents(pb: Problem, mf: dict, t_prev: float) -> np.ndarray:
    """I_ch^k at the vertices of each facet, shape (n_ions, n_f, m+1) (Eq. 2.15 and the leak model).

    Facet conductances are piecewise constant; the nodal driving terms are P1.
    """
    g = pb.geo
    fv = g["fv"]
    phi_M, E, w = mf["phi_M"], mf["E"], mf["w"]
    n_g, m_g, h_g = w
    drive = phi_M[None, :] - E                             # (K, n_mv)
    gstim = membrane.stimulus_conductance(pb.stim_kind, pb.stim_gbar, t_prev, pb.stim_t0,
                                          pb.stim_t1, pb.stim_a, pb.stim_tau)
    hh = (pb.facet_model == HH).astype(float)
    kir = pb.facet_model == KIR
    I = np.empty((pb.n_ions,) + fv.shape)
    for k in range(pb.n_ions):
        I[k] = pb.facet_gleak[:, k][:, None] * drive[k][fv]
    # ion 0 = Na, 1 = K (Table 2 order)
    I[0] += (gstim * pb.stim_mask)[:, None] * drive[0][fv]
    I[0] += (hh * pb.gbar_Na)[:, None] * (m_g ** 3 * h_g * drive[0])[fv]
    I[1] += (hh * pb.gbar_K)[:, None] * (n_g ** 4 * drive[1])[fv]
    if kir.any():
        # Kir-Na/K: K leak g_leak^K (phi_M - E_K) f_Kir, pump 3 F z_Na j and -2 F z_K j
        f_kir = membrane.kir_factor(mf["c_e"][1], drive[1], phi_M, pb.E_K0, pb.cKe0)
        j = membrane.pump_flux(mf["c_i"][0], mf["c_e"][1], pb.rho_pump, pb.P_Na, pb.P_K)
        I[1][kir] = pb.facet_gleak[kir, 1][:, None] * (drive[1] * f_kir)[fv[kir]]
        I[0][kir] += 3.0 * pb.F * pb.z[0] * j[fv[kir]]
        I[1][kir] -= 2.0 * pb.F * pb.z[1] * j[fv[kir]]
    return I


def assemble(pb: Problem, s: State, source=None):
    """A_{n-1} (csr) and f_n for the step from s = (u_{n-1}, w_{n-1}, t_{n-1}); also returns w_n."""
    t = pb.topo
    g = pb.geo
    K = pb.n_ions
    Ni, Ne = t.N_i, t.N_e
    dt, z, psi = pb.dt, pb.z, pb.psi
    mf = membrane_fields(pb, s)
    I = channel_currents(pb, mf, s.t)
    fv, area = g["fv"], g["area"]
    if source is None and (pb.source_i is not None or pb.source_e is not None):
        # the problem's own bulk source, evaluated at t_n = t_{n-1} + dt
        if pb.source_t0 < s.t + dt <= pb.source_t1:
            source = {"i": pb.source_i if pb.source_i is not None else np.zeros((K, Ni)),
                      "e": pb.source_e if pb.source_e is not None else np.zeros((K, Ne))}
    blocks = [[None] * (2 * (K + 1)) for _ in range(2 * (K + 1))]
    rhs = []
    regions = (("i", "e", +1.0, s.c_i, pb.D_i, mf["a_i"], mf["C_i"], g["fi"], g["fe"], Ni, Ne, 0),
               ("e", "i", -1.0, s.c_e, pb.D_e, mf["a_e"], mf["C_e"], g["fe"], g["fi"], Ne, Ni, K + 1))
    for (r, q, sgn, c_r, D_r, a_r, C_r, fr, fq, Nr, Nq, o) in regions:
        oq = (K + 1) - o
        M, A = g["M_" + r], g["A_" + r]
        tau = dt * D_r
        taut = tau * z / psi
        Ak = [pb.fe.weighted_stiffness(g["cache_" + r], c_r[k], g["en_" + r], Nr) for k in range(K)]
        phi_blk = (pb.Cm / pb.F) * g["MG_" + r]
        phi_q = -(pb.Cm / pb.F) * g["MG_" + r + q]
        f_phi = np.zeros(Nr)
        I_tot = I.sum(axis=0)
        for k in range(K):
            CM_r = pb.fe.membrane_mass(area, fr, fr, Nr, Nr, coef=C_r[k][fv])
            CM_rq = pb.fe.membrane_mass(area, fr, fq, Nr, Nq, coef=C_r[k][fv])
            blocks[o + k][o + k] = M + tau[k] * A
            blocks[o + k][o + K] = CM_r + taut[k] * Ak[k]
            blocks[o + k][oq + K] = -CM_rq
            blocks[o + K][o + k] = z[k] * tau[k] * A
            phi_blk = phi_blk + z[k] * taut[k] * Ak[k]
            # f_r^k = M c^{k,n-1} + dt M f^{k,n} - int_Gamma g_r^k v,
            # g_r^k = +-_r (dt I_ch^k - alpha_r^k C_m phi_M^{n-1}) / (F z_k)
            ICH = pb.fe.membrane_load(area, fr, I[k], Nr)
            aphi = pb.fe.membrane_mass(area, fr, fv, Nr, g["n_mv"], coef=a_r[k][fv]) @ mf["phi_M"]
            fk = M @ c_r[k] - sgn * (dt * ICH - pb.Cm * aphi) / (pb.F * z[k])
            if source is not None:
                fk = fk + dt * (M @ source[r][k])
            rhs.append(fk)
        blocks[o + K][o + K] = phi_blk
        blocks[o + K][oq + K] = phi_q
        # f_r^phi = - int_Gamma h_r w,  h_r = +-_r (dt I_ch - C_m phi_M^{n-1}) / F
        ICH = pb.fe.membrane_load(area, fr, I_tot, Nr)
        phiM_load = pb.fe.membrane_load(area, fr, mf["phi_M"][fv], Nr)
        rhs.append(-sgn * (dt * ICH - pb.Cm * phiM_load) / pb.F)
    # rhs order: i ions, i phi, e ions, e phi
    f = np.concatenate(rhs)
    Amat = sp.bmat(blocks, format="csr")
    Amat, f = apply_pin(pb, Amat, f)
    return Amat, f, mf


def pin_dof(pb: Problem) -> int:
    _, off_e, _ = offsets(pb)
    return off_e[pb.n_ions] + pb.geo["pin"]


def apply_pin(pb: Problem, A: sp.csr_matrix, f: np.ndarray):
    p = pin_dof(pb)
    n = A.shape[0]
    keep = np.ones(n)
    keep[p] = 0.0
    Dk = sp.diags(keep)
    A = (Dk @ A @ Dk).tocsr()
    A = A + sp.csr_matrix(([1.0], ([p], [p])), shape=(n, n))
    f = f.copy()
    f[p] = 0.0
    return A.tocsr(), f


def preconditioner_P0(pb: Problem, s0: State) -> sp.csr_matrix:
    """P_0 of Eq. 4.4 (block diagonal over the 2(|K|+1) fields), from the initial state."""
    g = pb.geo
    K = pb.n_ions
    z, psi, dt = pb.z, pb.psi, pb.dt
    diag = []
    for r, c_r, D_r, Nr in (("i", s0.c_i, pb.D_i, pb.topo.N_i), ("e", s0.c_e, pb.D_e, pb.topo.N_e)):
        M, A = g["M_" + r], g["A_" + r]
        tau = dt * D_r
        taut = tau * z / psi
        for k in range(K):
            diag.append(M + tau[k] * A)
        blk = (pb.Cm / pb.F) * g["MG_" + r]
        for k in range(K):
            blk = blk + z[k] * taut[k] * pb.fe.weighted_stiffness(g["cache_" + r], c_r[k], g["en_" + r], Nr)
        diag.append(blk)
    P = sp.block_diag(diag, format="csr")
    P, _ = apply_pin(pb, P, np.zeros(P.shape[0]))
    return P
