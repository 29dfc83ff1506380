"""Adjoint of the time loop (spec addition; the paper has no adjoint).

For step n the discrete equations are R_n = A_{n-1} u_n - f_n = 0 with A_{n-1} and f_n
built from (u_{n-1}, w_n, theta) and w_n = G(w_{n-1}, phi_M(u_{n-1})) (Section 3.2). For a
loss L(u_1..u_N) the Lagrangian gives, backwards in n,

    A_{n-1}^T lambda_n = dL/du_n + d/du_n [ Phi_{n+1} + gamma_{n+1}^T w_{n+1} ],
    Phi_n = lambda_n^T (f_n - A_{n-1} u_n)  (u_n, lambda_n held fixed),
    gamma_n = d/dw_n [ Phi_{n+1} + gamma_{n+1}^T w_{n+1} ],
    dL/dtheta = sum_n d Phi_n / d theta,   dL/du_0 = d/du_0 [ Phi_1 + gamma_1^T w_1 ].

The explicit partials of Phi_n are taken by PyTorch autograd on ``step_residual_form``,
a restatement of oracle.system's assembly in torch (CPU, float64) as a scalar function of
(u_{n-1}, w_{n-1}, the per-facet leak conductances). The transposed solves are sparse LU.
TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). Pinned by tests/test_oracle_adjoint.py:
the torch form reproduces lambda^T (f - A u) of oracle.system to rounding, and the gradients
match central finite differences of the forward oracle.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import torch

from . import fem, membrane, solve, step as ostep, system

LEAK, HH = 0, 1


def _sparse_t(A: sp.spmatrix) -> torch.Tensor:
    A = A.tocoo()
    idx = torch.tensor(np.vstack([A.row, A.col]), dtype=torch.long)
    return torch.sparse_coo_tensor(idx, torch.tensor(A.data), A.shape).coalesce()


class TorchForm:
    """Static pieces of the discretisation as torch tensors."""

    def __init__(self, pb: system.Problem):
        if pb.fe is not fem:
            raise ValueError("the adjoint residual form covers P1 elements only")
        g = pb.geo
        t = pb.topo
        self.pb = pb
        self.M = {r: _sparse_t(g["M_" + r]) for r in ("i", "e")}
        self.A = {r: _sparse_t(g["A_" + r]) for r in ("i", "e")}
        rows, cols, Ae = g["cache_i"]
        self.elem = {}
        for r in ("i", "e"):
            rows, cols, Ae = g["cache_" + r]
            self.elem[r] = dict(nodes=torch.tensor(g["en_" + r], dtype=torch.long),
                                Ae=torch.tensor(Ae))
        self.fv = torch.tensor(g["fv"], dtype=torch.long)
        self.fi = torch.tensor(g["fi"], dtype=torch.long)
        self.fe = torch.tensor(g["fe"], dtype=torch.long)
        self.area = torch.tensor(g["area"])
        m = t.dim - 1
        self.Mloc = torch.tensor(fem.local_mass(m))
        self.W = torch.tensor(fem.local_triple(m))
        self.mv_i = torch.tensor(g["mv_i"], dtype=torch.long)
        self.mv_e = torch.tensor(g["mv_e"], dtype=torch.long)
        self.pin = g["pin"]
        self.hh = torch.tensor((pb.facet_model == HH).astype(float))
        self.mask = torch.tensor(pb.stim_mask.astype(float))


def _vtrap(x):
    small = x.abs() < 1e-6
    xs = torch.where(small, torch.ones_like(x), x)
    return torch.where(small, 1.0 - x / 2.0 + x * x / 12.0, xs / torch.expm1(xs))


def _rush_larsen(pb, w, phi_M):
    V = 1e3 * (phi_M - pb.phi_rest)
    a = torch.stack([0.1 * _vtrap((10.0 - V) / 10.0), _vtrap((25.0 - V) / 10.0), 0.07 * torch.exp(-V / 20.0)])
    b = torch.stack([0.125 * torch.exp(-V / 80.0), 4.0 * torch.exp(-V / 18.0), 1.0 / (torch.exp((30.0 - V) / 10.0) + 1.0)])
    winf = a / (a + b)
    dec = torch.exp(-(a + b) * (1e3 * pb.dt / pb.n_ode))
    for _ in range(pb.n_ode):
        w = winf + (w - winf) * dec
    return w


def _facet_load(F: TorchForm, rows, vals_fa, n):
    """int_Gamma (facet-wise P1 function with vertex values vals_fa) phi_j, scattered to rows."""
    loc = F.area[:, None] * (vals_fa @ F.Mloc)
    out = torch.zeros(n, dtype=torch.float64)
    return out.index_add(0, rows.reshape(-1), loc.reshape(-1))


def _triple_load(F: TorchForm, rows, coef_fa, fun_fa, n):
    """int_Gamma (P1 coef)(P1 fun) phi_j, scattered to rows."""
    loc = F.area[:, None] * torch.einsum("fa,fb,abj->fj", coef_fa, fun_fa, F.W)
    out = torch.zeros(n, dtype=torch.float64)
    return out.index_add(0, rows.reshape(-1), loc.reshape(-1))


def _weighted_stiffness_apply(F: TorchForm, r, c_nodes, phi, n):
    """A_r^{k}(c) phi for P1 c: element mean of c times the element stiffness applied to phi."""
    e = F.elem[r]
    cbar = c_nodes[e["nodes"]].mean(dim=1)
    loc = cbar[:, None] * torch.einsum("tjl,tl->tj", e["Ae"], phi[e["nodes"]])
    out = torch.zeros(n, dtype=torch.float64)
    return out.index_add(0, e["nodes"].reshape(-1), loc.reshape(-1))


def step_residual_form(F: TorchForm, old: dict, w_old, gleak, new: dict, lam: dict, t_prev: float):
    """Phi = lambda^T (f_n - A_{n-1} u_n) and w_n, as torch functions of the old state, the old gates
    and the per-facet leak conductances (the same arithmetic as oracle.system.assemble)."""
    pb = F.pb
    K = pb.n_ions
    z = torch.tensor(pb.z)
    psi = pb.psi
    dt = pb.dt
    phi_M = old["phi_i"][F.mv_i] - old["phi_e"][F.mv_e]
    ci = old["c_i"][:, F.mv_i]
    ce = old["c_e"][:, F.mv_e]
    E = (pb.R * pb.T / (pb.F * z[:, None])) * torch.log(ce / ci)
    Di = torch.tensor(pb.D_i)[:, None]
    De = torch.tensor(pb.D_e)[:, None]
    wi = Di * z[:, None] ** 2 * ci
    we = De * z[:, None] ** 2 * ce
    C = {"i": wi / wi.sum(0, keepdim=True) * pb.Cm / (pb.F * z[:, None]),
         "e": we / we.sum(0, keepdim=True) * pb.Cm / (pb.F * z[:, None])}
    w_new = _rush_larsen(pb, w_old, phi_M)
    n_g, m_g, h_g = w_new
    drive = phi_M[None, :] - E
    gstim = membrane.stimulus_conductance(pb.stim_kind, pb.stim_gbar, t_prev, pb.stim_t0, pb.stim_t1, pb.stim_a,
                                          pb.stim_tau)
    fv = F.fv
    I = [gleak[:, k][:, None] * drive[k][fv] for k in range(K)]
    I[0] = I[0] + (gstim * F.mask)[:, None] * drive[0][fv] + (F.hh * pb.gbar_Na)[:, None] * (m_g ** 3 * h_g * drive[0])[fv]
    I[1] = I[1] + (F.hh * pb.gbar_K)[:, None] * ((n_g ** 2) * (n_g ** 2) * drive[1])[fv]
    Itot = sum(I)
    phi_M_new = new["phi_i"][F.mv_i] - new["phi_e"][F.mv_e]
    Phi = torch.zeros((), dtype=torch.float64)
    for r, q, sgn, rows, cols_q, N_r in (("i", "e", 1.0, F.fi, F.fe, pb.topo.N_i), ("e", "i", -1.0, F.fe, F.fi, pb.topo.N_e)):
        tau = dt * torch.tensor(pb.D_i if r == "i" else pb.D_e)
        taut = tau * z / psi
        lam_phi = lam["phi_" + r].clone()
        if r == "e":
            lam_phi = lam_phi.clone()
            lam_phi[F.pin] = 0.0
        phi_new_r = new["phi_" + r]
        # potential row
        Aphi = torch.zeros(N_r, dtype=torch.float64)
        for k in range(K):
            # f^k = M c_old - sgn (dt int I^k v - C_m int alpha phi_M^old v) / (F z_k)
            fk = torch.sparse.mm(F.M[r], old["c_" + r][k][:, None])[:, 0]
            fk = fk - sgn * dt / (pb.F * z[k]) * _facet_load(F, rows, I[k], N_r)
            fk = fk + sgn * _triple_load(F, rows, C[r][k][fv], phi_M[fv], N_r)
            # (A u)^k = (M + tau A) c^k + tau~ A^k phi_r + C^k M_{r,G} phi_r - C^k M_{rq,G} phi_q
            Au = torch.sparse.mm(F.M[r], new["c_" + r][k][:, None])[:, 0] + tau[k] * torch.sparse.mm(
                F.A[r], new["c_" + r][k][:, None])[:, 0]
            Akphi = _weighted_stiffness_apply(F, r, old["c_" + r][k], phi_new_r, N_r)
            Au = Au + taut[k] * Akphi + sgn * _triple_load(F, rows, C[r][k][fv], phi_M_new[fv], N_r)
            Phi = Phi + torch.dot(lam["c_" + r][k], fk - Au)
            Aphi = Aphi + z[k] * tau[k] * torch.sparse.mm(F.A[r], new["c_" + r][k][:, None])[:, 0] + z[k] * taut[k] * Akphi
        Aphi = Aphi + sgn * (pb.Cm / pb.F) * _facet_load(F, rows, phi_M_new[fv], N_r)
        fphi = -sgn * (dt * _facet_load(F, rows, Itot, N_r) - pb.Cm * _facet_load(F, rows, phi_M[fv], N_r)) / pb.F
        Phi = Phi + torch.dot(lam_phi, fphi - Aphi)
    return Phi, w_new


def _split(pb, u):
    Ni, Ne, K = pb.topo.N_i, pb.topo.N_e, pb.n_ions
    o = (K + 1) * Ni
    return dict(c_i=u[:K * Ni].reshape(K, Ni), phi_i=u[K * Ni:o], c_e=u[o:o + K * Ne].reshape(K, Ne),
                phi_e=u[o + K * Ne:])


def _as_torch(d, grad=False):
    return {k: torch.tensor(np.asarray(v, dtype=np.float64), requires_grad=grad) for k, v in d.items()}


def phi_and_grads(F: TorchForm, s_old: system.State, u_new: np.ndarray, lam: np.ndarray, gleak: np.ndarray,
                  gamma_next: np.ndarray):
    """Gradients of Phi_n + gamma_{n}^T w_n w.r.t. (u_{n-1}, w_{n-1}, g_leak) for step n from s_old."""
    pb = F.pb
    old = _as_torch(dict(c_i=s_old.c_i, phi_i=s_old.phi_i, c_e=s_old.c_e, phi_e=s_old.phi_e), grad=True)
    w_old = torch.tensor(s_old.w, requires_grad=True)
    gl = torch.tensor(gleak, requires_grad=True)
    new = _as_torch(_split(pb, u_new))
    lm = _as_torch(_split(pb, lam))
    Phi, w_new = step_residual_form(F, old, w_old, gl, new, lm, s_old.t)
    obj = Phi + torch.sum(torch.tensor(gamma_next) * w_new)
    obj.backward()
    gu = np.concatenate([old["c_i"].grad.numpy().ravel(), old["phi_i"].grad.numpy(), old["c_e"].grad.numpy().ravel(),
                         old["phi_e"].grad.numpy()])
    return float(Phi.detach()), gu, w_old.grad.numpy(), gl.grad.numpy()


def probe_matrix(pb: system.Problem, points: np.ndarray) -> sp.csr_matrix:
    """P1 interpolation of phi_e at points in Omega_e: rows = points, columns = unknowns (Eq. 4.3 order)."""
    t = pb.topo
    coords, elems = pb.coords, pb.elems
    E = elems[t.elems_e]
    x = coords[E]
    d = t.dim
    rows, cols, vals = [], [], []
    _, off_e, N = system.offsets(pb)
    for p, pt in enumerate(points):
        # barycentric coordinates in every extracellular element; pick the containing one
        J = (x[:, 1:, :] - x[:, :1, :]).transpose(0, 2, 1)
        lam = np.linalg.solve(J, (pt - x[:, 0, :])[:, :, None])[:, :, 0]
        bary = np.concatenate([1 - lam.sum(1, keepdims=True), lam], axis=1)
        inside = np.all(bary >= -1e-12, axis=1)
        k = np.flatnonzero(inside)[0]
        for j in range(d + 1):
            rows.append(p)
            cols.append(off_e[pb.n_ions] + t.loc_e[E[k, j]])
            vals.append(bary[k, j])
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(points), N))


def run_with_adjoint(pb: system.Problem, s0: system.State, n_steps: int, Pmat: sp.csr_matrix):
    """Forward (exact solves) and reverse sweep for L = sum_n sum_p (P u_n)_p^2.

    Returns dict(L, states, grad_gleak (n_f, K), dLdu0 (Eq. 4.3 order), dLdw0)."""
    F = TorchForm(pb)
    states, mats = [s0], []
    s = s0
    for _ in range(n_steps):
        A, f, mf = system.assemble(pb, s)
        mats.append(A)
        s, _ = ostep.step(pb, s)
        states.append(s)
    L = sum(float(np.sum((Pmat @ system.pack(pb, st)) ** 2)) for st in states[1:])
    rho = np.zeros(Pmat.shape[1])
    gamma = np.zeros_like(s0.w)
    grad_g = np.zeros_like(pb.facet_gleak)
    lams, rhos, grads = {}, {}, {}
    for n in range(n_steps, 0, -1):
        u_n = system.pack(pb, states[n])
        a_n = 2.0 * (Pmat.T @ (Pmat @ u_n))
        lam = solve.direct(mats[n - 1].T, a_n + rho)
        _, gu, gw, gg = phi_and_grads(F, states[n - 1], u_n, lam, pb.facet_gleak, gamma)
        rho, gamma = gu, gw
        grad_g += gg
        lams[n], rhos[n - 1], grads[n] = lam, gu, gg
    return dict(L=L, states=states, grad_gleak=grad_g, dLdu0=rho, dLdw0=gamma, lams=lams, rhos=rhos, grads=grads)


def loss_only(pb: system.Problem, s0: system.State, n_steps: int, Pmat: sp.csr_matrix) -> float:
    s = s0
    L = 0.0
    for _ in range(n_steps):
        s, _ = ostep.step(pb, s)
        L += float(np.sum((Pmat @ system.pack(pb, s)) ** 2))
    return L
