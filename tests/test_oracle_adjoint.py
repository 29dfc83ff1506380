"""Pins for oracle/adjoint.py: the torch residual form reproduces lambda^T (f - A u) of
oracle.system, and the reverse-sweep gradients match 4th-order central differences of the
forward oracle (leak workload and HH workload with its gate chain), with a Taylor test.

The loss is built from phi_e, which is about 1e-8 of phi_i at these scales; the forward
solves resolve it to roughly 1e-7 relative, which bounds the accuracy of the difference
quotients near 3e-6. The tolerance below is 1e-5; a missing or mis-signed term of the
adjoint changes the directional derivatives by far more.
"""
import warnings

import numpy as np
import pytest

from oracle import adjoint, problem, step, system
from synth import make_config
from synth.configs import probe_points

warnings.filterwarnings("ignore", category=UserWarning)


@pytest.mark.parametrize("cfg", [make_config(4).with_nx(32), make_config(2).with_nx(8), make_config(1)])
def test_torch_form_equals_assembly(cfg):
    rng = np.random.default_rng(0)
    pb, s0 = problem.from_config(cfg)
    s0.w = s0.w + 0.05 * rng.standard_normal(s0.w.shape)
    A, f, _ = system.assemble(pb, s0)
    s1, _ = step.step(pb, s0)
    u1 = system.pack(pb, s1) * (1 + 1e-3 * rng.standard_normal(A.shape[0]))
    u1[system.pin_dof(pb)] = 0
    lam = rng.standard_normal(A.shape[0])
    lam[system.pin_dof(pb)] = 0
    F = adjoint.TorchForm(pb)
    Phi, _, _, _ = adjoint.phi_and_grads(F, s0, u1, lam, pb.facet_gleak, np.zeros_like(s0.w))
    ref = lam @ (f - A @ u1)
    assert abs(Phi - ref) <= 1e-10 * abs(ref)


def _richardson(Lfun, eps):
    d1 = Lfun(eps) - Lfun(-eps)
    d2 = Lfun(eps / 2) - Lfun(-eps / 2)
    return (8 * d2 - d1) / (6 * eps)


@pytest.mark.parametrize("case", ["leak", "hh"])
def test_gradients_match_finite_differences(case):
    cfg, n_steps = (make_config(4).with_nx(32), 4) if case == "leak" else (make_config(2).with_nx(8), 3)
    pb, s0 = problem.from_config(cfg)
    P = adjoint.probe_matrix(pb, probe_points(cfg))
    res = adjoint.run_with_adjoint(pb, s0, n_steps, P)
    rng = np.random.default_rng(3)
    g0 = pb.facet_gleak.copy()
    Ni = pb.topo.N_i
    for _ in range(2):
        dg = np.zeros_like(g0)
        dg[:, 1] = rng.standard_normal(len(g0)) * 0.8
        def Lg(e):
            pb.facet_gleak = g0 + e * dg
            return adjoint.loss_only(pb, s0, n_steps, P)
        fd = _richardson(Lg, 0.2)
        an = np.sum(res["grad_gleak"] * dg)
        assert abs(fd - an) <= 1e-5 * abs(an)
        # Taylor test: the first-order remainder decays as eps^2
        L0 = Lg(0.0)
        rem = [abs(Lg(e) - L0 - e * an) for e in (0.08, 0.04, 0.02)]
        pb.facet_gleak = g0
        assert rem[0] / rem[1] > 3.2 and rem[1] / rem[2] > 3.2, rem
        dc = rng.standard_normal(Ni) * 125.0
        def Lc(e):
            s = s0.copy()
            s.c_i[1] = s.c_i[1] + e * dc
            return adjoint.loss_only(pb, s, n_steps, P)
        fd = _richardson(Lc, 0.01)
        an = res["dLdu0"][Ni:2 * Ni] @ dc
        assert abs(fd - an) <= 1e-5 * abs(an)
    if case == "hh":
        dw = rng.standard_normal(s0.w.shape) * 0.1
        def Lw(e):
            s = s0.copy()
            s.w = s.w + e * dw
            return adjoint.loss_only(pb, s, n_steps, P)
        fd = _richardson(Lw, 0.05)
        an = np.sum(res["dLdw0"] * dw)
        assert abs(fd - an) <= 1e-5 * abs(an)


def test_phi_e_is_fixed_loosely_in_fp64():
    """Why the phi_e-based gradients carry a 1e-5 bar: on the 16-cell workload's 32^2 version,
    perturbing every stored entry of A_0 at the rounding level (1 + 1e-16 xi) moves the exact
    solution's phi_e by far more than 1e-16 (about 2.5e-7 of itself), while the concentrations
    move at the rounding level. Two FP64 assemblies that round differently disagree on phi_e at
    that level whatever their solvers do."""
    from oracle import solve as osolve
    pb, s0 = problem.from_config(make_config(4).with_nx(32))
    A, f, _ = system.assemble(pb, s0)
    off_i, off_e, N = system.offsets(pb)
    u = osolve.direct(A, f, refine=4)
    A2 = A.copy().tocsr()
    A2.data = A2.data * (1 + 1e-16 * np.random.default_rng(0).standard_normal(A2.nnz))
    u2 = osolve.direct(A2, f, refine=4)
    phe = slice(off_e[3], N)
    conc = np.r_[0:off_i[3], off_e[0]:off_e[3]]
    d_phe = np.linalg.norm(u2[phe] - u[phe]) / np.linalg.norm(u[phe])
    d_c = np.linalg.norm(u2[conc] - u[conc]) / np.linalg.norm(u[conc])
    assert 1e-8 < d_phe < 1e-5, d_phe
    assert d_c < 1e-14, d_c
