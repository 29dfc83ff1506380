"""GPU adjoint against the oracle's adjoint (autograd of its torch residual form, exact LU
solves): the transposed operator, and the gradients of L = sum_n sum_p phi_e(x_p, t_n)^2 with
respect to the per-facet K leak conductance, u_0 and the HH gates w_0; the torch.autograd.Function
with checkpointing; and finite differences of the GPU forward loss on the full differentiation
workload.

Given the oracle's forward states, the GPU reverse sweep matches to relative l2 1e-6. From the
GPU's own forward run the bar is 1e-5. The loss is built from phi_e, about 1e-6 of phi_i on the
16-cell workload, and FP64 fixes phi_e only loosely: perturbing the oracle's assembled entries by
1e-16 moves its phi_e by 2.5e-7, and the GPU's phi_e differs from the oracle's by up to 2.8e-6 at
any solver tolerance, phi_e floor or preconditioner, i.e. by the rounding of the two assemblies.
"""
import numpy as np
import pytest

from helpers import blockwise_vector_error
from oracle import adjoint as oadj, problem as oproblem, system as osystem
from synth import make_config
from synth.configs import probe_points

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


CASES = {"cfg4-16cells-32": (make_config(4).with_nx(32), 4), "cfg2-hh-8": (make_config(2).with_nx(8), 3)}


@pytest.mark.parametrize("name", list(CASES))
def test_transposed_operator(name):
    from paper_2403_04491_gb300 import problem_from_config
    cfg, _ = CASES[name]
    pb, s0 = oproblem.from_config(cfg)
    A, f, _ = osystem.assemble(pb, s0)
    _, prob = problem_from_config(cfg)
    prob.assemble_step()
    x = np.random.default_rng(5).standard_normal(A.shape[0])
    assert blockwise_vector_error(pb, prob.apply_operator_transpose(x), A.T @ x) < 1e-12


def _gpu_sweep(cfg, n_steps, Pmat, oracle_states=None):
    """Reverse sweep on the GPU, from its own forward run (rtol 1e-12, extracellular potentials
    tested as their own group) or from given states."""
    from paper_2403_04491_gb300 import problem_from_config
    _, prob = problem_from_config(cfg)
    prob.amg_setup()
    pack = lambda s: np.concatenate([s["c_i"].ravel(), s["phi_i"], s["c_e"].ravel(), s["phi_e"]])
    if oracle_states is None:
        states = [prob.state_get()]
        for _ in range(n_steps):
            prob.step(1, rtol=1e-12, phi_e_group=True)
            states.append(prob.state_get())
    else:
        states = [dict(c_i=s.c_i, phi_i=s.phi_i, c_e=s.c_e, phi_e=s.phi_e, w=s.w, t=s.t) for s in oracle_states]
    prob.adjoint_begin()
    for n in range(n_steps, 0, -1):
        u_n = pack(states[n])
        dLdu = 2.0 * (Pmat.T @ (Pmat @ u_n))
        s = states[n - 1]
        prob.state_set(s["c_i"], s["phi_i"], s["c_e"], s["phi_e"], s["w"], s["t"])
        prob.adjoint_step(u_n, dLdu, rtol=1e-12)
    return prob.adjoint_get(), prob


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("own_forward", [False, True], ids=["oracle-states", "gpu-forward"])
@pytest.mark.parametrize("name", list(CASES))
def test_gradients_match_oracle_adjoint(name, own_forward):
    cfg, n_steps = CASES[name]
    pb, s0 = oproblem.from_config(cfg)
    Pmat = oadj.probe_matrix(pb, probe_points(cfg))
    ref = oadj.run_with_adjoint(pb, s0, n_steps, Pmat)
    got, prob = _gpu_sweep(cfg, n_steps, Pmat, None if own_forward else ref["states"])
    Ni = pb.topo.N_i
    tol = 1e-5 if own_forward else 1e-6
    assert _rel(got["grad_gleak"], ref["grad_gleak"]) < tol
    assert _rel(got["dLdu0"][Ni:2 * Ni], ref["dLdu0"][Ni:2 * Ni]) < tol      # initial [K]_i
    mask = np.ones(len(ref["dLdu0"]), bool)
    mask[osystem.pin_dof(pb)] = False                                        # the pinned unknown is not a variable
    assert _rel(got["dLdu0"][mask], ref["dLdu0"][mask]) < tol
    if np.linalg.norm(ref["dLdw0"]) > 0:
        assert _rel(got["dLdw0"], ref["dLdw0"]) < tol


def test_autograd_function_with_checkpoints():
    import torch
    from paper_2403_04491_gb300 import KNPFunction, Simulation, problem_from_config, probe_weights
    cfg = make_config(4).with_nx(32)
    n_steps = 5
    mesh, prob = problem_from_config(cfg)
    prob.amg_setup()
    m = cfg.mesh
    ni, ne = mesh.nodes()
    idx, w = probe_weights(m.coords, m.elems, m.elem_tag, ne, prob.N_i, prob.N_e, probe_points(cfg))
    sim = Simulation(prob, idx, w, n_steps, checkpoint_every=2, rtol=1e-12)
    gK = torch.tensor(prob._facet_gleak[:, 1].copy(), requires_grad=True)
    cK = torch.tensor(sim.s0["c_i"][1].copy(), requires_grad=True)
    traces = KNPFunction.apply(gK, cK, sim)
    loss = (traces ** 2).sum()
    loss.backward()
    pb, s0 = oproblem.from_config(cfg)
    Pmat = oadj.probe_matrix(pb, probe_points(cfg))
    ref = oadj.run_with_adjoint(pb, s0, n_steps, Pmat)
    assert abs(float(loss) - ref["L"]) < 1e-6 * ref["L"]
    Ni = pb.topo.N_i
    assert _rel(gK.grad.numpy(), ref["grad_gleak"][:, 1]) < 1e-5
    assert _rel(cK.grad.numpy(), ref["dLdu0"][Ni:2 * Ni]) < 1e-5


def test_adjoint_rejects_kir_facets():
    """The adjoint's partial derivatives cover leak and HH facets; Kir-Na/K facets are refused."""
    from paper_2403_04491_gb300 import problem_from_config
    from paper_2403_04491_gb300.knp import KnpError
    _, prob = problem_from_config(make_config(7))
    prob.amg_setup()
    with pytest.raises(KnpError, match="Kir"):
        prob.adjoint_begin()


@pytest.mark.slow
def test_full_gradient_against_finite_differences():
    """The differentiation workload at its full size (256^2 mesh, 16 cells, per-facet g_K, 200 steps
    of 0.1 ms, checkpoints every 20, loss = sum over steps of phi_e^2 at 64 probes): the
    checkpointed adjoint's directional derivatives match central differences of the GPU forward run
    on 16 Gaussian directions (PCG64 seed 3): 8 in the per-facet g_K, 8 in the initial [K]_i.

    The quotients combine two step sizes to fourth order (Richardson), as the oracle's own
    finite-difference pins do; their accuracy is bounded by how precisely FP64 fixes the loss.
    phi_e is about 1e-6 of phi_i, and perturbing the assembled operator at the rounding level moves
    phi_e by about 2.5e-7 of itself (tests/test_oracle_adjoint.py), so two runs whose inputs
    differ slightly disagree on the loss at that level, whatever the solver tolerance (measured:
    the same at rtol 1e-12 with the phi_e floor at 1e-14 and at rtol 1e-13 with 1e-16): on this
    200-step run the loss carries about 1e-5 relative noise, and the same direction's quotient
    moved between 1e-5 and 8e-5 with the solver settings alone. A 20% perturbation of g_K changes
    the loss by 5-20% along these directions, and the quotients agree to 1e-5 .. 5e-4 (bar 2e-3).
    After 200 steps the loss hardly depends on the initial [K]_i (2.5e-3 of it per 1.25 mM), so
    those quotients agree to 2e-3 .. 1.5e-2 (bar 5e-2). A missing or mis-signed adjoint term moves
    a derivative by order one."""
    import torch
    from paper_2403_04491_gb300 import KNPFunction, Simulation, problem_from_config, probe_weights
    cfg = make_config(4)
    mesh, prob = problem_from_config(cfg)
    prob.amg_setup()
    m = cfg.mesh
    ni, ne = mesh.nodes()
    idx, w = probe_weights(m.coords, m.elems, m.elem_tag, ne, prob.N_i, prob.N_e, probe_points(cfg))
    sim = Simulation(prob, idx, w, cfg.n_steps, checkpoint_every=20, rtol=1e-12)
    g0 = torch.tensor(prob._facet_gleak[:, 1].copy())
    c0 = torch.tensor(sim.s0["c_i"][1].copy())
    gK, cK = g0.clone().requires_grad_(True), c0.clone().requires_grad_(True)
    loss = (KNPFunction.apply(gK, cK, sim) ** 2).sum()
    loss.backward()
    grad_g, grad_c = gK.grad.numpy().copy(), cK.grad.numpy().copy()

    def L(g, c):
        with torch.no_grad():
            return float((KNPFunction.apply(g, c, sim) ** 2).sum())

    rng = np.random.Generator(np.random.PCG64(3))
    for q in range(16):
        if q < 8:
            d, eps, bar = 0.8 * rng.standard_normal(len(g0)), 0.2, 2e-3
            Le = lambda e: L(g0 + e * torch.tensor(d), c0)
            an = float(grad_g @ d)
        else:
            d, eps, bar = 125.0 * rng.standard_normal(len(c0)), 0.02, 5e-2
            Le = lambda e: L(g0, c0 + e * torch.tensor(d))
            an = float(grad_c @ d)
        d1 = Le(eps) - Le(-eps)
        d2 = Le(eps / 2) - Le(-eps / 2)
        fd = (8 * d2 - d1) / (6 * eps)
        print(f"direction {q}: adjoint {an:.10e} finite differences {fd:.10e} rel {abs(fd - an) / abs(an):.2e}")
        assert abs(fd - an) <= bar * abs(an), (q, an, fd)
