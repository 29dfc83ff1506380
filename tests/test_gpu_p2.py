"""GPU parity of the P2 path (Section 3.3 with p = 2) through the C ABI against the P2 oracle.

The P2 kernels (element pair values of A_r^{k}, P2 membrane pairs and right-hand side) are
compared with the P2 oracle's assembly entry by entry, and whole time steps with its states.
Their host side is also checked on the CPU: the P2 node tables, the static M_r and A_r, and the
per-step element arithmetic of A_r^{k} (tests/test_library_cpu.py). Same bars as the P1 parity
tests.
"""
import numpy as np
import pytest

from helpers import blockscaled_entry_error, blockwise_vector_error, oracle_run, rel_errors
from oracle import problem as oproblem, system as osystem
from synth import make_config
from synth.configs import model_a

pytestmark = pytest.mark.gpu

TOL = 1e-8


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _cfgs():
    return {
        "2d-leak-16": make_config(1).with_nx(16),
        "3d-hh-8": make_config(2).with_nx(8),
        "2d-16cells-32": make_config(4).with_nx(32),
        "kir-2d-16": make_config(7).with_nx(16),
        "modelA-3d-4": model_a(3, 4, 1e-4),
    }


@pytest.mark.parametrize("name", list(_cfgs()))
def test_p2_assembly_and_operator(name):
    from paper_2403_04491_gb300 import problem_from_config
    cfg = _cfgs()[name]
    pb, s0 = oproblem.from_config(cfg, degree=2)
    A, f, _ = osystem.assemble(pb, s0)
    _, prob = problem_from_config(cfg, degree=2)
    assert prob.n_dof == A.shape[0]
    prob.assemble_step()
    Acoo = A.tocoo()
    vals = prob.operator_entries(Acoo.row, Acoo.col)
    assert blockscaled_entry_error(pb, A, vals) < 1e-12
    assert blockwise_vector_error(pb, prob.rhs_get(), f) < 1e-12
    x = np.random.default_rng(3).standard_normal(A.shape[0])
    assert blockwise_vector_error(pb, prob.apply_operator(x), A @ x) < 1e-12


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64-amg", "fp32-amg"])
@pytest.mark.parametrize("name,n_steps,exact", [("2d-leak-16", 5, "direct"), ("3d-hh-8", 4, "lu_p0"),
                                                ("kir-2d-16", 5, "direct")])
def test_p2_time_steps_match_oracle(name, n_steps, exact, precision):
    from paper_2403_04491_gb300 import problem_from_config
    cfg = _cfgs()[name]
    pb, ref = oracle_run(cfg, n_steps, exact, degree=2)
    _, prob = problem_from_config(cfg, degree=2)
    prob.amg_setup(precision=precision)
    for n in range(1, n_steps + 1):
        st = prob.step(1, rtol=1e-10)
        s = prob.state_get()
        ec, ep = rel_errors(s, ref[n])
        assert ec <= TOL and ep <= TOL, (n, ec, ep, st)
        np.testing.assert_allclose(s["w"], ref[n].w, rtol=1e-12 if n == 1 else TOL, atol=1e-14)


def test_p2_adjoint_is_refused():
    from paper_2403_04491_gb300 import problem_from_config
    from paper_2403_04491_gb300.knp import KnpError
    _, prob = problem_from_config(make_config(1).with_nx(8), degree=2)
    with pytest.raises(KnpError):
        prob.adjoint_begin()


@pytest.mark.slow
def test_p2_bench_workload_full_size():
    """The P2 bench workload at its full size (3D HH, 32^3 mesh with P2 elements: the node
    lattice of the 64^3 P1 workload) in the bench's launch configuration: the operator at 20,000
    sampled entries, the right-hand side and an operator product against the oracle's assembly;
    then five steps whose true residuals stay at the solver tolerance and which conserve the
    charge of the cell and of the extracellular space."""
    import scipy.sparse as sp
    from paper_2403_04491_gb300 import problem_from_config
    cfg = make_config(2).with_nx(32)
    pb, s0 = oproblem.from_config(cfg, degree=2)
    A, f, _ = osystem.assemble(pb, s0)
    _, prob = problem_from_config(cfg, degree=2)
    assert prob.n_dof == A.shape[0]
    prob.assemble_step()
    Acoo = A.tocoo()
    pick = np.random.default_rng(7).choice(Acoo.nnz, 20000, replace=False)
    As = sp.coo_matrix((Acoo.data[pick], (Acoo.row[pick], Acoo.col[pick])), shape=A.shape)
    assert blockscaled_entry_error(pb, As, prob.operator_entries(As.row, As.col)) < 1e-12
    assert blockwise_vector_error(pb, prob.rhs_get(), f) < 1e-12
    x = np.random.default_rng(8).standard_normal(A.shape[0])
    assert blockwise_vector_error(pb, prob.apply_operator(x), A @ x) < 1e-12
    g, z = pb.geo, pb.z

    def charges(st):
        qi = sum(z[k] * (g["M_i"] @ st["c_i"][k]) for k in range(3))
        return np.bincount(pb.topo.node_cell_i, weights=qi), sum(z[k] * (g["M_e"] @ st["c_e"][k]).sum() for k in range(3))

    scale = sum((g["M_e"] @ s0.c_e[k]).sum() for k in range(3))
    q0 = charges(prob.state_get())
    prob.amg_setup()
    for _ in range(5):
        prob.assemble_step()
        st = prob.solve(rtol=1e-10)
        assert st["true_relres"] < 1e-9, st
    q1 = charges(prob.state_get())
    assert np.abs(q1[0] - q0[0]).max() < 1e-9 * scale and abs(q1[1] - q0[1]) < 1e-9 * scale
