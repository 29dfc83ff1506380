"""Pins for oracle/solve.py: GMRES against a dense solve, across restarts, with and
without a preconditioner; the direct solve on a random sparse system."""
import numpy as np
import scipy.sparse as sp

from oracle import solve


def _system(n, seed):
    rng = np.random.default_rng(seed)
    A = sp.random(n, n, density=0.05, random_state=seed) + sp.eye(n) * 4.0
    b = rng.standard_normal(n)
    return A.tocsr(), b


def test_gmres_matches_dense_solve_across_restarts():
    A, b = _system(200, 1)
    x_ref = np.linalg.solve(A.toarray(), b)
    for restart in (5, 30):
        x, its, ok, hist = solve.gmres(A, b, rtol=1e-12, restart=restart, maxit=500)
        assert ok and np.linalg.norm(x - x_ref) < 1e-9 * np.linalg.norm(x_ref)
        assert np.all(np.diff(hist[: restart]) <= 1e-15)      # GMRES residuals do not increase


def test_gmres_left_preconditioned_exact_preconditioner_one_iteration():
    A, b = _system(100, 3)
    lu = solve.lu_P0(A)
    x, its, ok, _ = solve.gmres(A, b, M=lu, rtol=1e-10)
    assert ok and its == 1


def test_gmres_initial_guess_already_converged():
    A, b = _system(50, 4)
    x_ref = solve.direct(A, b)
    x, its, ok, _ = solve.gmres(A, b, x0=x_ref, rtol=1e-8)
    assert ok and its == 0


def test_direct():
    A, b = _system(300, 5)
    x = solve.direct(A, b)
    assert np.linalg.norm(A @ x - b) < 1e-12 * np.linalg.norm(b)


def test_block_lu_P0_equals_dense_solve_of_the_block_diagonal_matrix():
    """block_lu_P0 is P_0^{-1} for a block-diagonal matrix: on P_0 of a small 3D HH workload (eight
    field blocks, the pin included) it equals a dense solve, and lu_P0."""
    from oracle import problem, system
    from synth import make_config
    pb, s0 = problem.from_config(make_config(2).with_nx(4))
    P = system.preconditioner_P0(pb, s0)
    off_i, off_e, N = system.offsets(pb)
    v = np.random.default_rng(6).standard_normal(N)
    x_ref = np.linalg.solve(P.toarray(), v)
    x = solve.block_lu_P0(P, off_i + off_e + [N])(v)
    assert np.linalg.norm(x - x_ref) <= 1e-12 * np.linalg.norm(x_ref)
    assert np.linalg.norm(solve.lu_P0(P)(v) - x_ref) <= 1e-12 * np.linalg.norm(x_ref)
