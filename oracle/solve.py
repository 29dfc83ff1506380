"""Linear solves for the oracle (Section 6.2).

* ``direct``  - the exact solution of A_{n-1} u_n = f_n by a sparse LU (SuperLU via scipy) with
  iterative refinement.
* ``gmres``   - textbook restarted GMRES(m): modified Gram-Schmidt Arnoldi, Givens
  rotations, left preconditioning, initial guess x0 and the preconditioned relative
  residual test ||M^{-1} r|| <= rtol ||M^{-1} b|| (the solver settings of Section 6.2).
* ``lu_P0``   - the exact preconditioner LU(P_0) of Section 6.3 (``block_lu_P0``: the same
  operator factored per field block, for the larger 3D meshes).
Pinned by tests/test_oracle_solve.py (dense solves on random systems, restart logic)
and by the Section 6.3 iteration counts in tests/test_oracle_system.py.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def direct(A: sp.spmatrix, b: np.ndarray, refine: int = 2) -> np.ndarray:
    """Sparse LU solve with ``refine`` steps of iterative refinement (the extracellular potential is
    some 1e-8 of the intracellular one, so one LU pass leaves it with relative errors near 1e-7)."""
    lu = spla.splu(A.tocsc())
    x = lu.solve(b)
    for _ in range(refine):
        x = x + lu.solve(b - A @ x)
    return x


def lu_P0(P: sp.spmatrix):
    lu = spla.splu(P.tocsc())
    return lu.solve


def block_lu_P0(P: sp.spmatrix, bounds):
    """The same exact P_0^{-1} as lu_P0, factored block by block: P_0 is block diagonal over its
    2(|K|+1) field blocks (Eq. 4.4), given by their row ranges [bounds[i], bounds[i+1]); each
    block is symmetric and factored with a symmetric minimum-degree ordering, which keeps the
    fill of the 3D blocks far below that of one factorisation of the whole matrix."""
    P = P.tocsr()
    lus = []
    for a, b in zip(bounds[:-1], bounds[1:]):
        lus.append((a, b, spla.splu(P[a:b, a:b].tocsc(), permc_spec="MMD_AT_PLUS_A",
                                    options=dict(SymmetricMode=True)) if b > a else None))

    def apply(v):
        out = np.empty_like(v)
        for a, b, lu in lus:
            if lu is not None:
                out[a:b] = lu.solve(v[a:b])
        return out
    return apply


def gmres(A, b, x0=None, M=None, rtol=1e-6, restart=30, maxit=1000):
    """Left-preconditioned restarted GMRES. Returns (x, iterations, converged, history)."""
    n = b.shape[0]
    Mi = (lambda v: v) if M is None else M
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    bnorm = np.linalg.norm(Mi(b))
    if bnorm == 0.0:
        return np.zeros(n), 0, True, [0.0]
    its = 0
    hist = []
    while its < maxit:
        r = Mi(b - A @ x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta <= rtol * bnorm:
            return x, its, True, hist
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(restart):
            w = Mi(A @ V[j])
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                tmp = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = tmp
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= rtol * bnorm or its >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + V[:j_done].T @ y
        if abs(g[j_done]) <= rtol * bnorm:
            return x, its, True, hist
    r = Mi(b - A @ x)
    return x, its, np.linalg.norm(r) <= rtol * bnorm, hist
