"""P1 finite-element matrices of Section 4.1, by exact quadrature.

For a d-simplex T with barycentric coordinates lambda_j:
  * mass      int_T lambda_j lambda_l = |T| (1 + delta_jl) / ((d+1)(d+2))
  * stiffness int_T grad lambda_j . grad lambda_l = |T| grad lambda_j . grad lambda_l
  * weighted  int_T c grad lambda_j . grad lambda_l = cbar_T |T| grad lambda_j . grad lambda_l
    for P1 c (cbar_T = vertex mean; exact because the gradients are constant).
On an m-simplex facet f the barycentric moment formula
  int_f prod_a lambda_a^{k_a} = m! prod_a k_a! |f| / (m + sum_a k_a)!
gives the membrane mass (two factors) and the coefficient-weighted membrane
mass int_f (P1 C) lambda_j lambda_l (three factors).
Pinned by tests/test_oracle_fem.py (brute-force Gauss quadrature on random
simplices, row sums, symmetry, constant reproduction).
"""
from __future__ import annotations

from math import factorial

import numpy as np
import scipy.sparse as sp


def simplex_geometry(coords: np.ndarray, elems: np.ndarray):
    """Volumes |T| and barycentric gradients G[T, j, :] = grad lambda_j."""
    x = coords[elems]                                  # (n, d+1, d)
    J = (x[:, 1:, :] - x[:, :1, :]).transpose(0, 2, 1)  # columns x_j - x_0, (n, d, d)
    d = coords.shape[1]
    det = np.linalg.det(J)
    vol = np.abs(det) / factorial(d)
    Binv = np.linalg.inv(J)                            # rows: grad lambda_1..d
    G = np.empty((elems.shape[0], d + 1, d))
    G[:, 1:, :] = Binv
    G[:, 0, :] = -Binv.sum(axis=1)
    return vol, G


def vertex_volumes(coords: np.ndarray, elems: np.ndarray, n_vertices: int, chunk: int = 4_000_000) -> np.ndarray:
    """M 1 per vertex over the given elements: the row sums of the consistent P1 mass matrix, which
    for P1 are sum over the elements containing the vertex of |T| / (d+1) (the mass formula above
    summed over l). Charge per region is then sum_k z_k (M 1) . c^k. Chunked, volumes only, so it
    runs on meshes of 1e8 elements."""
    d = coords.shape[1]
    out = np.zeros(n_vertices)
    for a in range(0, elems.shape[0], chunk):
        e = elems[a:a + chunk]
        x = coords[e]
        J = x[:, 1:, :] - x[:, :1, :]
        vol = np.abs(np.linalg.det(J)) / factorial(d)
        for j in range(d + 1):
            out += np.bincount(e[:, j], weights=vol / (d + 1), minlength=n_vertices)
    return out


def facet_measure(coords: np.ndarray, facets: np.ndarray) -> np.ndarray:
    """|f| of (d-1)-simplices embedded in R^d (Gram determinant)."""
    x = coords[facets]
    E = x[:, 1:, :] - x[:, :1, :]                      # (n, m, d)
    m = E.shape[1]
    gram = np.einsum("nid,njd->nij", E, E)
    return np.sqrt(np.linalg.det(gram)) / factorial(m)


def moment(m: int, powers) -> float:
    """int over a unit-measure m-simplex of prod lambda_a^{k_a} (the moment formula)."""
    num = factorial(m)
    for k in powers:
        num *= factorial(k)
    return num / factorial(m + sum(powers))


def local_mass(d: int) -> np.ndarray:
    """Mass matrix of a unit-measure d-simplex."""
    n = d + 1
    M = np.empty((n, n))
    for j in range(n):
        for l in range(n):
            M[j, l] = moment(d, [2] if j == l else [1, 1])
    return M


def local_triple(m: int) -> np.ndarray:
    """W[a, j, l] = int over a unit-measure m-simplex of lambda_a lambda_j lambda_l."""
    n = m + 1
    W = np.empty((n, n, n))
    for a in range(n):
        for j in range(n):
            for l in range(n):
                counts = {}
                for v in (a, j, l):
                    counts[v] = counts.get(v, 0) + 1
                W[a, j, l] = moment(m, list(counts.values()))
    return W


def _scatter(rows, cols, vals, n_rows, n_cols):
    return sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=(n_rows, n_cols)).tocsr()


def assemble_bulk(coords, elems, loc, n_nodes):
    """M_r and A_r over the elements of one region; ``loc`` maps vertex -> region node."""
    d = coords.shape[1]
    vol, G = simplex_geometry(coords, elems)
    Mloc = local_mass(d)
    nodes = loc[elems]                                  # (n, d+1)
    rows = np.repeat(nodes[:, :, None], d + 1, axis=2)
    cols = np.repeat(nodes[:, None, :], d + 1, axis=1)
    Me = vol[:, None, None] * Mloc[None]
    Ae = vol[:, None, None] * np.einsum("njx,nlx->njl", G, G)
    return _scatter(rows, cols, Me, n_nodes, n_nodes), _scatter(rows, cols, Ae, n_nodes, n_nodes), (rows, cols, Ae)


def weighted_stiffness(cache, c_nodes, elems_nodes, n_nodes):
    """A_r^{k} for a nodal P1 concentration c (vertex mean per element times the element stiffness)."""
    rows, cols, Ae = cache
    cbar = c_nodes[elems_nodes].mean(axis=1)
    return _scatter(rows, cols, cbar[:, None, None] * Ae, n_nodes, n_nodes)


def membrane_mass(facet_area, row_nodes, col_nodes, n_rows, n_cols, coef=None):
    """int_Gamma (P1 coef) phi_j phi_l over the membrane facets, or int_Gamma phi_j phi_l.

    ``row_nodes``/``col_nodes`` give, per facet, the region-local node of each facet
    vertex on the row side and on the column side (M_{r,Gamma} or M_{rq,Gamma}).
    ``coef`` holds the coefficient's value at each facet vertex, shape (n_f, m+1).
    """
    m1 = row_nodes.shape[1]
    m = m1 - 1
    rows = np.repeat(row_nodes[:, :, None], m1, axis=2)
    cols = np.repeat(col_nodes[:, None, :], m1, axis=1)
    if coef is None:
        vals = facet_area[:, None, None] * (local_mass(m)[None])
    else:
        W = local_triple(m)
        vals = facet_area[:, None, None] * np.einsum("fa,ajl->fjl", coef, W)
    return _scatter(rows, cols, vals, n_rows, n_cols)


def membrane_load(facet_area, row_nodes, q, n_rows):
    """int_Gamma (P1 q) phi_j over the membrane facets; q given at facet vertices (n_f, m+1)."""
    m = row_nodes.shape[1] - 1
    vals = facet_area[:, None] * (q @ local_mass(m))
    return np.bincount(row_nodes.ravel(), weights=vals.ravel(), minlength=n_rows)
