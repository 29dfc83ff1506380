"""Pins for oracle/fem.py against brute-force Gauss quadrature (collapsed coordinates)
on random simplices, and against identities of the global matrices."""
from math import factorial

import numpy as np
import pytest

from oracle import fem
from oracle.topology import build_topology
from synth.configs import model_a


def _duffy_rule(d, n=6):
    """Points and weights on the reference d-simplex via the Duffy map of a tensor Gauss rule."""
    g, w = np.polynomial.legendre.leggauss(n)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    pts, wts = [], []
    if d == 1:
        return g[:, None], w
    if d == 2:
        for i in range(n):
            for j in range(n):
                u, v = g[i], g[j]
                pts.append((u, v * (1 - u)))
                wts.append(w[i] * w[j] * (1 - u))
    if d == 3:
        for i in range(n):
            for j in range(n):
                for k in range(n):
                    u, v, s = g[i], g[j], g[k]
                    pts.append((u, v * (1 - u), s * (1 - u) * (1 - v)))
                    wts.append(w[i] * w[j] * w[k] * (1 - u) ** 2 * (1 - v))
    return np.array(pts), np.array(wts)


def _bary(verts, x):
    """Barycentric coordinates of point x in the simplex by a linear solve."""
    d = verts.shape[1]
    T = np.vstack([verts.T, np.ones(d + 1)])
    return np.linalg.solve(T, np.append(x, 1.0))


def _rand_simplex(rng, d, dim=None):
    dim = d if dim is None else dim
    while True:
        v = rng.standard_normal((d + 1, dim))
        E = v[1:] - v[:1]
        if np.sqrt(abs(np.linalg.det(E @ E.T))) > 0.3:
            return v


@pytest.mark.parametrize("d", [2, 3])
def test_bulk_local_matrices_by_quadrature(d):
    rng = np.random.default_rng(11 + d)
    for _ in range(3):
        v = _rand_simplex(rng, d)
        elems = np.arange(d + 1)[None].astype(np.int32)
        vol, G = fem.simplex_geometry(v, elems)
        ref_pts, ref_w = _duffy_rule(d)
        J = (v[1:] - v[:1]).T
        jac = abs(np.linalg.det(J))
        c = rng.uniform(1, 3, d + 1)
        M_q = np.zeros((d + 1, d + 1))
        Ak_q = np.zeros((d + 1, d + 1))
        h = 1e-6
        for p, w in zip(ref_pts, ref_w):
            x = v[0] + J @ p
            lam = _bary(v, x)
            grads = np.array([[(_bary(v, x + h * e)[j] - _bary(v, x - h * e)[j]) / (2 * h)
                               for e in np.eye(d)] for j in range(d + 1)])
            M_q += w * jac * np.outer(lam, lam)
            Ak_q += w * jac * (c @ lam) * grads @ grads.T
        assert np.isclose(vol[0], jac / factorial(d))
        np.testing.assert_allclose(vol[0] * fem.local_mass(d), M_q, rtol=1e-12, atol=1e-14)
        Ae = vol[0] * G[0] @ G[0].T
        np.testing.assert_allclose(c.mean() * Ae, Ak_q, rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("m,dim", [(1, 2), (2, 3)])
def test_facet_triple_products_by_quadrature(m, dim):
    rng = np.random.default_rng(5 + m)
    v = _rand_simplex(rng, m, dim)
    area = fem.facet_measure(v, np.arange(m + 1)[None])[0]
    E = (v[1:] - v[:1])
    gram_area = np.sqrt(np.linalg.det(E @ E.T)) / factorial(m)
    assert np.isclose(area, gram_area)
    ref_pts, ref_w = _duffy_rule(m)
    W_q = np.zeros((m + 1,) * 3)
    M_q = np.zeros((m + 1,) * 2)
    for p, w in zip(ref_pts, ref_w):
        lam = np.concatenate([[1 - p.sum()], p])
        W_q += w * factorial(m) * area * np.einsum("a,j,l->ajl", lam, lam, lam)
        M_q += w * factorial(m) * area * np.outer(lam, lam)
    np.testing.assert_allclose(area * fem.local_triple(m), W_q, rtol=1e-12)
    np.testing.assert_allclose(area * fem.local_mass(m), M_q, rtol=1e-12)
    # coefficient-weighted membrane mass on this single facet
    coef = rng.uniform(-1, 2, m + 1)
    nodes = np.arange(m + 1)[None]
    Mc = fem.membrane_mass(np.array([area]), nodes, nodes, m + 1, m + 1, coef=coef[None]).toarray()
    np.testing.assert_allclose(Mc, np.einsum("a,ajl->jl", coef, W_q), rtol=1e-12)
    # load vector of a P1 function
    q = rng.standard_normal(m + 1)
    L = fem.membrane_load(np.array([area]), nodes, q[None], m + 1)
    np.testing.assert_allclose(L, M_q @ q, rtol=1e-12)


@pytest.mark.parametrize("d,nx", [(2, 8), (3, 4)])
def test_global_matrix_identities(d, nx):
    cfg = model_a(d, nx, 1e-4)
    m = cfg.mesh
    t = build_topology(m.coords, m.elems, m.elem_tag)
    M, A, cache = fem.assemble_bulk(m.coords, m.elems[t.elems_e], t.loc_e, t.N_e)
    vol_e = 1e-6 ** d * (1 - 0.5 ** d)
    assert np.isclose(M.sum(), vol_e, rtol=1e-12)
    assert np.abs(A @ np.ones(t.N_e)).max() < 1e-12 * np.abs(A).max()
    assert abs(M - M.T).max() == 0 and abs(A - A.T).max() < 1e-12 * np.abs(A).max()
    en = t.loc_e[m.elems[t.elems_e]]
    A1 = fem.weighted_stiffness(cache, np.ones(t.N_e), en, t.N_e)
    assert abs(A1 - A).max() < 1e-14 * np.abs(A).max()
    # A^k with a linear c: rows still sum to zero (the constant is in the kernel)
    c = m.coords[t.nodes_e, 0] * 1e6 + 2.0
    Ak = fem.weighted_stiffness(cache, c, en, t.N_e)
    assert np.abs(Ak @ np.ones(t.N_e)).max() < 1e-12 * np.abs(Ak).max()


def test_vertex_volumes_are_the_mass_row_sums():
    """vertex_volumes equals M 1 of the assembled consistent mass matrix (chunked or not) and sums
    to the region's volume."""
    from synth import make_config
    from oracle import fem
    cfg = make_config(2).with_nx(6)
    m = cfg.mesh
    n = m.coords.shape[0]
    loc = np.arange(n)
    M, _, _ = fem.assemble_bulk(m.coords, m.elems, loc, n)
    for chunk in (10_000_000, 97):
        v = fem.vertex_volumes(m.coords, m.elems, n, chunk=chunk)
        assert np.allclose(v, np.asarray(M.sum(axis=1)).ravel(), rtol=1e-12, atol=0)
    assert abs(v.sum() - cfg.length ** 3) < 1e-12 * cfg.length ** 3
