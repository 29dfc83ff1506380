"""P2 Lagrange elements for the KNP-EMI system (Section 3.3 with p = 2; Section 6.3; Table 4).

TEST INFRASTRUCTURE ONLY, like the rest of this package.

Section 3.3 leaves the polynomial degree p of the Lagrange spaces free, and Section 6.3 runs
p in {1, 2}. This module gives the p = 2 space on the same conforming tessellation as the P1
oracle, and the matrices of Section 4.1 in it:
  * nodes: every vertex and every edge; a node belongs to a region when it is a node of one of
    the region's elements, so the nodes on Gamma (vertices and edges of membrane facets) are
    repeated for Omega_i and Omega_e, as the vertices are for p = 1;
  * global node ids: the vertices 0..n_v-1, then the edges in lexicographic order of their
    sorted vertex pair (an edge node sits at the edge midpoint); region node order is increasing
    global id;
  * element nodes: the d+1 vertices in the element's order, then the edges (a, b), a < b, in
    lexicographic order of the local pair; facet nodes likewise, from the sorted facet vertices;
  * basis on a simplex with barycentric coordinates lambda: lambda_a (2 lambda_a - 1) for vertex
    a and 4 lambda_a lambda_b for edge (a, b).
Every basis function, and every partial derivative of one in a barycentric coordinate, is a
polynomial in lambda, and grad phi = sum_a (d phi / d lambda_a) grad lambda_a, so each integral
of Section 4.1 is an exact sum of barycentric moments (fem.moment): M_r, A_r, A_r^{k} with a P2
concentration, the membrane masses, and the membrane masses weighted by a P2 coefficient.
Membrane coefficients are nodal, as for p = 1, now at the P2 membrane nodes; the gating ODEs are
solved at those nodes (Section 3.3).

weighted_stiffness, membrane_mass and membrane_load take the arguments of their P1 counterparts
in ``fem``; with ``Problem.fe`` set to this module, system.assemble and system.preconditioner_P0
build the p = 2 system unchanged.

Pinned by tests/test_oracle_p2.py: local matrices against brute-force quadrature of the closed-form
basis on random simplices; exact energies of quadratic fields (P2 reproduces quadratics, P1 does
not) for M_r, A_r, A_r^{k}, M_{r,Gamma} and the weighted membrane mass on Model A meshes; the
Model A count of Section 5.1 with p = 2 and the 4.2e6 unknowns of Section 6.3 for (N_x, p) =
(512, 2); the resting steady state, charge conservation, species balance and a manufactured
discrete solution of the p = 2 system; the LU(P_0)-GMRES iteration counts of Section 6.3, which
the paper states for p = 2 as well.
"""
from __future__ import annotations

from dataclasses import dataclass
from functools import lru_cache

import numpy as np
import scipy.sparse as sp

from . import fem
from .topology import InvalidMesh, Topology, build_topology as build_p1_topology


# ---------------------------------------------------------------- polynomials in barycentrics
# A polynomial in lambda_0..lambda_m is a dict {exponent tuple: coefficient}. The representation
# is not unique (the lambdas sum to 1), which does not matter: integrals and the chain rule hold
# for any polynomial expression in lambda.

def local_pairs(m: int):
    """The edges (a, b), a < b, of an m-simplex in lexicographic order."""
    return [(a, b) for a in range(m + 1) for b in range(a + 1, m + 1)]


def _exp(n, *idx):
    return tuple(sum(1 for i in idx if i == k) for k in range(n))


def _mul(p, q):
    out = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            out[e] = out.get(e, 0.0) + ca * cb
    return out


def _dlam(p, a):
    """d p / d lambda_a."""
    out = {}
    for e, c in p.items():
        if e[a]:
            ne = list(e)
            ne[a] -= 1
            ne = tuple(ne)
            out[ne] = out.get(ne, 0.0) + c * e[a]
    return out


def _integral(m, p):
    """int over a unit-measure m-simplex of p (moment formula, term by term)."""
    return sum(c * fem.moment(m, list(e)) for e, c in p.items())


@lru_cache(maxsize=None)
def basis(m: int):
    """The P2 Lagrange basis of an m-simplex: vertices 0..m, then the edges of local_pairs(m)."""
    n = m + 1
    out = [{_exp(n, a, a): 2.0, _exp(n, a): -1.0} for a in range(n)]
    out += [{_exp(n, a, b): 4.0} for a, b in local_pairs(m)]
    return tuple(out)


def n_local(m: int) -> int:
    return (m + 1) * (m + 2) // 2


@lru_cache(maxsize=None)
def local_mass(m: int) -> np.ndarray:
    """Mloc[j, l] = int phi_j phi_l over a unit-measure m-simplex."""
    B = basis(m)
    return np.array([[_integral(m, _mul(bj, bl)) for bl in B] for bj in B])


@lru_cache(maxsize=None)
def local_triple(m: int) -> np.ndarray:
    """W[c, j, l] = int phi_c phi_j phi_l over a unit-measure m-simplex."""
    B = basis(m)
    n = len(B)
    W = np.empty((n, n, n))
    for c in range(n):
        for j in range(n):
            cj = _mul(B[c], B[j])
            for l in range(n):
                W[c, j, l] = _integral(m, _mul(cj, B[l]))
    return W


@lru_cache(maxsize=None)
def _partials(d: int):
    B = basis(d)
    return [[_dlam(b, a) for a in range(d + 1)] for b in B]


@lru_cache(maxsize=None)
def local_stiffness(d: int) -> np.ndarray:
    """K[j, l, a, b] = int (d phi_j / d lambda_a)(d phi_l / d lambda_b) over a unit-measure d-simplex;
    the element stiffness is |T| sum_ab K[j, l, a, b] grad lambda_a . grad lambda_b."""
    P = _partials(d)
    n = len(P)
    K = np.empty((n, n, d + 1, d + 1))
    for j in range(n):
        for l in range(n):
            for a in range(d + 1):
                for b in range(d + 1):
                    K[j, l, a, b] = _integral(d, _mul(P[j][a], P[l][b]))
    return K


@lru_cache(maxsize=None)
def local_weighted(d: int) -> np.ndarray:
    """S[c, j, l, a, b] = int phi_c (d phi_j / d lambda_a)(d phi_l / d lambda_b) over a unit-measure
    d-simplex; A^{k} of an element is |T| sum_{c,a,b} [k]_c S[c, j, l, a, b] grad lambda_a . grad lambda_b."""
    B = basis(d)
    P = _partials(d)
    n = len(B)
    S = np.empty((n, n, n, d + 1, d + 1))
    for j in range(n):
        for l in range(n):
            for a in range(d + 1):
                for b in range(d + 1):
                    q = _mul(P[j][a], P[l][b])
                    for c in range(n):
                        S[c, j, l, a, b] = _integral(d, _mul(B[c], q))
    return S


def _facet_dim(n_nodes_per_facet: int) -> int:
    for m in (0, 1, 2):
        if n_local(m) == n_nodes_per_facet:
            return m
    raise ValueError("not a P2 facet node table")


# ---------------------------------------------------------------- matrices (fem's signatures)

def _scatter(rows, cols, vals, n_rows, n_cols):
    return sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=(n_rows, n_cols)).tocsr()


def assemble_bulk(coords, elems, enodes, n_nodes):
    """M_r and A_r over the region's elements; ``elems`` (n, d+1) vertex ids, ``enodes`` (n, n_loc)
    region-local P2 nodes. Returns (M_r, A_r, cache) with cache = (rows, cols, |T|, Gab)."""
    d = coords.shape[1]
    vol, G = fem.simplex_geometry(coords, elems)
    Gab = np.einsum("nax,nbx->nab", G, G)
    nl = enodes.shape[1]
    rows = np.repeat(enodes[:, :, None], nl, axis=2)
    cols = np.repeat(enodes[:, None, :], nl, axis=1)
    Me = vol[:, None, None] * local_mass(d)[None]
    Ae = vol[:, None, None] * np.einsum("jlab,nab->njl", local_stiffness(d), Gab)
    return _scatter(rows, cols, Me, n_nodes, n_nodes), _scatter(rows, cols, Ae, n_nodes, n_nodes), (rows, cols, vol, Gab)


def weighted_stiffness(cache, c_nodes, elems_nodes, n_nodes):
    """A_r^{k} = [int [k] grad phi_j . grad phi_l] for a nodal P2 concentration [k]."""
    rows, cols, vol, Gab = cache
    d = Gab.shape[1] - 1
    ce = c_nodes[elems_nodes]                                      # (n, n_loc)
    T = np.einsum("nc,cjlab->njlab", ce, local_weighted(d), optimize=True)
    vals = vol[:, None, None] * np.einsum("njlab,nab->njl", T, Gab, optimize=True)
    return _scatter(rows, cols, vals, n_nodes, n_nodes)


def membrane_mass(facet_area, row_nodes, col_nodes, n_rows, n_cols, coef=None):
    """int_Gamma (P2 coef) phi_j phi_l, or int_Gamma phi_j phi_l, over the membrane facets.

    ``row_nodes``/``col_nodes`` (n_f, n_floc): per facet, the node of each facet P2 node on the row
    and on the column side; ``coef`` the coefficient's values at the facet nodes, (n_f, n_floc).
    """
    nl = row_nodes.shape[1]
    m = _facet_dim(nl)
    rows = np.repeat(row_nodes[:, :, None], nl, axis=2)
    cols = np.repeat(col_nodes[:, None, :], nl, axis=1)
    if coef is None:
        vals = facet_area[:, None, None] * local_mass(m)[None]
    else:
        vals = facet_area[:, None, None] * np.einsum("fa,ajl->fjl", coef, local_triple(m))
    return _scatter(rows, cols, vals, n_rows, n_cols)


def membrane_load(facet_area, row_nodes, q, n_rows):
    """int_Gamma (P2 q) phi_j over the membrane facets; q at the facet nodes, (n_f, n_floc)."""
    m = _facet_dim(row_nodes.shape[1])
    vals = facet_area[:, None] * (q @ local_mass(m))
    return np.bincount(row_nodes.ravel(), weights=vals.ravel(), minlength=n_rows)


# ---------------------------------------------------------------- topology

@dataclass
class P2Topology:
    base: Topology             # the vertex-level topology (facets, regions, checks)
    edges: np.ndarray          # (n_edges, 2) sorted vertex pairs, lexicographic
    elem_nodes: np.ndarray     # (n_e, n_loc) global P2 node ids
    facet_nodes: np.ndarray    # (n_f, n_floc) global P2 node ids
    node_coords: np.ndarray    # (n_nodes, d)
    nodes_i: np.ndarray        # global ids of the region nodes, increasing
    nodes_e: np.ndarray
    loc_i: np.ndarray          # global id -> region-local index (-1 if absent)
    loc_e: np.ndarray
    membrane_nodes: np.ndarray  # sorted global ids of the nodes on Gamma
    node_cell_i: np.ndarray    # (N_i,) cell tag of each intracellular node
    pin_node: int              # global id of the pinned extracellular node

    @property
    def dim(self):
        return self.base.dim

    @property
    def elems_i(self):
        return self.base.elems_i

    @property
    def elems_e(self):
        return self.base.elems_e

    @property
    def facets(self):
        return self.base.facets

    @property
    def N_i(self):
        return len(self.nodes_i)

    @property
    def N_e(self):
        return len(self.nodes_e)

    def n_dof(self, n_ions: int) -> int:
        return (self.N_i + self.N_e) * (n_ions + 1)


def _edge_ids(edges, n_v, pairs):
    """Global edge index of each sorted vertex pair in ``pairs`` (..., 2)."""
    keys = edges[:, 0].astype(np.int64) * n_v + edges[:, 1]
    q = pairs[..., 0].astype(np.int64) * n_v + pairs[..., 1]
    idx = np.searchsorted(keys, q)
    if np.any(idx >= len(keys)) or np.any(keys[np.minimum(idx, len(keys) - 1)] != q):
        raise InvalidMesh("a facet edge is not an element edge")
    return idx


def build_topology(coords: np.ndarray, elems: np.ndarray, tag: np.ndarray, pin_point=None) -> P2Topology:
    """P2 nodes, their region copies and the element and facet node tables (Section 3.3, p = 2)."""
    base = build_p1_topology(coords, elems, tag, pin_point=pin_point)
    n_v, d = coords.shape
    pe = local_pairs(d)
    e_all = np.sort(np.stack([elems[:, [a, b]] for a, b in pe], axis=1), axis=2)   # (n_e, n_pairs, 2)
    edges, inv = np.unique(e_all.reshape(-1, 2), axis=0, return_inverse=True)
    elem_edges = inv.reshape(elems.shape[0], len(pe))
    elem_nodes = np.hstack([elems.astype(np.int64), n_v + elem_edges])
    pf = local_pairs(d - 1)
    fpairs = np.stack([base.facets[:, [a, b]] for a, b in pf], axis=1)             # sorted facets
    facet_nodes = np.hstack([base.facets.astype(np.int64), n_v + _edge_ids(edges, n_v, fpairs)])
    node_coords = np.vstack([coords, 0.5 * (coords[edges[:, 0]] + coords[edges[:, 1]])])
    n_nodes = len(node_coords)

    in_i = np.zeros(n_nodes, bool)
    in_i[elem_nodes[base.elems_i].ravel()] = True
    in_e = np.zeros(n_nodes, bool)
    in_e[elem_nodes[base.elems_e].ravel()] = True
    on_gamma = np.zeros(n_nodes, bool)
    on_gamma[facet_nodes.ravel()] = True
    if np.any((in_i & in_e) != on_gamma):
        raise InvalidMesh("regions share an edge outside the membrane facets")
    nodes_i = np.nonzero(in_i)[0]
    nodes_e = np.nonzero(in_e)[0]
    loc_i = np.full(n_nodes, -1, np.int64)
    loc_i[nodes_i] = np.arange(len(nodes_i))
    loc_e = np.full(n_nodes, -1, np.int64)
    loc_e[nodes_e] = np.arange(len(nodes_e))
    # cell of an intracellular node: the cell of its elements (one cell per vertex, checked by the
    # P1 topology, hence one per edge)
    cell = np.zeros(n_nodes, np.int64)
    ei = base.elems_i
    cell[elem_nodes[ei].ravel()] = np.repeat(tag[ei], elem_nodes.shape[1])
    # pin: extracellular node nearest to the pin point (origin by default), ties by lowest id
    p0 = np.zeros(d) if pin_point is None else np.asarray(pin_point, float)
    d2 = np.sum((node_coords[nodes_e] - p0) ** 2, axis=1)
    k = np.flatnonzero(d2 == d2.min())[0]
    return P2Topology(base, edges, elem_nodes, facet_nodes, node_coords, nodes_i, nodes_e, loc_i,
                      loc_e, np.nonzero(on_gamma)[0], cell[nodes_i], int(nodes_e[k]))


def discretize(pb) -> None:
    """Static geometry of a p = 2 problem: the same ``geo`` entries as system.discretize."""
    t = pb.topo
    g = pb.geo
    el = pb.elems
    g["en_i"] = t.loc_i[t.elem_nodes[t.elems_i]]
    g["en_e"] = t.loc_e[t.elem_nodes[t.elems_e]]
    g["M_i"], g["A_i"], g["cache_i"] = assemble_bulk(pb.coords, el[t.elems_i], g["en_i"], t.N_i)
    g["M_e"], g["A_e"], g["cache_e"] = assemble_bulk(pb.coords, el[t.elems_e], g["en_e"], t.N_e)
    g["area"] = fem.facet_measure(pb.coords, t.facets)
    g["fv"] = np.searchsorted(t.membrane_nodes, t.facet_nodes)      # facet node -> membrane index
    g["fi"] = t.loc_i[t.facet_nodes]
    g["fe"] = t.loc_e[t.facet_nodes]
    g["mv_i"] = t.loc_i[t.membrane_nodes]
    g["mv_e"] = t.loc_e[t.membrane_nodes]
    g["pin"] = int(t.loc_e[t.pin_node])
    g["MG_i"] = membrane_mass(g["area"], g["fi"], g["fi"], t.N_i, t.N_i)
    g["MG_e"] = membrane_mass(g["area"], g["fe"], g["fe"], t.N_e, t.N_e)
    g["MG_ie"] = membrane_mass(g["area"], g["fi"], g["fe"], t.N_i, t.N_e)
    g["MG_ei"] = membrane_mass(g["area"], g["fe"], g["fi"], t.N_e, t.N_i)
    g["n_mv"] = len(t.membrane_nodes)
    if pb.stim_mask is None:
        pb.stim_mask = np.ones(len(t.facets), bool)
