"""Membrane detection, node duplication and DOF numbering (Section 3.3; Section 5.1 Model A).

The conforming tessellation T = T_i U T_e matches at Gamma; every membrane
vertex carries one degree of freedom per field in each region (the DOFs on
Gamma are repeated for Omega_i and Omega_e, Section 5.1). Region node order is
increasing vertex id; the membrane facet order is lexicographic in the sorted
vertex tuple. Pinned by tests/test_oracle_topology.py (DOF-count formula of
Section 5.1 and the N column of Table 3).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Topology:
    dim: int
    n_vertices: int
    # region node sets: vertex ids in increasing order
    nodes_i: np.ndarray
    nodes_e: np.ndarray
    # vertex id -> local node index in region (-1 if absent)
    loc_i: np.ndarray
    loc_e: np.ndarray
    elems_i: np.ndarray        # element ids with tag >= 1
    elems_e: np.ndarray        # element ids with tag == 0
    facets: np.ndarray         # (n_f, dim) sorted vertex ids of membrane facets, lexicographic
    facet_cell: np.ndarray     # (n_f,) cell tag (>=1) of the facet's intracellular element
    facet_elem_i: np.ndarray   # (n_f,) intracellular element id
    facet_opp_i: np.ndarray    # (n_f,) local index (0..dim) of the i-element vertex opposite the facet
    membrane_vertices: np.ndarray  # sorted vertex ids on Gamma
    node_cell_i: np.ndarray    # (N_i,) cell tag of each intracellular node
    pin_vertex: int            # vertex id of the pinned extracellular node

    @property
    def N_i(self):
        return len(self.nodes_i)

    @property
    def N_e(self):
        return len(self.nodes_e)

    def n_dof(self, n_ions: int) -> int:
        return (self.N_i + self.N_e) * (n_ions + 1)


class InvalidMesh(ValueError):
    pass


def build_topology(coords: np.ndarray, elems: np.ndarray, tag: np.ndarray, pin_point=None) -> Topology:
    n_v, dim = coords.shape
    n_e = elems.shape[0]
    # all (element, local facet) pairs; facet s is opposite local vertex s
    fac = []
    for s in range(dim + 1):
        cols = [c for c in range(dim + 1) if c != s]
        fac.append(np.sort(elems[:, cols], axis=1))
    fac = np.stack(fac, axis=1).reshape(-1, dim)        # (n_e*(dim+1), dim)
    owner = np.repeat(np.arange(n_e), dim + 1)
    opp = np.tile(np.arange(dim + 1), n_e)
    order = np.lexsort(fac.T[::-1])
    fs = fac[order]
    same_as_next = np.all(fs[1:] == fs[:-1], axis=1)
    # interior facets: appear exactly twice in a conforming mesh
    idx = np.nonzero(same_as_next)[0]
    a, b = order[idx], order[idx + 1]
    ta, tb = tag[owner[a]], tag[owner[b]]
    diff = ta != tb
    if np.any(diff & (ta > 0) & (tb > 0)):
        raise InvalidMesh("two cells share a facet")
    mem = np.nonzero(diff)[0]
    a, b, ta, tb = a[mem], b[mem], ta[mem], tb[mem]
    i_slot = np.where(ta > 0, a, b)
    facets = fac[i_slot]
    facet_elem_i = owner[i_slot]
    facet_opp_i = opp[i_slot]
    facet_cell = tag[facet_elem_i]
    o = np.lexsort(facets.T[::-1])
    facets, facet_elem_i, facet_opp_i, facet_cell = facets[o], facet_elem_i[o], facet_opp_i[o], facet_cell[o]

    elems_i = np.nonzero(tag > 0)[0]
    elems_e = np.nonzero(tag == 0)[0]
    in_i = np.zeros(n_v, bool)
    in_i[elems[elems_i].ravel()] = True
    in_e = np.zeros(n_v, bool)
    in_e[elems[elems_e].ravel()] = True
    on_gamma = np.zeros(n_v, bool)
    on_gamma[facets.ravel()] = True
    if np.any((in_i & in_e) != on_gamma):
        raise InvalidMesh("regions touch outside the membrane facets")
    # a vertex may not belong to two different cells
    cell_of = np.full(n_v, 0, np.int64)
    ecell = np.repeat(tag[elems_i], dim + 1)
    ev = elems[elems_i].ravel()
    cell_min = np.full(n_v, np.iinfo(np.int64).max)
    cell_max = np.full(n_v, -1)
    np.minimum.at(cell_min, ev, ecell)
    np.maximum.at(cell_max, ev, ecell)
    if np.any(in_i & (cell_min != cell_max)):
        raise InvalidMesh("a vertex belongs to two cells")
    cell_of[in_i] = cell_min[in_i]

    nodes_i = np.nonzero(in_i)[0]
    nodes_e = np.nonzero(in_e)[0]
    loc_i = np.full(n_v, -1, np.int64)
    loc_i[nodes_i] = np.arange(len(nodes_i))
    loc_e = np.full(n_v, -1, np.int64)
    loc_e[nodes_e] = np.arange(len(nodes_e))
    cells_present = np.unique(tag[elems_i])
    if not np.all(np.isin(cells_present, facet_cell)):
        raise InvalidMesh("a cell has no membrane facet")

    # pin: extracellular vertex nearest to the pin point (the origin corner by default), ties by
    # lowest id (Remark 4.1 allows any extracellular node)
    p0 = np.zeros(coords.shape[1]) if pin_point is None else np.asarray(pin_point, float)
    d2 = np.sum((coords[nodes_e] - p0) ** 2, axis=1)
    k = np.flatnonzero(d2 == d2.min())[0]
    return Topology(dim, n_v, nodes_i, nodes_e, loc_i, loc_e, elems_i, elems_e, facets,
                    facet_cell, facet_elem_i, facet_opp_i, np.nonzero(on_gamma)[0],
                    cell_of[nodes_i], int(nodes_e[k]))


def model_a_dof_count(d: int, nx: int, p: int, n_ions: int) -> int:
    """The closed-form count of Section 5.1 for Model A (cell [0.25,0.75]^d)."""
    return int(((p * nx + 1) ** d + (3 - d / 2) * (p * nx) ** (d - 1) + 2 * (d - 2)) * (n_ions + 1))
