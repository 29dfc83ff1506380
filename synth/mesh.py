"""Structured simplicial meshes shaped like the paper's Model A (Section 5.1).

The unit square/cube is cut into N_x intervals per side. In 2D each square is
split into two right triangles along its (0,0)-(1,1) diagonal; in 3D each cube
is split into the six Kuhn (Freudenthal) tetrahedra that share the main
diagonal, which gives a conforming tessellation. Vertex ids are lexicographic
with x fastest. Cells are axis-aligned boxes whose faces are snapped to grid
planes, so every element lies entirely inside one region.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np


@dataclass
class StructuredMesh:
    dim: int
    nx: int
    coords: np.ndarray      # (n_vertices, dim) float64, metres
    elems: np.ndarray       # (n_elems, dim+1) int32 vertex ids
    elem_tag: np.ndarray    # (n_elems,) int32: 0 = extracellular, j>=1 = cell j
    boxes: np.ndarray       # (n_cells, 2, dim) int64 snapped grid-index boxes [lo, hi]
    length: float           # side of the domain in metres


def _vid(idx, n1s):
    v = idx[..., 0].astype(np.int64)
    stride = n1s[0]
    for a in range(1, len(n1s)):
        v = v + idx[..., a].astype(np.int64) * stride
        stride *= n1s[a]
    return v


def structured_mesh(dim: int, nx: int, length: float, axes=None):
    """Vertices and simplices of the grid of [0, length]^dim: uniform with nx intervals per side,
    or with the grid-plane coordinates ``axes[a]`` (increasing, from 0 to length) along axis a."""
    if axes is None:
        axes = [np.arange(nx + 1, dtype=np.float64) / nx * length] * dim
    n1s = [len(ax) for ax in axes]
    grid = np.meshgrid(*axes, indexing="ij")
    # lexicographic with x fastest
    coords = np.stack([g.transpose(tuple(range(dim))[::-1]).reshape(-1) for g in grid], axis=1)
    base = np.stack(np.meshgrid(*[np.arange(n - 1) for n in n1s], indexing="ij"), axis=-1)
    base = base.transpose(tuple(range(dim))[::-1] + (dim,)).reshape(-1, dim)
    elems = []
    for perm in itertools.permutations(range(dim)):
        if dim == 2 and perm not in ((0, 1), (1, 0)):
            continue
        path = [base.copy()]
        cur = base.copy()
        for ax in perm:
            cur = cur.copy()
            cur[:, ax] += 1
            path.append(cur)
        elems.append(np.stack([_vid(p, n1s) for p in path], axis=1))
    # interleave so that the simplices of one grid box are consecutive
    elems = np.stack(elems, axis=1).reshape(-1, dim + 1).astype(np.int32)
    return coords, elems


def interface_refined_axis(nx: int, length: float, faces, ratio: int, width: int):
    """Grid planes of one axis: the uniform grid of nx intervals with every interval within
    ``width`` intervals of a face plane (uniform grid index) cut into ``ratio`` equal pieces.
    Returns the plane coordinates and the new index of each uniform plane."""
    faces = np.unique(np.asarray(faces))
    pts, new_index = [0.0], [0]
    for i in range(nx):
        near = np.any(np.abs(i + 0.5 - faces) <= width)
        k = ratio if near else 1
        for j in range(1, k + 1):
            pts.append((i + j / k) / nx * length)
        new_index.append(len(pts) - 1)
    return np.array(pts), np.array(new_index)


def snap_boxes(lo: np.ndarray, hi: np.ndarray, nx: int) -> np.ndarray:
    """Snap box corners (fractions of the side) to grid planes, half away from zero."""
    lo_i = np.floor(np.asarray(lo) * nx + 0.5).astype(np.int64)
    hi_i = np.floor(np.asarray(hi) * nx + 0.5).astype(np.int64)
    return np.stack([lo_i, hi_i], axis=-2)


def box_cells(n_per_side: int, side: float, gap: float, dim: int, jitter=None, rng=None):
    """Centred n^dim array of cubic cells with the given side and gap (fractions of the domain).

    With ``jitter`` = (a, b), each side of each cell is scaled about the cell centre by
    an independent U(a, b) factor drawn from ``rng``.
    """
    extent = n_per_side * side + (n_per_side - 1) * gap
    start = 0.5 - extent / 2
    lows, highs = [], []
    for idx in itertools.product(range(n_per_side), repeat=dim):
        lo = np.array([start + i * (side + gap) for i in idx[::-1]])
        hi = lo + side
        if jitter is not None:
            c = 0.5 * (lo + hi)
            s = rng.uniform(jitter[0], jitter[1], size=dim) * side
            lo, hi = c - s / 2, c + s / 2
        lows.append(lo)
        highs.append(hi)
    return np.array(lows), np.array(highs)


def tag_grid_boxes(dim: int, counts, boxes: np.ndarray) -> np.ndarray:
    """Tag of every grid box (flattened with x fastest): the last cell box [lo, hi] (grid plane
    indices) that contains it, 0 if none. ``counts`` is the number of grid boxes along each axis
    (an int for all). A simplex lies in one grid box, and its centroid is strictly inside a
    cell box exactly when its grid box is, so this is the tag of every simplex of that grid box."""
    counts = (counts,) * dim if np.isscalar(counts) else tuple(counts)
    tag = np.zeros(counts[::-1], dtype=np.int32)          # axes (z, y, x) / (y, x)
    for j, (lo, hi) in enumerate(boxes):
        tag[tuple(slice(int(lo[a]), int(hi[a])) for a in range(dim)[::-1])] = j + 1
    return tag.reshape(-1)


def make_mesh(dim: int, nx: int, length: float, lo, hi, refine=None) -> StructuredMesh:
    """Mesh with box cells snapped to the uniform nx grid. With ``refine`` = (ratio, width), the
    grid intervals within ``width`` intervals of a cell face plane are cut into ``ratio`` slabs
    (interface refinement on a tensor grid; the cells do not move). ``boxes`` stay in uniform
    grid units."""
    boxes = snap_boxes(np.atleast_2d(lo), np.atleast_2d(hi), nx)
    if np.any(boxes[:, 1] - boxes[:, 0] < 1):
        raise ValueError("a cell snapped to zero width")
    if np.any(boxes[:, 0] < 1) or np.any(boxes[:, 1] > nx - 1):
        raise ValueError("cells must stay inside the domain interior")
    if refine is None:
        coords, elems = structured_mesh(dim, nx, length)
        counts, rboxes = (nx,) * dim, boxes
    else:
        ratio, width = refine
        axes, maps = [], []
        for a in range(dim):
            ax, mp = interface_refined_axis(nx, length, boxes[:, :, a], ratio, width)
            axes.append(ax)
            maps.append(mp)
        coords, elems = structured_mesh(dim, nx, length, axes)
        counts = tuple(len(ax) - 1 for ax in axes)
        rboxes = np.stack([np.stack([maps[a][boxes[:, e, a]] for a in range(dim)], axis=1) for e in range(2)],
                          axis=1)
    # structured_mesh emits the simplices of one grid box consecutively, grid boxes x fastest
    per_box = elems.shape[0] // int(np.prod(counts))
    tag = np.repeat(tag_grid_boxes(dim, counts, rboxes), per_box)
    return StructuredMesh(dim, nx, coords, elems, tag, boxes, length)
