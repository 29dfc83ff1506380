"""Workload definitions: Table 2 parameters and the five synthetic scenarios.

Everything here is input data (numbers, meshes, seeded draws). Values follow
Table 2 of the paper unless a scenario overrides them; the scenarios are
structured meshes shaped like Model A (Section 5.1) scaled to a 100 um box.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

from .mesh import StructuredMesh, box_cells, make_mesh


def table2() -> dict:
    """Physical parameters and initial values of Table 2 (SI units; C_M read as F/m^2)."""
    return dict(
        R=8.314, T=300.0, F=9.648e4, Cm=0.02,
        ions=("Na", "K", "Cl"), z=(1.0, 1.0, -1.0),
        D=(1.33e-9, 1.96e-9, 2.03e-9),
        g_leak=(1.0, 4.0, 0.0), gbar_K=360.0, gbar_Na=1200.0,
        gbar_stim=40.0, stim_a=2e-3, stim_tau=10e-3,
        c_i0=(12.0, 125.0, 137.0), c_e0=(100.0, 4.0, 104.0),
        phi_M0=-67.74e-3, phi_rest=-65e-3,
        m0=0.0379, h0=0.688, n0=0.276,
        rho_pump=1.115e-6, P_Na=10.0, P_K=1.5,
    )


# stimulus kinds
STIM_NONE, STIM_WINDOW, STIM_PERIODIC_EXP = 0, 1, 2
# membrane models
MODEL_LEAK, MODEL_HH, MODEL_KIR = 0, 1, 2


@dataclass
class Config:
    name: str
    dim: int
    nx: int
    length: float                 # metres
    cell_lo: np.ndarray           # (n_cells, dim) fractions of the side
    cell_hi: np.ndarray
    model: int                    # MODEL_LEAK, MODEL_HH or MODEL_KIR (all facets)
    g_leak: tuple                 # (Na, K, Cl) S/m^2
    dt: float                     # s
    n_steps: int
    rtol: float
    mixed: bool = False           # FP32 AMG hierarchy under FP64 FGMRES
    stim_kind: int = STIM_NONE
    stim_gbar: float = 0.0
    stim_t0: float = 0.0
    stim_t1: float = 0.0
    stim_a: float = 2e-3
    stim_tau: float = 10e-3
    stim_xmax: float = np.inf     # stimulated facets: centroid x < stim_xmax (metres)
    gK_sigma: float = 0.0         # per-facet g_K = g_leak_K * exp(sigma * xi)
    seed_gK: int = 1
    source_e: Optional[tuple] = None  # bulk source (Na, K, Cl), mol/(m^3 s), on extracellular
    source_xmax: float = np.inf       # vertices with x < source_xmax (metres), switched on
    source_t0: float = 0.0            # for source_t0 < t_n <= source_t1
    source_t1: float = 0.0
    refine: Optional[tuple] = None    # (ratio, width): interface refinement of the tensor grid
    params: dict = field(default_factory=table2)
    _mesh: Optional[StructuredMesh] = None

    @property
    def mesh(self) -> StructuredMesh:
        if self._mesh is None:
            self._mesh = make_mesh(self.dim, self.nx, self.length, self.cell_lo, self.cell_hi, self.refine)
        return self._mesh

    def elem_facet_xi(self) -> np.ndarray:
        """Standard normal draws, one per (element, local facet) slot (PCG64, seed_gK).

        A membrane facet takes the draw of its intracellular element's slot whose
        local facet is the one opposite local vertex ``s``.
        """
        m = self.mesh
        rng = np.random.Generator(np.random.PCG64(self.seed_gK))
        return rng.standard_normal((m.elems.shape[0], self.dim + 1))

    def vertex_source_e(self) -> Optional[np.ndarray]:
        """(n_vertices, n_ions) bulk source values for the extracellular copy of each vertex:
        source_e where the vertex's x < source_xmax, else 0; None without a source."""
        return self.source_e_at(self.mesh.coords)

    def source_e_at(self, points: np.ndarray) -> Optional[np.ndarray]:
        """(n_points, n_ions) extracellular bulk source values at arbitrary points (P2 nodes)."""
        if self.source_e is None:
            return None
        on = (np.asarray(points)[:, 0] < self.source_xmax).astype(float)
        return on[:, None] * np.asarray(self.source_e, float)[None, :]

    def with_nx(self, nx: int) -> "Config":
        return replace(self, nx=nx, _mesh=None)


def _single(dim, lo, hi):
    return np.full((1, dim), lo), np.full((1, dim), hi)


def make_config(i: int) -> Config:
    """Configs 1..5: the synthetic workloads; 6, 7: the Kir-Na/K workloads with a bulk source."""
    L = 100e-6
    if i == 1:
        lo, hi = _single(2, 0.25, 0.75)
        return Config("cfg1-2d-32-leak", 2, 32, L, lo, hi, MODEL_LEAK, (0.2, 0.8, 0.0),
                      dt=1e-4, n_steps=10, rtol=1e-10)
    if i == 2:
        lo, hi = _single(3, 0.3, 0.7)
        return Config("cfg2-3d-64-hh", 3, 64, L, lo, hi, MODEL_HH, (0.2, 0.8, 0.0),
                      dt=5e-5, n_steps=100, rtol=1e-10, stim_kind=STIM_WINDOW,
                      stim_gbar=40.0, stim_t0=0.0, stim_t1=1e-3, stim_xmax=0.4 * L)
    if i == 3:
        lo, hi = box_cells(5, 0.12, 0.04, 3)
        return Config("cfg3-3d-128-125cells-mixed", 3, 128, L, lo, hi, MODEL_HH, (0.2, 0.8, 0.0),
                      dt=5e-5, n_steps=100, rtol=1e-8, mixed=True, stim_kind=STIM_WINDOW,
                      stim_gbar=40.0, stim_t0=0.0, stim_t1=1e-3, stim_xmax=0.4 * L)
    if i == 4:
        lo, hi = box_cells(4, 0.15, 0.05, 2)
        return Config("cfg4-2d-256-16cells-adjoint", 2, 256, L, lo, hi, MODEL_LEAK, (0.2, 0.8, 0.0),
                      dt=1e-4, n_steps=200, rtol=1e-10, gK_sigma=0.2)
    if i == 5:
        rng = np.random.Generator(np.random.PCG64(0))
        lo, hi = box_cells(8, 0.08, 0.03, 3, jitter=(0.8, 1.2), rng=rng)
        return Config("cfg5-3d-256-512cells-mixed", 3, 256, L, lo, hi, MODEL_HH, (0.2, 0.8, 0.0),
                      dt=5e-5, n_steps=50, rtol=1e-8, mixed=True, stim_kind=STIM_WINDOW,
                      stim_gbar=40.0, stim_t0=0.0, stim_t1=1e-3, stim_xmax=0.4 * L)
    if i == 6:
        # Kir-Na/K membrane with a K bolus and Na removal in the extracellular half x < L/2 for
        # 0 < t <= 2 ms (Section 5.2's stimulus on a Model-A-shaped box; Table 2 leak values); the
        # window ends half a step after 2 ms so that the accumulated t_20 = 2 ms (+ rounding) is in
        lo, hi = _single(3, 0.3, 0.7)
        return Config("kir-3d-64-bolus", 3, 64, L, lo, hi, MODEL_KIR, (1.0, 4.0, 0.0),
                      dt=1e-4, n_steps=50, rtol=1e-10, source_e=(-1.0, 1.0, 0.0), source_xmax=0.5 * L,
                      source_t0=0.0, source_t1=2e-3 + 0.5e-4)
    if i == 7:
        lo, hi = _single(2, 0.25, 0.75)
        return Config("kir-2d-32-bolus", 2, 32, L, lo, hi, MODEL_KIR, (1.0, 4.0, 0.0),
                      dt=1e-4, n_steps=30, rtol=1e-10, source_e=(-1.0, 1.0, 0.0), source_xmax=0.5 * L,
                      source_t0=0.0, source_t1=2e-3 + 0.5e-4)
    if i == 8:
        # the 3D HH workload on a 32^3 grid whose intervals next to the cell faces are cut into 4
        # slabs (Section 6.4's interface-based refinement, here on a tensor grid): 44^3 grid boxes
        lo, hi = _single(3, 0.3, 0.7)
        return Config("hh-3d-32-interface-refined", 3, 32, L, lo, hi, MODEL_HH, (0.2, 0.8, 0.0),
                      dt=5e-5, n_steps=100, rtol=1e-10, stim_kind=STIM_WINDOW,
                      stim_gbar=40.0, stim_t0=0.0, stim_t1=1e-3, stim_xmax=0.4 * L, refine=(4, 1))
    raise ValueError(i)


def model_a(dim: int, nx: int, dt: float) -> Config:
    """The paper's Model A: [0,1]^d um, cell [0.25,0.75]^d, HH with Table 2 leak and the
    periodic exponential stimulus on the whole membrane (Section 5.1)."""
    lo, hi = _single(dim, 0.25, 0.75)
    p = table2()
    return Config(f"modelA-{dim}d-{nx}", dim, nx, 1e-6, lo, hi, MODEL_HH, p["g_leak"], dt=dt,
                  n_steps=1, rtol=1e-6, stim_kind=STIM_PERIODIC_EXP, stim_gbar=p["gbar_stim"],
                  stim_a=p["stim_a"], stim_tau=p["stim_tau"])


CONFIGS = {i: (lambda i=i: make_config(i)) for i in range(1, 9)}


def probe_points(cfg: Config, n: int = 64, seed: int = 2) -> np.ndarray:
    """n points uniform in the extracellular space (rejection against the snapped cell boxes),
    strictly inside the domain; PCG64(seed)."""
    m = cfg.mesh
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = []
    while len(pts) < n:
        p = rng.uniform(0.02, 0.98, size=cfg.dim)
        g = p * cfg.nx
        inside = np.any(np.all((g >= m.boxes[:, 0] - 1e-9) & (g <= m.boxes[:, 1] + 1e-9), axis=1))
        if not inside:
            pts.append(p * cfg.length)
    return np.array(pts)
