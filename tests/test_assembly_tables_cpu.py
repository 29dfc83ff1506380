"""The assembly kernels' arithmetic on the library's own tables, on the CPU.

knp_problem_create with KNP_DRY_RUN_TABLES builds every host table a problem uploads (the
sliced-ELL pattern with its static mass and stiffness values, the incidences of the per-step
weighted stiffness, the membrane tables, the bulk source) and writes them to a file instead of
the GPU. Here the per-step assembly kernels (element values, edge sums, row pass, membrane pairs,
membrane right-hand side) and the operator kernel are replayed in numpy on those tables,
following the kernels' loops, from the oracle's membrane update; the operator product and the
right-hand side must equal the oracle's assembly of Eq. 4.3.

For P1 the kernels themselves are checked against the oracle on the GPU, so the P1 cases check
this replay. The P2 cases then check the P2 tables and the P2 kernels' arithmetic on the CPU
(Section 3.3 with p = 2), beside their GPU parity tests."""
import os

import numpy as np
import pytest

from helpers import blockwise_vector_error
from oracle import fem, membrane as omem, p2 as op2, problem as oproblem, system as osystem
from synth import make_config
from synth.configs import model_a


@pytest.fixture(scope="module")
def lib():
    from paper_2403_04491_gb300.build import build_library
    build_library()
    from paper_2403_04491_gb300 import knp
    return knp.load_library()


def dry_run_tables(cfg, degree, path):
    from paper_2403_04491_gb300 import KnpError, problem_from_config
    if os.path.exists(path):
        os.remove(path)
    os.environ["KNP_DRY_RUN_TABLES"] = str(path)
    try:
        with pytest.raises(KnpError) as ei:
            problem_from_config(cfg, degree=degree)
    finally:
        del os.environ["KNP_DRY_RUN_TABLES"]
    assert ei.value.code == 7 and "dry run" in str(ei.value)
    types = {1: np.uint8, 4: np.int32}
    out = {}
    with open(path, "rb") as f:
        while True:
            head = f.read(24)
            if not head:
                break
            ln, cnt, sz = np.frombuffer(head, np.int64)
            name = f.read(int(ln)).decode()
            dt = np.float64 if name in ("sell_m", "sell_a", "el_g", "ecoef", "f_area", "f_gleak", "src") else \
                (np.int64 if sz == 8 else types[int(sz)])
            out[name] = np.frombuffer(f.read(int(cnt * sz)), dt)
    return out


def replay(pb, s0, mfo, T):
    """The assembly and operator kernels on the dumped tables; returns (A x, f, x) node-major."""
    degree, dim, Ni, Ne, pin, nmv, ne = (int(v) for v in T["info"])
    n, K = Ni + Ne, 3
    m = dim - 1
    if degree == 1:
        npe, nfn, bits = dim + 1, dim, 2
        Wt, Mf = fem.local_triple(m), fem.local_mass(m)
    else:
        npe, nfn, bits = (dim + 1) * (dim + 2) // 2, dim * (dim + 1) // 2, 3
        Wt, Mf = op2.local_triple(m), op2.local_mass(m)
    u = np.zeros((n, 4))
    u[:Ni, :3], u[:Ni, 3] = s0.c_i.T, s0.phi_i
    u[Ni:, :3], u[Ni:, 3] = s0.c_e.T, s0.phi_e
    # the membrane fields as the node kernel lays them out (rows 0..13), from the oracle's update
    mf = np.zeros((14, nmv))
    drive = mfo["phi_M"][None] - mfo["E"]
    n_g, m_g, h_g = mfo["w"]
    mf[0], mf[1:4], mf[4:7], mf[7:10] = mfo["phi_M"], mfo["C_i"], mfo["C_e"], drive
    mf[10], mf[11] = m_g ** 3 * h_g * drive[0], n_g ** 4 * drive[1]
    mf[12] = drive[1] * omem.kir_factor(mfo["c_e"][1], drive[1], mfo["phi_M"], pb.E_K0, pb.cKe0)
    mf[13] = omem.pump_flux(mfo["c_i"][0], mfo["c_e"][1], pb.rho_pump, pb.P_Na, pb.P_K)
    # element values: P1 element means of c; P2 the off-diagonal pair values of each element
    eln = T["el_nodes"].reshape(ne, npe)
    if degree == 1:
        V = np.stack([u[eln, k].mean(axis=1) for k in range(K)])
    else:
        G = T["el_g"].reshape(ne, 4, 4)[:, :dim + 1, :dim + 1]
        pairs = [(j, l) for j in range(npe) for l in range(j + 1, npe)]
        S = op2.local_weighted(dim)
        V = []
        for k in range(K):
            full = np.einsum("nc,cjlab,nab->njl", u[eln, k], S, G, optimize=True)
            V.append(np.stack([full[:, j, l] for j, l in pairs], axis=1).ravel())
        V = np.stack(V)
    # edge sums
    eptr, einc, ecoef = T["eptr"], T["einc"], T["ecoef"]
    n_edges = len(eptr) - 1
    owner = np.repeat(np.arange(n_edges), np.diff(eptr))
    ak = np.stack([np.bincount(owner, weights=V[k][einc] * ecoef, minlength=n_edges) for k in range(K)])
    # row pass over the sliced-ELL layout
    sp, col, edge, msv, asv = T["slice_ptr"], T["col"], T["sell_edge"], T["sell_m"], T["sell_a"]
    row = np.empty(len(col), np.int64)
    for s in range(len(sp) - 1):
        w = (sp[s + 1] - sp[s]) // 32
        row[sp[s]:sp[s + 1]] = s * 32 + np.tile(np.arange(32), w)
    live = edge != -2
    reg = (row >= Ni).astype(int)
    taut = np.stack([pb.dt * pb.D_i * pb.z / pb.psi, pb.dt * pb.D_e * pb.z / pb.psi])
    tau = np.stack([pb.dt * pb.D_i, pb.dt * pb.D_e])
    e = np.zeros((K, len(col)))
    off = live & (edge >= 0)
    for k in range(K):
        e[k, off] = taut[reg[off], k] * ak[k, edge[off]]
        rs = np.bincount(row[off], weights=e[k, off], minlength=n)
        diag = live & (edge == -1)
        e[k, diag] = -rs[row[diag]]
    f = np.zeros((n, 4))
    t_n = s0.t + pb.dt
    src = T["src"].reshape(n, 4) if len(T["src"]) and pb.source_t0 < t_n <= pb.source_t1 else None
    for k in range(K):
        f[:, k] = np.bincount(row[live], weights=msv[live] * u[col[live], k], minlength=n)
        if src is not None:
            f[:, k] += pb.dt * np.bincount(row[live], weights=msv[live] * src[col[live], k], minlength=n)
    # membrane pairs
    area, fmv = T["f_area"], T["f_mv"].reshape(-1, nfn)
    mp_ptr, mpf, tgt = T["mp_ptr"], T["mpf"].astype(np.int64), T["mp_tgt"].reshape(-1, 4)
    xcol = T["xcol"]
    xe = np.zeros((K, len(xcol)))
    pair = np.repeat(np.arange(len(mp_ptr) - 1), np.diff(mp_ptr))
    fa, sa, sb = mpf >> (2 * bits), (mpf >> bits) & ((1 << bits) - 1), mpf & ((1 << bits) - 1)
    for k in range(K):
        vi = sum(np.bincount(pair, weights=area[fa] * Wt[c, sa, sb] * mf[1 + k, fmv[fa, c]], minlength=len(tgt))
                 for c in range(nfn))
        ve = sum(np.bincount(pair, weights=area[fa] * Wt[c, sa, sb] * mf[4 + k, fmv[fa, c]], minlength=len(tgt))
                 for c in range(nfn))
        np.add.at(e[k], tgt[:, 0], vi)
        np.add.at(e[k], tgt[:, 1], ve)
        xe[k, tgt[:, 2]] = -vi
        xe[k, tgt[:, 3]] = -ve
    # membrane right-hand side
    mvf_ptr, mvf = T["mvf_ptr"], T["mvf"].astype(np.int64)
    node = np.repeat(np.arange(nmv), np.diff(mvf_ptr))
    fid, slot = mvf >> bits, mvf & ((1 << bits) - 1)
    fmodel, fgl, fmask = T["f_model"], T["f_gleak"].reshape(-1, 3), T["f_mask"]
    g_stim = omem.stimulus_conductance(pb.stim_kind, pb.stim_gbar, s0.t, pb.stim_t0, pb.stim_t1, pb.stim_a,
                                       pb.stim_tau)
    intI = np.zeros((K, nmv))
    intPhi = np.zeros(nmv)
    cpi = np.zeros((K, nmv))
    cpe = np.zeros((K, nmv))
    hh, kir = fmodel[fid] == 1, fmodel[fid] == 2
    gst = np.where(fmask[fid] != 0, g_stim, 0.0)
    for c in range(nfn):
        mc = fmv[fid, c]
        Mcs = area[fid] * Mf[c, slot]
        I = fgl[fid].T * mf[7:10, mc]
        I[0] += gst * mf[7, mc]
        I[0] += np.where(hh, pb.gbar_Na * mf[10, mc], 0.0)
        I[1] += np.where(hh, pb.gbar_K * mf[11, mc], 0.0)
        j = mf[13, mc]
        I[1] = np.where(kir, fgl[fid, 1] * mf[12, mc] - 2.0 * pb.F * pb.z[1] * j, I[1])
        I[0] = np.where(kir, I[0] + 3.0 * pb.F * pb.z[0] * j, I[0])
        for k in range(K):
            intI[k] += np.bincount(node, weights=Mcs * I[k], minlength=nmv)
        intPhi += np.bincount(node, weights=Mcs * mf[0, mc], minlength=nmv)
        for b in range(nfn):
            W = area[fid] * Wt[c, b, slot] * mf[0, fmv[fid, b]]
            for k in range(K):
                cpi[k] += np.bincount(node, weights=W * mf[1 + k, mc], minlength=nmv)
                cpe[k] += np.bincount(node, weights=W * mf[4 + k, mc], minlength=nmv)
    mvg = T["mv_g"].reshape(2, nmv)
    jk = pb.dt * intI / (pb.F * pb.z[:, None])
    np.add.at(f[:, :3], mvg[0], -(jk - cpi).T)
    np.add.at(f[:, :3], mvg[1], (jk - cpe).T)
    hphi = (pb.dt * intI.sum(axis=0) - pb.Cm * intPhi) / pb.F
    np.add.at(f[:, 3], mvg[0], -hphi)
    keep = mvg[1] != pin
    np.add.at(f[:, 3], mvg[1][keep], hphi[keep])
    # the operator's node blocks built from the stored m, a, e (the form the transposed product
    # uses; the forward product folds m + tau a per ion) on a random x
    x = np.random.default_rng(3).standard_normal((n, 4))
    phi = np.where(np.arange(n) == pin, 0.0, x[:, 3])
    y = np.zeros((n, 4))
    aa = np.zeros((K, n))
    for k in range(K):
        am = np.bincount(row[live], weights=msv[live] * x[col[live], k], minlength=n)
        aa[k] = np.bincount(row[live], weights=asv[live] * x[col[live], k], minlength=n)
        ae = np.bincount(row[live], weights=e[k, live] * phi[col[live]], minlength=n)
        xrow = np.repeat(np.arange(n), np.diff(T["xptr"]))
        ae += np.bincount(xrow, weights=xe[k] * phi[xcol], minlength=n)
        ta = tau[(np.arange(n) >= Ni).astype(int), k] * aa[k]
        y[:, k] = am + ta + ae
        y[:, 3] += pb.z[k] * (ta + ae)
    y[pin, 3] = x[pin, 3]
    return y, f, x


def _eq43(v, Ni):
    return np.concatenate([v[:Ni, :3].T.ravel(), v[:Ni, 3], v[Ni:, :3].T.ravel(), v[Ni:, 3]])


CASES = {
    "modelA-2d-8": lambda: model_a(2, 8, 1e-4),
    "leak-2d-16": lambda: make_config(1).with_nx(16),
    "kir-source-2d-16": lambda: make_config(7).with_nx(16),
    "modelA-3d-4": lambda: model_a(3, 4, 1e-4),
    "16cells-2d-32": lambda: make_config(4).with_nx(32),
    "iref-3d-8": lambda: make_config(8).with_nx(8),
}


@pytest.mark.parametrize("degree", [1, 2], ids=["P1", "P2"])
@pytest.mark.parametrize("name", list(CASES))
def test_assembly_replay_on_library_tables(lib, tmp_path, name, degree):
    cfg = CASES[name]()
    T = dry_run_tables(cfg, degree, tmp_path / "tables.bin")
    pb, s0 = oproblem.from_config(cfg, degree=degree)
    A, f_ref, mfo = osystem.assemble(pb, s0)
    assert int(T["info"][2]) == pb.topo.N_i and int(T["info"][3]) == pb.topo.N_e
    y, f, x = replay(pb, s0, mfo, T)
    Ni = pb.topo.N_i
    assert blockwise_vector_error(pb, _eq43(y, Ni), A @ _eq43(x, Ni)) < 1e-12
    assert blockwise_vector_error(pb, _eq43(f, Ni), f_ref) < 1e-12
