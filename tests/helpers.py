"""Shared test helpers: oracle runs and the comparisons used by the GPU parity tests."""
import numpy as np

from oracle import problem as oproblem, solve as osolve, step as ostep, system as osystem


def oracle_run(cfg, n_steps, exact="direct", degree=1):
    """Oracle states u_0..u_n. exact='direct' (sparse LU of A) or 'lu_p0' (GMRES with LU(P_0) to 1e-14);
    degree 1 (P1) or 2 (P2)."""
    pb, s0 = oproblem.from_config(cfg, degree=degree)
    kw = {}
    if exact == "lu_p0":
        kw = dict(method="gmres", M=osolve.lu_P0(osystem.preconditioner_P0(pb, s0)), rtol=1e-14)
    states = [s0]
    s = s0
    for _ in range(n_steps):
        s, _ = ostep.step(pb, s, **kw)
        states.append(s)
    return pb, states


def rel_errors(gpu_state, ref):
    """Relative l2 errors of the concentrations (all six vectors) and of phi = [phi_i; phi_e]."""
    cg = np.concatenate([gpu_state["c_i"].ravel(), gpu_state["c_e"].ravel()])
    cr = np.concatenate([ref.c_i.ravel(), ref.c_e.ravel()])
    pg = np.concatenate([gpu_state["phi_i"], gpu_state["phi_e"]])
    pr = np.concatenate([ref.phi_i, ref.phi_e])
    return np.linalg.norm(cg - cr) / np.linalg.norm(cr), np.linalg.norm(pg - pr) / np.linalg.norm(pr)


def block_bounds(pb):
    off_i, off_e, N = osystem.offsets(pb)
    return np.array(off_i + off_e + [N])


def blockscaled_entry_error(pb, A, vals):
    """max |gpu - oracle| over the pattern, relative to the largest entry of the same field block."""
    Acoo = A.tocoo()
    b = block_bounds(pb)
    rb = np.searchsorted(b, Acoo.row, side="right") - 1
    cb = np.searchsorted(b, Acoo.col, side="right") - 1
    key = rb * 16 + cb
    scale = np.zeros(256)
    np.maximum.at(scale, key, np.abs(Acoo.data))
    return float((np.abs(vals - Acoo.data) / scale[key]).max())


def blockwise_vector_error(pb, y, yr):
    b = block_bounds(pb)
    errs = []
    for a, c in zip(b[:-1], b[1:]):
        den = np.abs(yr[a:c]).max()
        errs.append(np.abs(y[a:c] - yr[a:c]).max() / den if den > 0 else np.abs(y[a:c]).max())
    return float(max(errs))


def paper_values():
    """Values printed in the paper, with their citations (tests/golden/paper_values.json)."""
    import json
    import os
    return json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
