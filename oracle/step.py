"""The time loop of Section 3.2: for n = 1..N_t, membrane update, assembly of A_{n-1} and f_n,
and the solve of Eq. 4.3 (exact, or GMRES with x0 = u_{n-1})."""
from __future__ import annotations

import numpy as np

from . import solve, system


def step(pb: system.Problem, s: system.State, method="direct", M=None, rtol=1e-12, source=None):
    A, f, mf = system.assemble(pb, s, source=source)
    info = {}
    if method == "direct":
        u = solve.direct(A, f)
    else:
        u, its, ok, hist = solve.gmres(A, f, x0=system.pack(pb, s), M=M, rtol=rtol)
        info = dict(iterations=its, converged=ok, history=hist)
    ns = system.unpack(pb, u, s)
    ns.w = mf["w"]
    ns.t = s.t + pb.dt
    return ns, info


def run(pb, s0, n_steps, **kw):
    states = [s0]
    s = s0
    for _ in range(n_steps):
        s, _ = step(pb, s, **kw)
        states.append(s)
    return states
