"""ctypes binding of include/knp.h (argument marshalling only).

The names follow the C functions: ``Mesh`` wraps knp_mesh_*, ``Problem`` wraps
knp_problem_*, knp_assemble_step, knp_amg_setup, knp_solve, knp_step and the state and
inspection calls. Loading fails loudly if libknp.so is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libknp.so")

KNP_OK = 0
STATUS = {0: "KNP_OK", 1: "KNP_ERR_INVALID_ARG", 2: "KNP_ERR_INVALID_MESH", 3: "KNP_ERR_OOM", 4: "KNP_ERR_CUDA",
          5: "KNP_ERR_NOT_CONVERGED", 6: "KNP_ERR_NUMERIC", 7: "KNP_ERR_STATE"}
KNP_HOST, KNP_DEVICE = 0, 1
KNP_PREC_FP64, KNP_PREC_FP32 = 0, 1
KNP_TEST_SCALED, KNP_TEST_PAPER = 0, 1
MAX_IONS = 4

_lib = None


class KnpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class MeshDesc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_vertices", C.c_int64), ("coords", C.POINTER(C.c_double)),
                ("n_elems", C.c_int64), ("elems", C.POINTER(C.c_int32)), ("elem_tag", C.POINTER(C.c_int32)),
                ("pin_point", C.POINTER(C.c_double))]


class P2Info(C.Structure):
    _fields_ = [("n_edges", C.c_int64), ("n_nodes", C.c_int64), ("N_i", C.c_int64), ("N_e", C.c_int64),
                ("n_membrane_nodes", C.c_int64), ("pin_node", C.c_int64), ("n_dof", C.c_int64)]


class MeshInfo(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_vertices", C.c_int64), ("n_elems", C.c_int64), ("N_i", C.c_int64),
                ("N_e", C.c_int64), ("n_facets", C.c_int64), ("n_membrane_vertices", C.c_int64),
                ("n_cells", C.c_int32), ("pin_vertex", C.c_int64), ("n_dof", C.c_int64)]


D4 = C.c_double * MAX_IONS


class ProblemDesc(C.Structure):
    _fields_ = [("n_ions", C.c_int32), ("z", D4), ("D_i", D4), ("D_e", D4), ("R", C.c_double), ("T", C.c_double),
                ("F", C.c_double), ("Cm", C.c_double), ("dt", C.c_double), ("c_i0", D4), ("c_e0", D4),
                ("phi_M0", C.c_double), ("facet_model", C.POINTER(C.c_int32)),
                ("facet_gleak", C.POINTER(C.c_double)), ("ion_na", C.c_int32), ("ion_k", C.c_int32),
                ("gbar_na", C.c_double), ("gbar_k", C.c_double), ("phi_rest", C.c_double),
                ("w0", C.c_double * 3), ("n_ode", C.c_int32), ("stim_kind", C.c_int32),
                ("stim_gbar", C.c_double), ("stim_t0", C.c_double), ("stim_t1", C.c_double),
                ("stim_a", C.c_double), ("stim_tau", C.c_double), ("stim_mask", C.POINTER(C.c_uint8)),
                ("rho_pump", C.c_double), ("P_na", C.c_double), ("P_k", C.c_double),
                ("source_i", C.POINTER(C.c_double)), ("source_e", C.POINTER(C.c_double)),
                ("source_t0", C.c_double), ("source_t1", C.c_double), ("degree", C.c_int32)]


class AmgOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("theta", C.c_double), ("coarse_max", C.c_int32),
                ("max_levels", C.c_int32), ("cheb_degree", C.c_int32), ("cheb_ratio", C.c_double),
                ("theta_coarse", C.c_double), ("p_drop", C.c_double), ("host_setup", C.c_int32),
                ("inner_cg_max_it", C.c_int32), ("inner_cg_rtol", C.c_double), ("cheb_degree_pre", C.c_int32)]


class AmgSetupRecord(C.Structure):
    _fields_ = [("on_gpu", C.c_int32), ("long_rows_p", C.c_int64), ("long_rows_rap", C.c_int64),
                ("setup_ms", C.c_double)]


class SolveOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("restart", C.c_int32), ("max_it", C.c_int32), ("phi_e_group", C.c_int32),
                ("deflate", C.c_int32), ("stop_test", C.c_int32), ("phi_e_floor", C.c_double),
                ("x0_extrapolate", C.c_int32)]


class SolveStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("restarts", C.c_int32), ("true_relres", C.c_double), ("ms", C.c_double),
                ("inner_iterations", C.c_int64)]


class ProblemInfo(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("nnz_region", C.c_int64), ("nnz_padded", C.c_int64),
                ("nnz_cross", C.c_int64), ("n_membrane_pairs", C.c_int64), ("n_edges", C.c_int64),
                ("edge_incidences", C.c_int64), ("step_index", C.c_int64)]


class StepStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("true_relres", C.c_double)]


_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int32)
_LP = C.POINTER(C.c_int64)

SIGNATURES = {
    "knp_mesh_create": [C.POINTER(MeshDesc), C.POINTER(C.c_void_p)],
    "knp_mesh_get_info": [C.c_void_p, C.POINTER(MeshInfo)],
    "knp_mesh_nodes": [C.c_void_p, _IP, _IP],
    "knp_mesh_facets": [C.c_void_p, _IP, _IP, _IP, _IP],
    "knp_mesh_destroy": [C.c_void_p],
    "knp_mesh_p2_get_info": [C.c_void_p, C.POINTER(P2Info)],
    "knp_mesh_p2_tables": [C.c_void_p, _IP, _IP, _IP, _IP, _IP, _IP, _IP],
    "knp_mesh_p2_region_matrices": [C.c_void_p, C.c_int32, _DP, _LP, _IP, _IP, _DP, _DP, _DP],
    "knp_problem_create": [C.c_void_p, C.POINTER(ProblemDesc), C.c_void_p, C.POINTER(C.c_void_p)],
    "knp_problem_destroy": [C.c_void_p],
    "knp_sync": [C.c_void_p],
    "knp_assemble_step": [C.c_void_p],
    "knp_amg_setup": [C.c_void_p, C.POINTER(AmgOpts)],
    "knp_solve": [C.c_void_p, C.POINTER(SolveOpts), C.POINTER(SolveStats)],
    "knp_step": [C.c_void_p, C.c_int32, C.POINTER(SolveOpts), C.POINTER(StepStats)],
    "knp_state_get": [C.c_void_p, C.c_int32, _DP, _DP, _DP, _DP, _DP, _DP],
    "knp_state_set": [C.c_void_p, C.c_int32, _DP, _DP, _DP, _DP, _DP, C.c_double],
    "knp_rhs_get": [C.c_void_p, _DP],
    "knp_apply_operator": [C.c_void_p, _DP, _DP],
    "knp_operator_entries": [C.c_void_p, C.c_int64, _LP, _LP, _DP],
    "knp_apply_preconditioner": [C.c_void_p, _DP, _DP],
    "knp_apply_deflated_preconditioner": [C.c_void_p, _DP, _DP, C.c_int32],
    "knp_apply_preconditioner_noalloc": [C.c_void_p, C.c_void_p, C.c_void_p],
    "knp_amg_info": [C.c_void_p, _IP, _LP, _LP, _DP],
    "knp_amg_setup_info": [C.c_void_p, C.c_void_p],
    "knp_problem_get_info": [C.c_void_p, C.c_void_p],
    "knp_problem_set_facet_gleak": [C.c_void_p, C.c_int32, C.c_void_p],
    "knp_adjoint_begin": [C.c_void_p],
    "knp_adjoint_step": [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.POINTER(SolveOpts), C.POINTER(SolveStats)],
    "knp_adjoint_get": [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "knp_apply_operator_transpose": [C.c_void_p, _DP, _DP],
    "knp_profile_begin": [C.c_void_p, C.c_int32],
    "knp_profile_end": [C.c_void_p, _LP, _DP],
    "knp_launch_count": [_LP],
    "knp_last_error": [],
}
VOID_FUNCS = {"knp_mesh_destroy", "knp_problem_destroy"}


def load_library(path: str = LIB_PATH):
    """Loads libknp.so (built by ``__graft_entry__.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libknp.so not found at {path}: build it with __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        if name == "knp_last_error":
            fn.restype = C.c_char_p
        elif name in VOID_FUNCS:
            fn.restype = None
        else:
            fn.restype = C.c_int32
    _lib = lib
    return lib


def _check(code):
    if code != KNP_OK:
        raise KnpError(code, _lib.knp_last_error().decode())


def _dptr(a):
    return None if a is None else a.ctypes.data_as(_DP)


def _iptr(a):
    return None if a is None else a.ctypes.data_as(_IP)


def _lptr(a):
    return None if a is None else a.ctypes.data_as(_LP)


class Mesh:
    """knp_mesh_create: conforming simplicial mesh with cell tags (0 = extracellular)."""

    def __init__(self, coords, elems, tag, pin_point=None):
        """pin_point: the phi_e pin goes on the extracellular vertex nearest to it (default: origin)."""
        lib = load_library()
        self._coords = np.ascontiguousarray(coords, dtype=np.float64)
        self._elems = np.ascontiguousarray(elems, dtype=np.int32)
        self._tag = np.ascontiguousarray(tag, dtype=np.int32)
        self._pin = None if pin_point is None else np.ascontiguousarray(pin_point, dtype=np.float64)
        d = MeshDesc(self._coords.shape[1], self._coords.shape[0], _dptr(self._coords), self._elems.shape[0],
                     _iptr(self._elems), _iptr(self._tag), None if self._pin is None else _dptr(self._pin))
        h = C.c_void_p()
        _check(lib.knp_mesh_create(C.byref(d), C.byref(h)))
        self.handle = h
        info = MeshInfo()
        _check(lib.knp_mesh_get_info(h, C.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in MeshInfo._fields_}

    def nodes(self):
        ni = np.empty(self.info["N_i"], np.int32)
        ne = np.empty(self.info["N_e"], np.int32)
        _check(_lib.knp_mesh_nodes(self.handle, _iptr(ni), _iptr(ne)))
        return ni, ne

    def facets(self):
        nf, dim = self.info["n_facets"], self.info["dim"]
        v = np.empty((nf, dim), np.int32)
        e = np.empty(nf, np.int32)
        o = np.empty(nf, np.int32)
        c = np.empty(nf, np.int32)
        _check(_lib.knp_mesh_facets(self.handle, _iptr(v), _iptr(e), _iptr(o), _iptr(c)))
        return v, e, o, c

    def p2(self):
        """P2 nodes (knp_mesh_p2_get_info / knp_mesh_p2_tables): a dict of the info fields and tables."""
        info = P2Info()
        _check(_lib.knp_mesh_p2_get_info(self.handle, C.byref(info)))
        out = {f: getattr(info, f) for f, _ in P2Info._fields_}
        d, ne, nf = self.info["dim"], self.info["n_elems"], self.info["n_facets"]
        t = dict(edges=np.empty((out["n_edges"], 2), np.int32),
                 elem_nodes=np.empty((ne, (d + 1) * (d + 2) // 2), np.int32),
                 facet_nodes=np.empty((nf, d * (d + 1) // 2), np.int32),
                 nodes_i=np.empty(out["N_i"], np.int32), nodes_e=np.empty(out["N_e"], np.int32),
                 membrane_nodes=np.empty(out["n_membrane_nodes"], np.int32),
                 node_cell_i=np.empty(out["N_i"], np.int32))
        _check(_lib.knp_mesh_p2_tables(self.handle, *(_iptr(t[k]) for k in
                                                      ("edges", "elem_nodes", "facet_nodes", "nodes_i", "nodes_e",
                                                       "membrane_nodes", "node_cell_i"))))
        out.update(t)
        return out

    def p2_region_matrices(self, region, c=None):
        """knp_mesh_p2_region_matrices: the P2 M_r, A_r (and A_r^{c} for nodal c on the region's P2
        nodes) of region 0 (i) or 1 (e) as scipy CSR matrices."""
        import scipy.sparse as sp
        cnt = C.c_int64()
        cc = None if c is None else np.ascontiguousarray(c, dtype=np.float64)
        _check(_lib.knp_mesh_p2_region_matrices(self.handle, int(region), _dptr(cc), C.byref(cnt), None, None, None,
                                                None, None))
        r = np.empty(cnt.value, np.int32)
        col = np.empty(cnt.value, np.int32)
        M, A = np.empty(cnt.value), np.empty(cnt.value)
        Ac = None if cc is None else np.empty(cnt.value)
        _check(_lib.knp_mesh_p2_region_matrices(self.handle, int(region), _dptr(cc), C.byref(cnt), _iptr(r),
                                                _iptr(col), _dptr(M), _dptr(A), _dptr(Ac)))
        n = self.p2()["N_i" if region == 0 else "N_e"]
        mk = lambda v: sp.coo_matrix((v, (r, col)), shape=(n, n)).tocsr()
        return (mk(M), mk(A)) if Ac is None else (mk(M), mk(A), mk(Ac))

    def close(self):
        if getattr(self, "handle", None):
            _lib.knp_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count():
    n = C.c_int64()
    _check(load_library().knp_launch_count(C.byref(n)))
    return n.value


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


class Problem:
    """knp_problem_create and the per-step calls on it."""

    def __init__(self, mesh: Mesh, desc: dict, stream=None):
        lib = load_library()
        self.mesh = mesh
        nf = mesh.info["n_facets"]
        n_ions = int(desc["n_ions"])
        self._facet_model = np.ascontiguousarray(desc["facet_model"], dtype=np.int32).reshape(nf)
        self._facet_gleak = np.ascontiguousarray(desc["facet_gleak"], dtype=np.float64).reshape(nf, n_ions)
        mask = desc.get("stim_mask")
        self._mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8).reshape(nf)
        d = ProblemDesc()
        d.n_ions = n_ions
        for key in ("z", "D_i", "D_e", "c_i0", "c_e0"):
            arr = getattr(d, key)
            for k, v in enumerate(desc[key]):
                arr[k] = float(v)
        for key in ("R", "T", "F", "Cm", "dt", "phi_M0", "gbar_na", "gbar_k", "phi_rest", "stim_gbar", "stim_t0",
                    "stim_t1", "stim_a", "stim_tau", "source_t0", "source_t1"):
            setattr(d, key, float(desc.get(key, 0.0)))
        # Kir-Na/K pump constants (Table 2 values unless given)
        d.rho_pump = float(desc.get("rho_pump", 1.115e-6))
        d.P_na = float(desc.get("P_na", 10.0))
        d.P_k = float(desc.get("P_k", 1.5))
        # polynomial degree (1: P1, 2: P2 on the nodes of Mesh.p2())
        self.degree = int(desc.get("degree", 1))
        d.degree = self.degree
        p2 = mesh.p2() if self.degree == 2 else None
        # bulk source per vertex (P1) or per global P2 node (P2), [n][n_ions], for the i and e copies
        nv = mesh.info["n_vertices"] if p2 is None else p2["n_nodes"]
        self._source = {}
        for key in ("source_i", "source_e"):
            v = desc.get(key)
            if v is not None:
                self._source[key] = np.ascontiguousarray(v, dtype=np.float64).reshape(nv, n_ions)
                setattr(d, key, _dptr(self._source[key]))
        for k, v in enumerate(desc["w0"]):
            d.w0[k] = float(v)
        d.ion_na = int(desc.get("ion_na", 0))
        d.ion_k = int(desc.get("ion_k", 1))
        d.n_ode = int(desc.get("n_ode", 25))
        d.stim_kind = int(desc.get("stim_kind", 0))
        d.facet_model = _iptr(self._facet_model)
        d.facet_gleak = _dptr(self._facet_gleak)
        d.stim_mask = None if self._mask is None else self._mask.ctypes.data_as(C.POINTER(C.c_uint8))
        if stream is None:
            stream = _current_stream()
        self.stream = stream
        h = C.c_void_p()
        _check(lib.knp_problem_create(mesh.handle, C.byref(d), C.c_void_p(stream) if stream else None, C.byref(h)))
        self.handle = h
        self.n_ions = n_ions
        if p2 is None:
            self.N_i, self.N_e = mesh.info["N_i"], mesh.info["N_e"]
            self.n_mv = mesh.info["n_membrane_vertices"]
        else:
            self.N_i, self.N_e = p2["N_i"], p2["N_e"]
            self.n_mv = p2["n_membrane_nodes"]
        self.n_dof = 4 * (self.N_i + self.N_e)

    def sync(self):
        """Wait for the work enqueued for this problem on its stream."""
        _check(_lib.knp_sync(self.handle))

    # -- per step
    def assemble_step(self):
        _check(_lib.knp_assemble_step(self.handle))

    def amg_setup(self, precision=KNP_PREC_FP64, theta=0.08, coarse_max=500, max_levels=12, cheb_degree=2,
                  cheb_ratio=3.0, theta_coarse=0.0, p_drop=0.0, host_setup=False, inner_cg_max_it=0,
                  inner_cg_rtol=1e-8, cheb_degree_pre=1):
        """inner_cg_max_it > 0 selects CG(P_0) (V-cycle-preconditioned CG per field block of P_0,
        to inner_cg_rtol) instead of one V-cycle. cheb_degree / cheb_degree_pre: Chebyshev steps
        after / before the coarse-grid correction."""
        o = AmgOpts(precision, theta, coarse_max, max_levels, cheb_degree, cheb_ratio, theta_coarse, p_drop,
                    int(host_setup), int(inner_cg_max_it), float(inner_cg_rtol), int(cheb_degree_pre))
        _check(_lib.knp_amg_setup(self.handle, C.byref(o)))

    def solve(self, rtol=1e-10, restart=30, max_it=1000, phi_e_group=False, deflate=True, stop_test=KNP_TEST_SCALED,
              phi_e_floor=0.0, x0_extrapolate=False):
        """deflate: the coarse correction of the potentials' near-null modes around P_0^{-1};
        stop_test: KNP_TEST_SCALED (per-group scaled test) or KNP_TEST_PAPER (Section 6.2's);
        x0_extrapolate: x_0 = 2 u_{n-1} - u_{n-2} after a previous extrapolating solve."""
        o = SolveOpts(rtol, restart, max_it, int(phi_e_group), int(deflate), int(stop_test), float(phi_e_floor),
                      int(x0_extrapolate))
        s = SolveStats()
        _check(_lib.knp_solve(self.handle, C.byref(o), C.byref(s)))
        return {"iterations": s.iterations, "restarts": s.restarts, "true_relres": s.true_relres, "ms": s.ms,
                "inner_iterations": s.inner_iterations}

    def step(self, nsteps=1, rtol=1e-10, restart=30, max_it=1000, phi_e_group=False, deflate=True,
             stop_test=KNP_TEST_SCALED, phi_e_floor=0.0, x0_extrapolate=False):
        o = SolveOpts(rtol, restart, max_it, int(phi_e_group), int(deflate), int(stop_test), float(phi_e_floor),
                      int(x0_extrapolate))
        st = (StepStats * max(nsteps, 1))()
        _check(_lib.knp_step(self.handle, nsteps, C.byref(o), st))
        return [{"iterations": st[i].iterations, "true_relres": st[i].true_relres} for i in range(nsteps)]

    # -- state
    def state_get(self):
        c_i = np.empty((self.n_ions, self.N_i))
        p_i = np.empty(self.N_i)
        c_e = np.empty((self.n_ions, self.N_e))
        p_e = np.empty(self.N_e)
        w = np.empty((3, self.n_mv))
        t = C.c_double()
        _check(_lib.knp_state_get(self.handle, KNP_HOST, _dptr(c_i), _dptr(p_i), _dptr(c_e), _dptr(p_e),
                                  _dptr(w) if self.n_mv else None, C.byref(t)))
        return dict(c_i=c_i, phi_i=p_i, c_e=c_e, phi_e=p_e, w=w, t=t.value)

    def state_get_device(self, c_i, phi_i, c_e, phi_e):
        """Device-to-device state copy into caller buffers (torch tensors or raw pointers)."""
        ptr = lambda a: None if a is None else C.cast(C.c_void_p(a if isinstance(a, int) else a.data_ptr()), _DP)
        t = C.c_double()
        _check(_lib.knp_state_get(self.handle, KNP_DEVICE, ptr(c_i), ptr(phi_i), ptr(c_e), ptr(phi_e), None,
                                  C.byref(t)))

    def state_set(self, c_i=None, phi_i=None, c_e=None, phi_e=None, w=None, t=0.0):
        conv = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
        c_i, phi_i, c_e, phi_e, w = map(conv, (c_i, phi_i, c_e, phi_e, w))
        _check(_lib.knp_state_set(self.handle, KNP_HOST, _dptr(c_i), _dptr(phi_i), _dptr(c_e), _dptr(phi_e),
                                  _dptr(w), float(t)))

    # -- inspection
    def rhs_get(self):
        f = np.empty(self.n_dof)
        _check(_lib.knp_rhs_get(self.handle, _dptr(f)))
        return f

    def apply_operator(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.n_dof)
        _check(_lib.knp_apply_operator(self.handle, _dptr(x), _dptr(y)))
        return y

    def apply_operator_transpose(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.n_dof)
        _check(_lib.knp_apply_operator_transpose(self.handle, _dptr(x), _dptr(y)))
        return y

    def set_facet_gleak(self, gleak):
        """knp_problem_set_facet_gleak from a numpy array or a CUDA tensor [n_facets, n_ions]."""
        if hasattr(gleak, "data_ptr") and getattr(gleak, "is_cuda", False):
            _check(_lib.knp_problem_set_facet_gleak(self.handle, KNP_DEVICE, C.c_void_p(gleak.data_ptr())))
        else:
            g = np.ascontiguousarray(gleak, dtype=np.float64)
            _check(_lib.knp_problem_set_facet_gleak(self.handle, KNP_HOST, g.ctypes.data_as(C.c_void_p)))

    # -- adjoint
    def adjoint_begin(self):
        _check(_lib.knp_adjoint_begin(self.handle))

    def adjoint_step(self, u_n, dLdu_n, rtol=1e-10, restart=30, max_it=1000, phi_e_group=True, phi_e_floor=0.0,
                     deflate=True):
        """u_n, dLdu_n in the Eq. 4.3 order: numpy arrays (host) or CUDA tensors (device)."""
        o = SolveOpts(rtol, restart, max_it, int(phi_e_group), int(deflate), KNP_TEST_SCALED, float(phi_e_floor), 0)
        s = SolveStats()
        if hasattr(u_n, "data_ptr"):
            _check(_lib.knp_adjoint_step(self.handle, KNP_DEVICE, C.c_void_p(u_n.data_ptr()),
                                         C.c_void_p(dLdu_n.data_ptr()), C.byref(o), C.byref(s)))
        else:
            a = np.ascontiguousarray(u_n, dtype=np.float64)
            b = np.ascontiguousarray(dLdu_n, dtype=np.float64)
            _check(_lib.knp_adjoint_step(self.handle, KNP_HOST, a.ctypes.data_as(C.c_void_p),
                                         b.ctypes.data_as(C.c_void_p), C.byref(o), C.byref(s)))
        return {"iterations": s.iterations, "true_relres": s.true_relres}

    def adjoint_get(self):
        du = np.empty(self.n_dof)
        dw = np.empty((3, max(self.n_mv, 1)))
        nf = self.mesh.info["n_facets"]
        gg = np.empty((max(nf, 1), self.n_ions))
        lam = np.empty(self.n_dof)
        _check(_lib.knp_adjoint_get(self.handle, KNP_HOST, du.ctypes.data_as(C.c_void_p), dw.ctypes.data_as(C.c_void_p),
                                    gg.ctypes.data_as(C.c_void_p), lam.ctypes.data_as(C.c_void_p)))
        return {"dLdu0": du, "dLdw0": dw[:, :self.n_mv], "grad_gleak": gg[:nf], "lambda": lam}

    def operator_entries(self, rows, cols):
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        cols = np.ascontiguousarray(cols, dtype=np.int64)
        v = np.empty(len(rows))
        _check(_lib.knp_operator_entries(self.handle, len(rows), _lptr(rows), _lptr(cols), _dptr(v)))
        return v

    def apply_preconditioner(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.empty(self.n_dof)
        _check(_lib.knp_apply_preconditioner(self.handle, _dptr(r), _dptr(z)))
        return z

    def apply_deflated_preconditioner(self, r, transpose=False):
        """M_D^{-1} r (knp_apply_deflated_preconditioner), host arrays in the Eq. 4.3 order; the
        adjoint solve's form (A^T, E^T) with transpose."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.empty(self.n_dof)
        _check(_lib.knp_apply_deflated_preconditioner(self.handle, _dptr(r), _dptr(z), int(bool(transpose))))
        return z

    def apply_preconditioner_noalloc(self, r_dev, z_dev):
        """knp_apply_preconditioner_noalloc on device buffers (torch tensors or raw pointers) in the
        same Eq. 4.3 order; allocates nothing (work vectors in the library's static device array)."""
        ptr = lambda a: C.c_void_p(a if isinstance(a, int) else a.data_ptr())
        _check(_lib.knp_apply_preconditioner_noalloc(self.handle, ptr(r_dev), ptr(z_dev)))

    def amg_info(self):
        lv = C.c_int32()
        nodes = np.zeros(64, np.int64)
        nnz = np.zeros(64, np.int64)
        oc = C.c_double()
        _check(_lib.knp_amg_info(self.handle, C.byref(lv), _lptr(nodes), _lptr(nnz), C.byref(oc)))
        return {"levels": lv.value, "nodes": nodes[:lv.value].tolist(), "nnz": nnz[:lv.value].tolist(),
                "op_complexity": oc.value}

    def amg_setup_info(self):
        """How the hierarchy was built: on the GPU or the host, the rows finished by the long-row
        kernels, and the setup's wall time."""
        r = AmgSetupRecord()
        _check(_lib.knp_amg_setup_info(self.handle, C.byref(r)))
        return {f: getattr(r, f) for f, _ in AmgSetupRecord._fields_}

    def info(self):
        i = ProblemInfo()
        _check(_lib.knp_problem_get_info(self.handle, C.byref(i)))
        return {f: getattr(i, f) for f, _ in ProblemInfo._fields_}

    def profile_begin(self, kernel_class):
        _check(_lib.knp_profile_begin(self.handle, int(kernel_class)))

    def profile_end(self):
        n = C.c_int64()
        ms = C.c_double()
        _check(_lib.knp_profile_end(self.handle, C.byref(n), C.byref(ms)))
        return n.value, ms.value

    def close(self):
        if getattr(self, "handle", None):
            _lib.knp_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def facet_arrays(cfg, mesh: Mesh):
    """Per-facet membrane model, leak conductances and stimulus mask in the library's facet order,
    from a workload description (same rule as the input recipe: the per-facet g_K draw of a facet
    is the slot of its intracellular element opposite the facet)."""
    v, elem_i, opp_i, _ = mesh.facets()
    nf = len(elem_i)
    model = np.full(nf, cfg.model, np.int32)
    gleak = np.tile(np.asarray(cfg.g_leak, np.float64), (nf, 1))
    if cfg.gK_sigma:
        xi = cfg.elem_facet_xi()[elem_i, opp_i]
        gleak[:, 1] = cfg.g_leak[1] * np.exp(cfg.gK_sigma * xi)
    cx = cfg.mesh.coords[v][:, :, 0].mean(axis=1)
    mask = (cx < cfg.stim_xmax).astype(np.uint8)
    return model, gleak, mask


def problem_from_config(cfg, stream=None, mesh: Mesh = None, degree: int = 1):
    """Mesh and Problem for a synthetic workload description (``synth.Config``); degree 1 (P1) or 2
    (P2 Lagrange elements, the bulk source evaluated at the P2 nodes)."""
    m = cfg.mesh
    if mesh is None:
        mesh = Mesh(m.coords, m.elems, m.elem_tag)
    p = cfg.params
    model, gleak, mask = facet_arrays(cfg, mesh)
    if degree == 2:
        e = mesh.p2()["edges"]
        source_e = cfg.source_e_at(np.vstack([m.coords, 0.5 * (m.coords[e[:, 0]] + m.coords[e[:, 1]])]))
    else:
        source_e = cfg.vertex_source_e()
    desc = dict(n_ions=3, z=p["z"], D_i=p["D"], D_e=p["D"], R=p["R"], T=p["T"], F=p["F"], Cm=p["Cm"], dt=cfg.dt,
                c_i0=p["c_i0"], c_e0=p["c_e0"], phi_M0=p["phi_M0"], facet_model=model, facet_gleak=gleak,
                ion_na=0, ion_k=1, gbar_na=p["gbar_Na"], gbar_k=p["gbar_K"], phi_rest=p["phi_rest"],
                w0=(p["n0"], p["m0"], p["h0"]), n_ode=25, stim_kind=cfg.stim_kind, stim_gbar=cfg.stim_gbar,
                stim_t0=cfg.stim_t0, stim_t1=cfg.stim_t1, stim_a=cfg.stim_a, stim_tau=cfg.stim_tau,
                stim_mask=mask, rho_pump=p["rho_pump"], P_na=p["P_Na"], P_k=p["P_K"],
                source_e=source_e, source_t0=cfg.source_t0, source_t1=cfg.source_t1, degree=degree)
    return mesh, Problem(mesh, desc, stream=stream)
