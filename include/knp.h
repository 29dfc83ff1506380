/*
 * knp.h - C ABI of the GB300 KNP-EMI step library (libknp.so).
 *
 * The library advances the KNP-EMI equations (ion concentrations [k]_r and
 * potentials phi_r in the intracellular (i) and extracellular (e) regions,
 * coupled across the membrane Gamma) with the implicit-explicit linearised
 * time step of Section 3.2 of Benedusi, Ellingsrud, Herlyng and Rognes,
 * "Scalable approximation and solvers for ionic electrodiffusion in cellular
 * geometries" (arXiv 2403.04491). Each step is: membrane update (Section 3.2),
 * assembly of A_{n-1} and f_n (Section 4.1, Eq. 4.3), and the solve of
 * A_{n-1} u_n = f_n by flexible GMRES(30) right-preconditioned with one
 * algebraic-multigrid V-cycle on the block-diagonal P_0 (Eq. 4.4, Section 4.2,
 * Section 6.2).
 *
 * Conventions shared by every entry point:
 *  - Every function returns knp_status; knp_last_error() gives a
 *    thread-local, human-readable message for the last failure.
 *    No C++ exception crosses this boundary.
 *  - Inputs are caller-owned and copied at create time. Handles are
 *    library-owned and freed by their *_destroy function.
 *  - Device work is enqueued on the CUDA stream given at problem creation
 *    (a cudaStream_t passed as void*; NULL = legacy default stream). Calls
 *    that return host data synchronise that stream first.
 *  - One handle is not thread-safe; separate handles are independent.
 *  - Units are SI: m, s, V, mol/m^3, S/m^2, F/m^2.
 *  - Region node order is increasing vertex id; the membrane facet order is
 *    lexicographic in the facet's sorted vertex ids (see knp_mesh_facets).
 */
#ifndef KNP_H
#define KNP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t knp_status;
#define KNP_OK                 0
#define KNP_ERR_INVALID_ARG    1  /* a NULL pointer, a size out of range, an inconsistent option */
#define KNP_ERR_INVALID_MESH   2  /* degenerate element, cells sharing a facet or a vertex, a cell without membrane */
#define KNP_ERR_OOM            3  /* host or device allocation failed */
#define KNP_ERR_CUDA           4  /* a CUDA runtime call failed (message has the CUDA error string) */
#define KNP_ERR_NOT_CONVERGED  5  /* GMRES reached max_it without meeting rtol; the iterate is kept */
#define KNP_ERR_NUMERIC        6  /* NaN/Inf in a residual, a non-positive diagonal, a singular coarse matrix */
#define KNP_ERR_STATE          7  /* call out of order (e.g. knp_solve before knp_assemble_step) */

typedef enum { KNP_HOST = 0, KNP_DEVICE = 1 } knp_memspace;
typedef enum { KNP_MODEL_LEAK = 0, KNP_MODEL_HH = 1, KNP_MODEL_KIR = 2 } knp_membrane_model;
typedef enum { KNP_STIM_NONE = 0, KNP_STIM_WINDOW = 1, KNP_STIM_PERIODIC_EXP = 2 } knp_stimulus_kind;
typedef enum { KNP_PREC_FP64 = 0, KNP_PREC_FP32 = 1 } knp_precision;

#define KNP_MAX_IONS 4

typedef struct knp_mesh knp_mesh;
typedef struct knp_problem knp_problem;

/* ------------------------------------------------------------------------- */
/* Mesh (Section 3.3: conforming simplicial T = T_i U T_e matched at Gamma)   */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t dim;               /* 2 (triangles) or 3 (tetrahedra) */
    int64_t n_vertices;
    const double* coords;      /* host [n_vertices * dim], metres, row-major */
    int64_t n_elems;
    const int32_t* elems;      /* host [n_elems * (dim+1)] vertex ids */
    const int32_t* elem_tag;   /* host [n_elems]: 0 = extracellular, j >= 1 = cell j */
    const double* pin_point;   /* host [dim] or NULL (= the origin): the phi_e pin of Remark 4.1 goes on
                                  the extracellular vertex nearest to this point, ties by lowest id */
} knp_mesh_desc;

typedef struct {
    int32_t dim;
    int64_t n_vertices, n_elems;
    int64_t N_i, N_e;            /* region node counts (membrane vertices counted in both) */
    int64_t n_facets;            /* membrane facets */
    int64_t n_membrane_vertices;
    int32_t n_cells;             /* largest cell tag */
    int64_t pin_vertex;          /* extracellular vertex of the point pin (Remark 4.1) */
    int64_t n_dof;               /* (N_i + N_e)(n_ions + 1) for n_ions = 3 */
} knp_mesh_info;

/* Builds the topology: membrane facets are the facets shared by an element of
 * tag 0 and one of tag >= 1; every membrane vertex gets one node in each
 * region (Section 3.3; the count of Section 5.1). The pin is the extracellular
 * vertex nearest to desc->pin_point (the origin when NULL), ties broken by lowest
 * id (Remark 4.1).
 * Errors: KNP_ERR_INVALID_ARG (NULL, dim not 2/3, ids out of range),
 * KNP_ERR_INVALID_MESH (zero-volume element, two cells sharing a facet or a
 * vertex, regions touching outside membrane facets, a cell with no facet). */
knp_status knp_mesh_create(const knp_mesh_desc* desc, knp_mesh** out);
knp_status knp_mesh_get_info(const knp_mesh* mesh, knp_mesh_info* info);
/* Region node -> vertex id: nodes_i[N_i], nodes_e[N_e] (host, caller-allocated; either may be NULL). */
knp_status knp_mesh_nodes(const knp_mesh* mesh, int32_t* nodes_i, int32_t* nodes_e);
/* Membrane facets in library order (host, caller-allocated, any may be NULL):
 * vertices[n_facets*dim] sorted vertex ids; elem_i[n_facets] intracellular
 * element; opp_i[n_facets] local index (0..dim) of elem_i's vertex opposite
 * the facet; cell[n_facets] cell tag. */
knp_status knp_mesh_facets(const knp_mesh* mesh, int32_t* vertices, int32_t* elem_i,
                           int32_t* opp_i, int32_t* cell);
void knp_mesh_destroy(knp_mesh* mesh);

/* P2 nodes (Section 3.3 with polynomial degree p = 2; Section 6.3 runs p in {1, 2}). Global
 * node ids are the vertex ids 0..n_vertices-1, then n_vertices + e for the edges e in
 * lexicographic order of their sorted vertex pair (an edge node sits at the edge midpoint). A
 * node belongs to a region when it is a node of one of the region's elements, so the vertices
 * and edges of membrane facets get one node in each region; region node order is increasing
 * global id. Built on the first call for a mesh (thread-safe), host only.
 * Errors: KNP_ERR_INVALID_ARG (NULL, more than 2^31 - 1 nodes), KNP_ERR_INVALID_MESH (the two
 * regions share an edge that lies in no membrane facet). */
typedef struct {
    int64_t n_edges;
    int64_t n_nodes;             /* n_vertices + n_edges */
    int64_t N_i, N_e;            /* P2 region node counts (membrane nodes counted in both) */
    int64_t n_membrane_nodes;
    int64_t pin_node;            /* global id of the extracellular node nearest to the pin point,
                                    ties by lowest id (Remark 4.1) */
    int64_t n_dof;               /* (N_i + N_e)(n_ions + 1) for n_ions = 3 */
} knp_p2_info;

knp_status knp_mesh_p2_get_info(const knp_mesh* mesh, knp_p2_info* info);
/* P2 tables (host, caller-allocated, any may be NULL):
 * edges[n_edges*2] sorted vertex pairs; elem_nodes[n_elems*(d+1)(d+2)/2] the element's vertices
 * in its own order, then its edges (a, b), a < b, in lexicographic order of the local pair;
 * facet_nodes[n_facets*d(d+1)/2] the facet's sorted vertices (knp_mesh_facets order), then its
 * edges likewise; nodes_i[N_i], nodes_e[N_e] region node -> global id; membrane_nodes[
 * n_membrane_nodes] increasing; node_cell_i[N_i] the cell tag of each intracellular node. */
knp_status knp_mesh_p2_tables(const knp_mesh* mesh, int32_t* edges, int32_t* elem_nodes, int32_t* facet_nodes,
                              int32_t* nodes_i, int32_t* nodes_e, int32_t* membrane_nodes, int32_t* node_cell_i);
/* The P2 matrices M_r, A_r and A_r^{c} = [int c grad phi_j . grad phi_l] of one region (Section
 * 4.1 with p = 2) as the element contributions, unsummed: for each element of the region (region
 * 0 = intracellular, elements with tag >= 1 in increasing id; 1 = extracellular, tag 0) and each
 * (j, l) of its (d+1)(d+2)/2 local nodes, rows/cols = region node indices and M/A/Ac the
 * element's entries. c: host [N_r] nodal values of the P2 coefficient (needed for Ac only). The
 * library's P2 problems use the same values and, per step, the same element arithmetic for
 * A_r^{k} (Ac's diagonal is minus the off-diagonal row sum, exact since the basis sums to one).
 * *count = n_region_elems * ((d+1)(d+2)/2)^2; any output may be NULL (all NULL: *count only).
 * Host only. Errors: KNP_ERR_INVALID_ARG (NULL mesh or count, region not 0/1, Ac without c). */
knp_status knp_mesh_p2_region_matrices(const knp_mesh* mesh, int32_t region, const double* c, int64_t* count,
                                       int32_t* rows, int32_t* cols, double* M, double* A, double* Ac);

/* ------------------------------------------------------------------------- */
/* Problem (Sections 2, 3.2, Table 2)                                        */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t n_ions;                  /* |K|, 1..KNP_MAX_IONS */
    double z[KNP_MAX_IONS];          /* valences z_k */
    double D_i[KNP_MAX_IONS];        /* D_i^k, m^2/s */
    double D_e[KNP_MAX_IONS];        /* D_e^k, m^2/s */
    double R, T, F;                  /* gas constant, temperature, Faraday constant (psi = RT/F) */
    double Cm;                       /* membrane capacitance, F/m^2 */
    double dt;                       /* time step, s */
    double c_i0[KNP_MAX_IONS];       /* uniform initial [k]_i^0 */
    double c_e0[KNP_MAX_IONS];       /* uniform initial [k]_e^0 */
    double phi_M0;                   /* initial membrane potential; phi_i^0 = phi_M0, phi_e^0 = 0 */
    /* membrane (Eq. 2.15, the leak model and Kir-Na/K of Section 2.4.2): per facet, in
       knp_mesh_facets order */
    const int32_t* facet_model;      /* host [n_facets]: KNP_MODEL_LEAK, KNP_MODEL_HH or KNP_MODEL_KIR */
    const double* facet_gleak;       /* host [n_facets * n_ions] leak conductances g_leak^k */
    int32_t ion_na, ion_k;           /* ions carrying the HH Na / K channels and the stimulus (Na) */
    double gbar_na, gbar_k;          /* HH maximal conductances on HH facets */
    double phi_rest;                 /* HH resting potential, V */
    double w0[3];                    /* initial gates (n, m, h) */
    int32_t n_ode;                   /* Rush-Larsen substeps per step (25 in Section 6.2) */
    /* stimulus g_stim^Na(t) on masked facets, evaluated at t_{n-1} */
    int32_t stim_kind;               /* knp_stimulus_kind */
    double stim_gbar, stim_t0, stim_t1, stim_a, stim_tau;
    const uint8_t* stim_mask;        /* host [n_facets] (1 = stimulated) or NULL = all facets */
    /* Kir-Na/K facets (Section 2.4.2): the K leak is g_leak^K (phi_M - E_K) f_Kir([K]_e, phi_M - E_K,
       phi_M) with E_K^0 and [K]_e^0 taken from c_i0, c_e0 of ion_k; the Na/K pump adds
       3 F z_Na j_pump to the Na current and -2 F z_K j_pump to the K current, with
       j_pump = rho_pump [Na]_i^1.5 / ([Na]_i^1.5 + P_na^1.5) [K]_e / ([K]_e + P_k). Nodal at the
       membrane vertices, P1 on the facets, like every membrane coefficient. */
    double rho_pump;                 /* maximum pump rate, mol/(m^2 s) (Table 2: 1.115e-6) */
    double P_na, P_k;                /* pump thresholds, mol/m^3 (Table 2: 10, 1.5) */
    /* bulk source f_r^k (Eq. 2.1), entering f_n as dt M f_r^{k,n} (Eq. 3.5 with the dt factor):
       host [n_vertices * n_ions] nodal values (mol/(m^3 s)) for the intracellular and the
       extracellular copy of each vertex, or NULL = none; on for steps with source_t0 < t_n <=
       source_t1 (t_n the end of the step) */
    const double* source_i;
    const double* source_e;
    double source_t0, source_t1;
    /* polynomial degree p of the Lagrange spaces (Section 3.3): 0 or 1 = P1, 2 = P2. With P2 the
       unknowns live on the P2 nodes of knp_mesh_p2_*: region node order, the membrane nodes
       (gates, membrane coefficients) and the pin are those of knp_mesh_p2_tables, and source_i /
       source_e are indexed by global P2 node id ([n_nodes * n_ions], knp_p2_info.n_nodes). The
       adjoint step covers P1 only. */
    int32_t degree;
} knp_problem_desc;

/* Creates device state for one simulation on `stream`; u_0 as in Section 2.3
 * with phi_i^0 = phi_M0 and phi_e^0 = 0, gates w_0 at every membrane vertex.
 * Errors: KNP_ERR_INVALID_ARG, KNP_ERR_OOM, KNP_ERR_CUDA.
 * Dry run: with the environment variable KNP_DRY_RUN_TABLES=<file>, the call builds the
 * problem's host tables (pattern, static values, incidences, membrane tables, source), appends
 * each of them to <file> as (int64 name length, int64 count, int64 element size, name, data),
 * does no device work at all and returns KNP_ERR_STATE with no handle. It lets a problem set-up
 * be inspected on a machine without a GPU. */
knp_status knp_problem_create(const knp_mesh* mesh, const knp_problem_desc* desc, void* stream,
                              knp_problem** out);
void knp_problem_destroy(knp_problem* prob);
/* Waits for all work the library has enqueued for this problem on its stream (the library's
 * calls are stream-ordered; knp_solve, knp_step and the getters that return host data
 * synchronise by themselves). Errors: KNP_ERR_INVALID_ARG, KNP_ERR_CUDA (the stream's error). */
knp_status knp_sync(knp_problem* prob);

/* Membrane update and assembly for the current step n (Section 3.2, Section
 * 4.1): from u_{n-1}, w_{n-1} and t_{n-1}, computes w_n by Rush-Larsen with
 * phi_M frozen, the explicit I_ch^{k,n-1}, alpha^{n-1}, C^{n-1}, the values of
 * A_{n-1} in its fixed pattern and f_n (Eq. 4.3), with the point pin of
 * Remark 4.1. Stream-ordered; returns without synchronising. */
knp_status knp_assemble_step(knp_problem* prob);

typedef struct {
    int32_t precision;          /* knp_precision of the hierarchy and V-cycle (FGMRES stays FP64) */
    double theta;               /* strength threshold of the aggregation graph (0.08 default) */
    int32_t coarse_max;         /* stop coarsening at <= this many nodes (dense coarse solve; 500) */
    int32_t max_levels;         /* (12) */
    int32_t cheb_degree;        /* Chebyshev steps after the coarse-grid correction on every level
                                   (2: with the coarse correction of knp_solve_opts.deflate, degree 2
                                   on [lambda_max/3, 1.1 lambda_max] took the 256^3 workload from 36 to
                                   24 FGMRES iterations per step, 20% less time, and was within 3% of
                                   degree 1 on the smallest 3D workload) */
    double cheb_ratio;          /* lower eigenvalue bound = lambda_max / cheb_ratio (3) */
    double theta_coarse;        /* strength threshold on levels >= 1 (< 0: same as theta; 0) */
    double p_drop;              /* drop prolongator entries below p_drop x the row's largest (0: keep all) */
    int32_t host_setup;         /* 1: build the hierarchy on the host (the reference a test compares the
                                   GPU build with); 0: on the GPU, with no host fallback (rows of P or of
                                   the Galerkin products too long for the short-row kernels are finished
                                   by the GPU's long-row kernels) */
    int32_t inner_cg_max_it;    /* 0: P_0^{-1} is one V-cycle (AMG(P_0), Section 4.2). > 0: CG(P_0) of
                                   Section 6.3: each of the 2(|K|+1) field blocks of P_0 is solved by
                                   CG preconditioned with the V-cycle, to inner_cg_rtol or this many
                                   iterations (FP64 hierarchy only) */
    double inner_cg_rtol;       /* relative residual of each block's CG */
    int32_t cheb_degree_pre;    /* Chebyshev steps before the coarse-grid correction; <= 0 selects 1.
                                   The first step starts from x = 0 and needs no operator product, so
                                   1 before and 2 after costs one finest-level product less per
                                   V-cycle than 2 and 2: 2.6%, 5% and 10% less time per step on the
                                   256^3, 128^3 and 64^3 workloads, for 2-5% more iterations. FGMRES
                                   takes the non-symmetric V-cycle; CG(P_0) (inner_cg_max_it > 0)
                                   uses cheb_degree on both sides. */
} knp_amg_opts;

/* Smoothed-aggregation AMG on P_0 (Eq. 4.4) assembled from the initial
 * state and reused for every step (Section 4.2). Must follow
 * knp_problem_create and precede knp_solve. P_0 is taken from the assembled
 * operator on the GPU; with host_setup = 0 the hierarchy is built there too and
 * handed to the V-cycle without passing through host memory. Synchronises the
 * problem's stream. Errors: KNP_ERR_INVALID_ARG, KNP_ERR_OOM, KNP_ERR_NUMERIC
 * (a non-positive diagonal of P_0, a singular coarse matrix), KNP_ERR_CUDA. */
knp_status knp_amg_setup(knp_problem* prob, const knp_amg_opts* opts);

/* How the last knp_amg_setup built the hierarchy (Section 4.2's setup, which the paper
 * counts as initialisation). */
typedef struct {
    int32_t on_gpu;           /* 1: built on the GPU; 0: on the host (host_setup = 1) */
    int64_t long_rows_p;      /* rows of the smoothed prolongators finished by the long-row kernel */
    int64_t long_rows_rap;    /* rows of A P and R (A P) finished by the long-row kernel */
    double setup_ms;          /* wall time of knp_amg_setup, P_0 extraction included */
} knp_amg_setup_record;
/* Errors: KNP_ERR_INVALID_ARG, KNP_ERR_STATE (no hierarchy yet). */
knp_status knp_amg_setup_info(const knp_problem* prob, knp_amg_setup_record* rec);

typedef struct {
    double rtol;       /* on the preconditioned residual: ||S M^-1 r||_g <= rtol max(||S x_c||_g,
                          ||S (x - x_c)||_g) for the concentration part and the potential part g,
                          S^2 = diag(P_0), M^-1 = one V-cycle on P_0, x_c = the iterate the current
                          restart cycle began from (the first: x_0 = u_{n-1}) (the paper's
                          preconditioned test, Section 6.2, in the scaled norm, relative to the
                          iterate or, for a cold start, to the computed correction); with
                          phi_e_group the phi_e part is floored at phi_e_floor ||S phi|| */
    int32_t restart;   /* 30 (Section 6.2) */
    int32_t max_it;    /* total iterations */
    int32_t phi_e_group;  /* 1: test the extracellular potentials as a third group (phi_e is some 1e-8
                             of phi_i; a loss built on phi_e needs it resolved on its own scale) */
    int32_t deflate;      /* 1: wrap P_0^{-1} in a coarse correction of the potentials' near-null modes
                             (each cell's constant phi_i, the constant phi_e; E = Z^T A Z solved
                             exactly). The potential blocks of P_0 are held only by the membrane
                             capacitance and the point pin, so one V-cycle amplifies residuals along
                             these modes; the paper's left-preconditioned GMRES minimises exactly that
                             amplified residual, right-preconditioned FGMRES needs the correction to
                             converge in the same norm. Also for the adjoint's A^T solve (E^T). */
    int32_t stop_test;    /* KNP_TEST_SCALED (0): the per-group scaled test above. KNP_TEST_PAPER (1):
                             the test of the paper's solver settings (Section 6.2),
                             ||M^-1 r||_2 <= rtol ||M^-1 f||_2 over the whole unscaled vector, for
                             comparing iteration counts with Tables 3 and 4 */
    double phi_e_floor;   /* with phi_e_group: the phi_e part is tested against
                             max(rtol ||S phi_e||, phi_e_floor ||S phi||); <= 0 selects 1e-14 */
    int32_t x0_extrapolate;  /* 1: start from x_0 = 2 u_{n-1} - u_{n-2} (linear extrapolation in time)
                                instead of the paper's x_0 = u_{n-1}, when the previous knp_solve on
                                this problem also extrapolated and succeeded and no knp_state_set came
                                between; otherwise x_0 = u_{n-1}. Changes the iteration count, not the
                                stopping test. Keeps one more state vector on the device. */
} knp_solve_opts;

enum { KNP_TEST_SCALED = 0, KNP_TEST_PAPER = 1 };

typedef struct {
    int32_t iterations;
    int32_t restarts;
    double true_relres;    /* scaled true residual ||S^-1 (f - A u)|| / ||S^-1 f|| at exit */
    double ms;             /* wall time of the solve (host clock, includes synchronisation) */
    int64_t inner_iterations;  /* inner CG iterations of CG(P_0) over the solve (0 for AMG(P_0)) */
} knp_solve_stats;

/* FGMRES(restart), FP64, x_0 = u_{n-1} (Section 6.2; or extrapolated, x0_extrapolate), right-preconditioned by
 * one V-cycle on P_0. On success the step is committed: the state becomes
 * (u_n, w_n) and t advances by dt. KNP_ERR_NOT_CONVERGED keeps the last
 * iterate in u and does not advance w or t. */
knp_status knp_solve(knp_problem* prob, const knp_solve_opts* opts, knp_solve_stats* stats);

typedef struct {
    int32_t iterations;
    double true_relres;
} knp_step_stats;

/* nsteps x (knp_assemble_step, knp_solve, t += dt). per_step may be NULL. */
knp_status knp_step(knp_problem* prob, int32_t nsteps, const knp_solve_opts* opts,
                    knp_step_stats* per_step);

/* Replaces the per-facet leak conductances g_leak^k ([n_facets * n_ions], facet order of
 * knp_mesh_facets, ion-minor) from host or device memory; takes effect at the next assembly.
 * (The gradient of knp_adjoint_get is with respect to these.) */
knp_status knp_problem_set_facet_gleak(knp_problem* prob, knp_memspace space, const double* gleak);

/* ------------------------------------------------------------------------- */
/* Adjoint (not in the paper: the discrete adjoint of the time loop)          */
/* ------------------------------------------------------------------------- */
/* For a loss L(u_1..u_N) the reverse sweep runs, for n = N..1,
 *     A_{n-1}^T lambda_n = dL/du_n + rho_n
 * where rho_n carries d/du_n of the later steps' explicit dependence on u_n (through
 * A^{k,n}, alpha, C, E_k, phi_M^n in I_ch and f, and the HH gates), and accumulates the
 * gradients with respect to the per-facet leak conductances, u_0 and w_0. The
 * transposed solve is FGMRES with the same P_0 hierarchy (P_0 is symmetric, Section
 * 4.2) and the same stopping test.
 * knp_adjoint_begin zeroes the carried quantities and the accumulators (allocating the
 * adjoint work arrays on first use); it returns KNP_ERR_INVALID_ARG for a problem with
 * Kir-Na/K facets, whose partial derivatives are not implemented. A bulk source does not
 * depend on the state or the conductances and needs nothing. */
knp_status knp_adjoint_begin(knp_problem* prob);
/* One reverse step n. Precondition: the problem's state is (u_{n-1}, w_{n-1}, t_{n-1})
 * (restore it with knp_state_set, e.g. from a checkpoint and a recomputed segment). u_n
 * is the forward solution of step n and dLdu_n the loss's partial derivative with
 * respect to u_n, both [n_dof] in the Eq. 4.3 order, in `space`. The call assembles
 * A_{n-1}, solves for lambda_n, and updates the carried quantities and the gradient
 * accumulators. The state itself is not changed. Errors: KNP_ERR_STATE (no
 * knp_adjoint_begin or knp_amg_setup), KNP_ERR_NOT_CONVERGED, KNP_ERR_CUDA. */
knp_status knp_adjoint_step(knp_problem* prob, knp_memspace space, const double* u_n, const double* dLdu_n,
                            const knp_solve_opts* opts, knp_solve_stats* stats);
/* After the step n = 1: dLdu0 [n_dof] (Eq. 4.3 order; the entries of c_i^k are the
 * gradient with respect to the initial intracellular concentrations), dLdw0 [3 *
 * n_membrane_vertices], grad_gleak [n_facets * n_ions], and the last lambda [n_dof].
 * Any pointer may be NULL; buffers in `space`. */
knp_status knp_adjoint_get(knp_problem* prob, knp_memspace space, double* dLdu0, double* dLdw0,
                           double* grad_gleak, double* lambda);

/* State access in region node order. Buffers are [n_ions * N_r] (ion-major)
 * for concentrations, [N_r] for potentials, [3 * n_membrane_vertices] (gate-
 * major n, m, h) for gates; any pointer may be NULL. `space` says where the
 * caller's buffers live. knp_state_get synchronises the stream. */
knp_status knp_state_get(const knp_problem* prob, knp_memspace space, double* c_i, double* phi_i,
                         double* c_e, double* phi_e, double* gates, double* t);
knp_status knp_state_set(knp_problem* prob, knp_memspace space, const double* c_i, const double* phi_i,
                         const double* c_e, const double* phi_e, const double* gates, double t);

/* ------------------------------------------------------------------------- */
/* Inspection entry points (for parity tests against an independent          */
/* implementation; not needed to run a simulation)                            */
/* ------------------------------------------------------------------------- */

/* Unknown order used by the inspection calls: the paper's Eq. 4.3 order
 * [c_i^1..c_i^K, phi_i, c_e^1..c_e^K, phi_e], each block in region node order;
 * n = n_dof. */

/* f_n of the last knp_assemble_step into rhs[n] (host). */
knp_status knp_rhs_get(const knp_problem* prob, double* rhs);
/* y = A_{n-1} x with the last assembled operator; x, y host [n]. */
knp_status knp_apply_operator(knp_problem* prob, const double* x, double* y);
/* y = A_{n-1}^T x with the last assembled operator; x, y host [n]. */
knp_status knp_apply_operator_transpose(knp_problem* prob, const double* x, double* y);
/* Entries of A_{n-1}: for each (row, col) pair in the Eq. 4.3 order, the value
 * (0 where the entry is outside the pattern). rows, cols, vals host [count]. */
knp_status knp_operator_entries(knp_problem* prob, int64_t count, const int64_t* rows,
                                const int64_t* cols, double* vals);
/* z = V-cycle(P_0) r (one application of the preconditioner, unscaled); host [n]. */
knp_status knp_apply_preconditioner(knp_problem* prob, const double* r, double* z);
/* z = M_D^{-1} r: the preconditioner of knp_solve with deflate = 1, P_0^{-1} wrapped in the coarse
 * correction of the potentials' near-null modes (each cell's constant phi_i and the constant
 * phi_e): y = E^{-1} Z^T r with E = Z^T A_{n-1} Z, z = V-cycle(P_0)(r - A_{n-1} Z y) + Z y, on the
 * operator of the current assembly; with transpose = 1 the adjoint solve's form, with A^T and
 * E^T in their places. Host [n] arrays in the Eq. 4.3 order. Errors: KNP_ERR_INVALID_ARG,
 * KNP_ERR_STATE (no hierarchy or no assembled step), KNP_ERR_CUDA. */
knp_status knp_apply_deflated_preconditioner(knp_problem* prob, const double* r, double* z, int32_t transpose);
/* Allocation-free variant of knp_apply_preconditioner. The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc when they need the
 * preconditioner - code running under a CUDA stream capture or while a CUDA graph is being
 * built, hosts that fix their device memory up front, and plugin or embedded hosts that
 * forbid allocation after start-up.
 * r and z are DEVICE pointers to [n_dof] doubles in the same Eq. 4.3 order as
 * knp_apply_preconditioner, owned by the caller; z = V-cycle(P_0) r with the same kernels
 * and hierarchy, so the result equals knp_apply_preconditioner's. The call allocates
 * nothing: its work vectors live in one static device array of 32 MiB that every GPU which
 * loads the library holds until the process exits. Hierarchies whose work vectors need more
 * than that (about 120,000 nodes with the FP64 hierarchy, 180,000 with FP32) are rejected with
 * KNP_ERR_INVALID_ARG and a message giving the size. The device that is current at the call
 * must be the one the problem was created on (else KNP_ERR_INVALID_ARG), because the array is
 * looked up on the current device. The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first call before any
 * stream capture. All calls share the array and keep the last call's
 * contents, so calls that overlap on the GPU (other streams, other problems, other host
 * threads) race and must be serialised by the caller. Stream-ordered on the problem's
 * stream; returns without synchronising. Errors: KNP_ERR_INVALID_ARG, KNP_ERR_STATE (no
 * hierarchy), KNP_ERR_CUDA. */
knp_status knp_apply_preconditioner_noalloc(knp_problem* prob, const double* r, double* z);
/* Hierarchy summary: levels, per-level node counts and nonzeros (host arrays of
 * length >= max_levels), operator complexity. */
knp_status knp_amg_info(const knp_problem* prob, int32_t* levels, int64_t* nodes, int64_t* nnz,
                        double* op_complexity);

typedef struct {
    int64_t n_nodes;          /* N_i + N_e */
    int64_t nnz_region;       /* stored same-region node-block entries of A (no padding) */
    int64_t nnz_padded;       /* the same in the sliced-ELL layout, with padding */
    int64_t nnz_cross;        /* cross-region membrane entries (B_rq) */
    int64_t n_membrane_pairs; /* membrane vertex pairs sharing a facet */
    int64_t n_edges;          /* undirected same-region edges */
    int64_t edge_incidences;  /* (edge, element) incidences used by the weighted-stiffness pass */
    int64_t step_index;       /* committed steps */
} knp_problem_info;
knp_status knp_problem_get_info(const knp_problem* prob, knp_problem_info* info);

/* Kernel timing for roofline measurements: while a class is active, the library
 * records a CUDA event pair on the problem's stream around every launch of that
 * class. knp_profile_end synchronises the stream and returns the launch count and
 * the summed device time. Classes: 0 operator SpMV (y = A x), 1 finest-level
 * Chebyshev step, 2 finest-level residual, 3 assembly (the six kernels of one
 * knp_assemble_step as one interval), 4 whole V-cycle, 5 Arnoldi orthogonalisation
 * (one iteration's kernels as one interval). */
knp_status knp_profile_begin(knp_problem* prob, int32_t kernel_class);
knp_status knp_profile_end(knp_problem* prob, int64_t* launches, double* total_ms);
/* Number of CUDA kernels this library has launched since it was loaded. */
knp_status knp_launch_count(int64_t* count);

const char* knp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* KNP_H */
