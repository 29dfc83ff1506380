#pragma once
#include <map>
#include <tuple>
#include <vector>

#include "amg.h"

struct knp_problem;

namespace knp {

// The coarse correction's two passes around the V-cycle, done inside it (device pointers and
// scalars; y == nullptr: none). The first kernel of the finest level forms the corrected input
// r - A Z y from r = s .* v (A Z y from the per-step row sums RS and the cross-region entries xe,
// as the coarse correction defines it), and the output kernel adds Z y to the potentials.
struct DeflFuse {
    const int32_t* rgrp = nullptr;   // intracellular node -> its cell group
    const double* RS = nullptr;      // [n][3] row sums of e^k over phi columns
    const int32_t* xptr = nullptr;   // cross-region entries of each row
    const int32_t* xg = nullptr;     // cross entry -> group of its column (-1: the pinned node)
    const double* xe = nullptr;      // [3][n_cross] cross-region values
    const double* y = nullptr;       // [groups + 1] the coarse solution, extracellular group last
    int64_t n_cross = 0, N_i = 0;
    int32_t pin = -1, ext_group = 0;
    double z[3] = {0, 0, 0};         // valences
};

// One captured V-cycle: a CUDA graph instantiated for a given (input, scale, output) triple.
struct VcycleGraph {
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
};

struct AmgHierarchy {
    int precision = 0;
    int levels = 0;
    std::vector<int64_t> nodes, nnz;
    void* h64 = nullptr;   // AmgDev<double>
    void* h32 = nullptr;   // AmgDev<float>
    // CUDA graphs of the V-cycle (one per FGMRES basis slot), captured on a private stream
    bool use_graphs = true;
    cudaStream_t gstream = nullptr;
    std::map<std::tuple<const double*, const double*, double*, const double*>, VcycleGraph> graphs;
    // CG(P_0): P_0^{-1} applied by V-cycle-preconditioned CG per field block (0 = one V-cycle)
    int inner_cg_max_it = 0;
    double inner_cg_rtol = 0.0;
    int64_t inner_its = 0;   // inner CG iterations so far
    // how the hierarchy was built: on the GPU (1) or on the host (0, host_setup), and the rows
    // of P and of the Galerkin products that the GPU setup finished with its long-row kernels
    int setup_on_gpu = 0;
    int64_t long_rows_p = 0, long_rows_rap = 0;
    double setup_ms = 0.0;
    ~AmgHierarchy();
};

// degree / pre: Chebyshev steps after / before the coarse-grid correction on every level
void amg_upload(knp_problem* p, const HostHierarchy& H, int precision, int degree, int pre);
struct GpuHierarchy;
// the hierarchy built by amg_build_gpu, taken over on the device (consumes H)
void amg_take_gpu(knp_problem* p, GpuHierarchy& H, int precision, int degree, int pre);
// z = V-cycle(s .* v); with df (y set), z = V-cycle(s .* v - A Z y) + Z y (the coarse correction's
// passes fused into the first and last kernels)
void vcycle_apply(knp_problem* p, const double* v, const double* s, double* z, const DeflFuse* df = nullptr);
// y = P_0 x with the finest level of the FP64 hierarchy; x, y [n][4] doubles on the device
void p0_apply(knp_problem* p, const double* x, double* y);
// z = P_0^{-1} (s .* v): one V-cycle, or CG(P_0) when the hierarchy was set up for it
void precond_apply(knp_problem* p, const double* v, const double* s, double* z);

}  // namespace knp
