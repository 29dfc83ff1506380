#pragma once
#include <map>
#include <tuple>
#include <vector>

#include "amg.h"

struct knp_problem;

namespace knp {

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
    std::map<std::tuple<const double*, const double*, double*>, VcycleGraph> graphs;
    ~AmgHierarchy();
};

void amg_upload(knp_problem* p, const HostHierarchy& H, int precision, int degree);
void vcycle_apply(knp_problem* p, const double* v, const double* s, double* z);

}  // namespace knp
