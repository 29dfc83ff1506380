#pragma once
#include <vector>

#include "amg.h"

struct knp_problem;

namespace knp {

struct AmgHierarchy {
    int precision = 0;
    int levels = 0;
    std::vector<int64_t> nodes, nnz;
    void* h64 = nullptr;   // AmgDev<double>
    void* h32 = nullptr;   // AmgDev<float>
    ~AmgHierarchy();
};

void amg_upload(knp_problem* p, const HostHierarchy& H, int precision, int degree);
void vcycle_apply(knp_problem* p, const double* v, const double* s, double* z);

}  // namespace knp
