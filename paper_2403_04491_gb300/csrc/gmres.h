#pragma once
#include "problem.h"

namespace knp {
struct knp_status_detail {
    knp_status code;
    int iterations;
    int restarts;
    double relres;
};
// Solves A x = f (or A^T x = f) in place, x holding the initial guess.
knp_status_detail fgmres(knp_problem* p, const knp_solve_opts& o, knp_solve_stats& stats, double* x, const double* f,
                         bool transpose);
void gmres_free(GmresWork* g);
}  // namespace knp
