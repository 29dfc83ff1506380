#pragma once
#include "problem.h"

namespace knp {
struct knp_status_detail {
    knp_status code;
    int iterations;
    int restarts;
    double relres;
};
knp_status_detail fgmres(knp_problem* p, const knp_solve_opts& o, knp_solve_stats& stats);
void gmres_free(GmresWork* g);
}  // namespace knp
