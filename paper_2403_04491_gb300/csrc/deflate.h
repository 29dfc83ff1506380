// Coarse correction of the potentials' near-null modes around P_0^{-1} (deflate.cu).
#pragma once
#include "problem.h"

namespace knp {
// Forms the per-step data of the correction (row sums of the membrane terms, the arrowhead
// E = Z^T A Z) from the current assembly; does nothing if it is already current.
void deflation_prepare(knp_problem* p);
// z = P_0^{-1} (r - A Z y) + Z y with r = s .* v, y = E^{-1} Z^T r (after deflation_prepare); with
// transpose, A^T and E^T in their places (P_0 is symmetric)
void deflated_precond_apply(knp_problem* p, const double* v, const double* s, double* z, bool transpose = false);
void deflation_free(Deflation* d);
}  // namespace knp
