// The element pair values of the P2 weighted stiffness (Section 4.1, A_r^{k} with a P2
// concentration), shared by the per-step kernel and the host query of the region matrices.
#pragma once

#include "p2_tables.h"

namespace knp {

// out[p] = int_T c grad phi_j . grad phi_l for the off-diagonal local pairs p = (j, l) of one
// element: the moments mu_q = sum_j mom[q][j] c_j against 1, lambda_x, lambda_x lambda_y, then
// sum_t coef_t G[a_t][b_t] mu[q_t] with G = |T| grad lambda_a . grad lambda_b (row-major 4x4).
template <int D>
__host__ __device__ __forceinline__ void p2_pair_values(const P2Dev& T, const double* __restrict__ G,
                                               const double* __restrict__ c, double* __restrict__ out) {
    constexpr int NPE = (D + 1) * (D + 2) / 2;
    constexpr int NMOM = 1 + (D + 1) + (D + 1) * (D + 2) / 2;
    constexpr int NPAIR = NPE * (NPE - 1) / 2;
    double mu[NMOM];
    for (int q = 0; q < NMOM; ++q) {
        double s = 0.0;
        for (int j = 0; j < NPE; ++j) s += T.mom[q][j] * c[j];
        mu[q] = s;
    }
    for (int p = 0; p < NPAIR; ++p) {
        double v = 0.0;
        for (int t = T.tptr[p]; t < T.tptr[p + 1]; ++t) {
            const int32_t w = T.tabq[t];
            v += T.tcoef[t] * G[(w & 3) * 4 + ((w >> 2) & 3)] * mu[w >> 4];
        }
        out[p] = v;
    }
}

}  // namespace knp
