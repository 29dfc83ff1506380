// Reference tables of the P2 Lagrange basis (Section 3.3 with polynomial degree p = 2).
//
// Local node order on a d-simplex: the d+1 vertices, then the edges (a, b), a < b, in
// lexicographic order; the basis is lambda_a (2 lambda_a - 1) at vertex a and 4 lambda_a lambda_b
// at edge (a, b). All integrals are over the simplex of unit measure and exact (moment formula
// int prod lambda^k = m! prod k! / (m + sum k)!); an element's integral is |T| times the table.
#pragma once

#include <cstdint>

namespace knp {

constexpr int P2_NPE_MAX = 10;    // nodes of a P2 tetrahedron
constexpr int P2_NFN_MAX = 6;     // nodes of a P2 triangle (the facet of a tetrahedron)
constexpr int P2_NMOM_MAX = 15;   // barycentric monomials of degree <= 2 in 4 variables
constexpr int P2_NPAIR_MAX = 45;  // off-diagonal local pairs j < l of a P2 tetrahedron
constexpr int P2_NTERM_MAX = 512;

// One term of an off-diagonal weighted-stiffness entry: coef * G[a][b] * mu[q], where
// G[a][b] = |T| grad lambda_a . grad lambda_b and mu[q] = sum_c mom[q][c] c_c.
struct P2Term {
    int32_t a, b, q;
    double coef;
};

struct P2Ref {
    int d = 0;        // element dimension (2 or 3)
    int npe = 0;      // (d+1)(d+2)/2
    int nfn = 0;      // d(d+1)/2 (nodes of a facet)
    int nmom = 0;     // 1 + (d+1) + (d+1)(d+2)/2
    int npairs = 0;   // npe (npe - 1) / 2
    int nterms = 0;
    double mass[P2_NPE_MAX][P2_NPE_MAX];             // int phi_j phi_l
    double stiff[P2_NPE_MAX][P2_NPE_MAX][4][4];      // int (d phi_j / d lambda_a)(d phi_l / d lambda_b)
    double fmass[P2_NFN_MAX][P2_NFN_MAX];            // facet: int phi_j phi_l
    double ftriple[P2_NFN_MAX][P2_NFN_MAX][P2_NFN_MAX];  // facet: int phi_c phi_j phi_l
    // moments of a P2 field c against the monomials 1, lambda_x, lambda_x lambda_y (x <= y):
    // mu[q] = sum_c mom[q][c] c_c (unit measure)
    double mom[P2_NMOM_MAX][P2_NPE_MAX];
    // off-diagonal pairs p: (pj[p], pl[p]), pj < pl, and their terms tptr[p] .. tptr[p+1]-1:
    // int c grad phi_j . grad phi_l = sum_t coef_t G[a_t][b_t] mu[q_t] (grad phi = sum_a
    // d phi / d lambda_a grad lambda_a, and each d phi / d lambda_a is linear in lambda)
    int32_t pj[P2_NPAIR_MAX], pl[P2_NPAIR_MAX];
    int32_t tptr[P2_NPAIR_MAX + 1];
    P2Term terms[P2_NTERM_MAX];
};

// The tables for d = 2 or 3 (built once, thread-safe).
const P2Ref& p2_ref(int d);

// The part of P2Ref that the per-step kernels read (held in constant memory on the device), with
// each term packed as a | b << 2 | q << 4.
struct P2Dev {
    int32_t npe, nfn, nmom, npairs;
    int32_t tptr[P2_NPAIR_MAX + 1];
    int32_t tabq[P2_NTERM_MAX];
    double tcoef[P2_NTERM_MAX];
    double mom[P2_NMOM_MAX][P2_NPE_MAX];
    double fmass[P2_NFN_MAX][P2_NFN_MAX];
    double ftriple[P2_NFN_MAX][P2_NFN_MAX][P2_NFN_MAX];
};

// P2Dev of dimension d = 2 or 3 (built once, thread-safe).
const P2Dev& p2_dev(int d);

}  // namespace knp
