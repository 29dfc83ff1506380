// Per-step membrane update and assembly of A_{n-1} and f_n (Section 3.2, Section 4.1,
// Eq. 4.3). Six stream-ordered launches, none of them using atomics:
//   membrane_nodes   phi_M, E_k, alpha_r^k, C_r^k, Rush-Larsen gates, channel driving terms
//   elem_means       element means of [k]^{n-1} (exact weight of A_r^{k,n-1} for P1)
//   edge_values      A_r^{k,n-1} on each undirected edge: sum over incident elements
//   row_assemble     per row: tau~ A^k off-diagonals, the diagonal as minus the row sum,
//                    and the bulk right-hand side M c^{k,n-1}
//   membrane_pairs   C_r^k-weighted membrane mass on same-region and cross-region entries
//   membrane_rhs     -int g_r^k v and -int h_r w at membrane nodes
// P2 elements replace elem_means by element pair values and use the P2 facet basis in the two
// membrane kernels (the P2 section at the end of the anonymous namespace).
#include <mutex>

#include "p2_pairs.cuh"
#include "problem.h"

namespace knp {

namespace {

__device__ __forceinline__ double vtrap(double x) {
    // x / (exp(x) - 1), continuous at 0
    if (fabs(x) < 1e-6) return 1.0 - 0.5 * x + x * x / 12.0;
    return x / expm1(x);
}

// Moment of lambda_a lambda_b lambda_c over a unit-measure m-simplex (m = 1 or 2).
__device__ __forceinline__ double moment3(int m, int a, int b, int c) {
    int eq = (a == b) + (a == c) + (b == c);  // 3: all equal, 1: one pair, 0: distinct
    if (m == 1) return eq == 3 ? 0.25 : 1.0 / 12.0;
    return eq == 3 ? 0.1 : (eq == 1 ? 1.0 / 30.0 : 1.0 / 60.0);
}

__device__ __forceinline__ double moment2(int m, int a, int b) {
    // int lambda_a lambda_b = (1 + delta_ab) / ((m+1)(m+2))
    double den = (double)((m + 1) * (m + 2));
    return (a == b ? 2.0 : 1.0) / den;
}

__global__ void k_membrane_nodes(StepParams sp, int64_t nmv, const int32_t* __restrict__ mv_g,
                                 const double* __restrict__ u, const double* __restrict__ gates,
                                 double* __restrict__ gates_new, double* __restrict__ mf) {
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= nmv) return;
    int64_t gi = mv_g[a], ge = mv_g[nmv + a];
    double ci[KI], ce[KI];
    for (int k = 0; k < KI; ++k) {
        ci[k] = u[4 * gi + k];
        ce[k] = u[4 * ge + k];
    }
    double phiM = u[4 * gi + 3] - u[4 * ge + 3];
    double E[KI], si = 0, se = 0, wi[KI], we[KI];
    for (int k = 0; k < KI; ++k) {
        E[k] = sp.R * sp.T / (sp.F * sp.z[k]) * log(ce[k] / ci[k]);
        wi[k] = sp.reg[0].tau[k] * sp.z[k] * sp.z[k] * ci[k];
        we[k] = sp.reg[1].tau[k] * sp.z[k] * sp.z[k] * ce[k];
        si += wi[k];
        se += we[k];
    }
    mf[a] = phiM;
    for (int k = 0; k < KI; ++k) {
        mf[(1 + k) * nmv + a] = (wi[k] / si) * sp.Cm / (sp.F * sp.z[k]);
        mf[(4 + k) * nmv + a] = (we[k] / se) * sp.Cm / (sp.F * sp.z[k]);
        mf[(7 + k) * nmv + a] = phiM - E[k];
    }
    // Hodgkin-Huxley gates (n, m, h): N_ode Rush-Larsen substeps with phi_M frozen
    double V = 1e3 * (phiM - sp.phi_rest);
    double al[3], be[3];
    al[0] = 0.1 * vtrap((10.0 - V) / 10.0);
    be[0] = 0.125 * exp(-V / 80.0);
    al[1] = 1.0 * vtrap((25.0 - V) / 10.0);
    be[1] = 4.0 * exp(-V / 18.0);
    al[2] = 0.07 * exp(-V / 20.0);
    be[2] = 1.0 / (exp((30.0 - V) / 10.0) + 1.0);
    double h = 1e3 * sp.dt / sp.n_ode;
    double w[3];
    for (int g = 0; g < 3; ++g) {
        double winf = al[g] / (al[g] + be[g]);
        double dec = exp(-(al[g] + be[g]) * h);
        double x = gates[g * nmv + a];
        for (int s = 0; s < sp.n_ode; ++s) x = winf + (x - winf) * dec;
        gates_new[g * nmv + a] = x;
        w[g] = x;
    }
    mf[10 * nmv + a] = w[1] * w[1] * w[1] * w[2] * (phiM - E[sp.ion_na]);
    mf[11 * nmv + a] = (w[0] * w[0]) * (w[0] * w[0]) * (phiM - E[sp.ion_k]);
    // Kir-Na/K (Section 2.4.2): the K drive rectified by f_Kir, and the pump flux density
    const double dK = phiM - E[sp.ion_k];
    const double fA = 1.0 + exp(0.433), fB = 1.0 + exp(-(0.1186 + sp.EK0) / 0.0441);
    const double fC = 1.0 + exp((dK + 0.0185) / 0.0425), fD = 1.0 + exp(-(0.1186 + phiM) / 0.0441);
    mf[12 * nmv + a] = dK * (fA * fB / (fC * fD) * sqrt(ce[sp.ion_k] / sp.cKe0));
    const double na15 = ci[sp.ion_na] * sqrt(ci[sp.ion_na]), pna15 = sp.P_na * sqrt(sp.P_na);
    mf[13 * nmv + a] = sp.rho_pump * (na15 / (na15 + pna15)) * (ce[sp.ion_k] / (ce[sp.ion_k] + sp.P_k));
}

__global__ void k_elem_means(int64_t ne, int nvpe, const int32_t* __restrict__ eln, const double* __restrict__ u,
                             double* __restrict__ cbar) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= ne) return;
    double s[KI] = {0, 0, 0};
    for (int j = 0; j < nvpe; ++j) {
        int64_t g = eln[e * nvpe + j];
        for (int k = 0; k < KI; ++k) s[k] += u[4 * g + k];
    }
    for (int k = 0; k < KI; ++k) cbar[k * ne + e] = s[k] / nvpe;
}

__global__ void k_edge_values(int64_t n_edges, int64_t ne, const int32_t* __restrict__ eptr,
                              const int32_t* __restrict__ einc, const double* __restrict__ ecoef,
                              const double* __restrict__ cbar, double* __restrict__ ak) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_edges) return;
    double s[KI] = {0, 0, 0};
    for (int t = eptr[e]; t < eptr[e + 1]; ++t) {
        int64_t el = einc[t];
        double c = ecoef[t];
        for (int k = 0; k < KI; ++k) s[k] += cbar[k * ne + el] * c;
    }
    for (int k = 0; k < KI; ++k) ak[k * n_edges + e] = s[k];
}

__global__ void k_row_assemble(StepParams sp, int64_t n, int64_t N_i, int32_t pin, int64_t n_entries,
                               int64_t n_edges, const int64_t* __restrict__ slice_ptr,
                               const int32_t* __restrict__ col, const int32_t* __restrict__ edge,
                               const double* __restrict__ msv, const double* __restrict__ ak,
                               const double* __restrict__ u, const double* __restrict__ src, double src_dt,
                               double* __restrict__ e, double* __restrict__ f) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const RegionCoef rc = sp.reg[r < N_i ? 0 : 1];
    int64_t s = r / SELL_C;
    int64_t base = slice_ptr[s] + r % SELL_C;
    int64_t w = (slice_ptr[s + 1] - slice_ptr[s]) / SELL_C;
    double sum[KI] = {0, 0, 0}, fm[KI] = {0, 0, 0}, fs[KI] = {0, 0, 0};
    int64_t dpos = -1;
    for (int64_t k = 0; k < w; ++k) {
        int64_t pos = base + k * SELL_C;
        int32_t ed = edge[pos];
        if (ed == -2) continue;
        int64_t c = col[pos];
        double mv = msv[pos];
        for (int i = 0; i < KI; ++i) fm[i] += mv * u[4 * c + i];
        if (src)
            for (int i = 0; i < KI; ++i) fs[i] += mv * src[4 * c + i];
        if (ed == -1) {
            dpos = pos;
            continue;
        }
        for (int i = 0; i < KI; ++i) {
            double v = rc.taut[i] * ak[i * n_edges + ed];
            sum[i] += v;
            e[i * n_entries + pos] = v;
        }
    }
    // the pinned phi_e column is not zeroed here: the operator kernels ignore it (see spmv.cu)
    for (int i = 0; i < KI; ++i) e[i * n_entries + dpos] = -sum[i];
    // f_r^k = M c^{k,n-1} + dt M f_r^{k,n} (the membrane terms are added by k_membrane_rhs)
    for (int i = 0; i < KI; ++i) f[4 * r + i] = src ? fm[i] + src_dt * fs[i] : fm[i];
    f[4 * r + 3] = 0.0;
}

__global__ void k_membrane_pairs(int64_t npairs, int64_t nmv, int dim, int32_t pin, int64_t n_entries,
                                 int64_t n_cross, const int32_t* __restrict__ mp_ptr, const int32_t* __restrict__ mpf,
                                 const int32_t* __restrict__ tgt, const int32_t* __restrict__ mv_g,
                                 const int32_t* __restrict__ fmv, const double* __restrict__ area,
                                 const double* __restrict__ mf, double* __restrict__ e, double* __restrict__ xe) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= npairs) return;
    const int m = dim - 1;
    double vi[KI] = {0, 0, 0}, ve[KI] = {0, 0, 0};
    for (int q = mp_ptr[t]; q < mp_ptr[t + 1]; ++q) {
        int32_t pk = mpf[q];
        int64_t f = pk >> 4;
        int sa = (pk >> 2) & 3, sb = pk & 3;
        double A = area[f];
        for (int c = 0; c < dim; ++c) {
            int64_t mvc = fmv[f * dim + c];
            double W = A * moment3(m, c, sa, sb);
            for (int k = 0; k < KI; ++k) {
                vi[k] += W * mf[(1 + k) * nmv + mvc];
                ve[k] += W * mf[(4 + k) * nmv + mvc];
            }
        }
    }
    const int32_t* tg = tgt + 4 * t;
    for (int k = 0; k < KI; ++k) {
        e[k * n_entries + tg[0]] += vi[k];
        e[k * n_entries + tg[1]] += ve[k];
        xe[k * n_cross + tg[2]] = -vi[k];
        xe[k * n_cross + tg[3]] = -ve[k];
    }
}

__global__ void k_membrane_rhs(StepParams sp, int64_t nmv, int dim, int32_t pin, const int32_t* __restrict__ mv_g,
                               const int32_t* __restrict__ mvf_ptr, const int32_t* __restrict__ mvf,
                               const int32_t* __restrict__ fmv, const double* __restrict__ area,
                               const int32_t* __restrict__ fmodel, const double* __restrict__ fgleak,
                               const uint8_t* __restrict__ fmask, const double* __restrict__ mf,
                               double* __restrict__ f) {
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= nmv) return;
    const int m = dim - 1;
    double intI[KI] = {0, 0, 0}, cphi_i[KI] = {0, 0, 0}, cphi_e[KI] = {0, 0, 0}, intPhi = 0;
    for (int q = mvf_ptr[a]; q < mvf_ptr[a + 1]; ++q) {
        int64_t fid = mvf[q] >> 2;
        int s = mvf[q] & 3;
        double A = area[fid];
        const bool hh = fmodel[fid] == KNP_MODEL_HH, kir = fmodel[fid] == KNP_MODEL_KIR;
        double gst = fmask[fid] ? sp.g_stim : 0.0;
        double gl[KI];
        for (int k = 0; k < KI; ++k) gl[k] = fgleak[fid * KI + k];
        for (int c = 0; c < dim; ++c) {
            int64_t mc = fmv[fid * dim + c];
            double Mcs = A * moment2(m, c, s);
            double I[KI];
            for (int k = 0; k < KI; ++k) I[k] = gl[k] * mf[(7 + k) * nmv + mc];
            I[sp.ion_na] += gst * mf[(7 + sp.ion_na) * nmv + mc];
            if (hh) {
                I[sp.ion_na] += sp.gbar_na * mf[10 * nmv + mc];
                I[sp.ion_k] += sp.gbar_k * mf[11 * nmv + mc];
            }
            if (kir) {
                // rectified K leak and the pump: 3 F z_Na j out of Na, -2 F z_K j in K
                const double j = mf[13 * nmv + mc];
                I[sp.ion_k] = gl[sp.ion_k] * mf[12 * nmv + mc] - 2.0 * sp.F * sp.z[sp.ion_k] * j;
                I[sp.ion_na] += 3.0 * sp.F * sp.z[sp.ion_na] * j;
            }
            for (int k = 0; k < KI; ++k) intI[k] += Mcs * I[k];
            intPhi += Mcs * mf[mc];
            for (int b = 0; b < dim; ++b) {
                int64_t mb = fmv[fid * dim + b];
                double W = A * moment3(m, c, b, s) * mf[mb];
                for (int k = 0; k < KI; ++k) {
                    cphi_i[k] += W * mf[(1 + k) * nmv + mc];
                    cphi_e[k] += W * mf[(4 + k) * nmv + mc];
                }
            }
        }
    }
    int64_t gi = mv_g[a], ge = mv_g[nmv + a];
    double Itot = 0;
    for (int k = 0; k < KI; ++k) {
        double jk = sp.dt * intI[k] / (sp.F * sp.z[k]);
        f[4 * gi + k] -= jk - cphi_i[k];
        f[4 * ge + k] += jk - cphi_e[k];
        Itot += intI[k];
    }
    double hphi = (sp.dt * Itot - sp.Cm * intPhi) / sp.F;
    f[4 * gi + 3] -= hphi;
    if (ge != pin) f[4 * ge + 3] += hphi;
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ---- P2 elements (Section 3.3 with p = 2) -------------------------------------------------------
// The membrane update, the row pass and the edge sums are the P1 kernels; the element pair values
// of A_r^{k} and the membrane integrals with the P2 facet basis are computed here.

__constant__ P2Dev c_p2[2];   // element dimension 2 and 3

// V[k][e * npairs + p] = int_T [k]^{n-1} grad phi_j . grad phi_l for the off-diagonal local pair p
// = (j, l) of element e (p2_pair_values).
template <int D>
__global__ void __launch_bounds__(128) k_p2_elem_pairs(int64_t ne, const int32_t* __restrict__ eln,
                                                       const double* __restrict__ elg, const double* __restrict__ u,
                                                       double* __restrict__ V) {
    constexpr int NPE = (D + 1) * (D + 2) / 2;
    constexpr int NPAIR = NPE * (NPE - 1) / 2;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= ne) return;
    double G[16];
    for (int i = 0; i < 16; ++i) G[i] = elg[e * 16 + i];
    int32_t g[NPE];
    for (int j = 0; j < NPE; ++j) g[j] = eln[e * NPE + j];
    const int64_t nslot = ne * NPAIR;
    for (int k = 0; k < KI; ++k) {
        double c[NPE], out[NPAIR];
        for (int j = 0; j < NPE; ++j) c[j] = u[4 * (int64_t)g[j] + k];
        p2_pair_values<D>(c_p2[D - 2], G, c, out);
        for (int p = 0; p < NPAIR; ++p) V[k * nslot + e * NPAIR + p] = out[p];
    }
}

// C_r^k-weighted P2 membrane mass on same-region and cross-region entries (cf. k_membrane_pairs)
template <int D>
__global__ void k_membrane_pairs_p2(int64_t npairs, int64_t nmv, int64_t n_entries, int64_t n_cross,
                                    const int32_t* __restrict__ mp_ptr, const int32_t* __restrict__ mpf,
                                    const int32_t* __restrict__ tgt, const int32_t* __restrict__ fmv,
                                    const double* __restrict__ area, const double* __restrict__ mf,
                                    double* __restrict__ e, double* __restrict__ xe) {
    constexpr int NFN = D * (D + 1) / 2;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= npairs) return;
    const P2Dev& T = c_p2[D - 2];
    double vi[KI] = {0, 0, 0}, ve[KI] = {0, 0, 0};
    for (int q = mp_ptr[t]; q < mp_ptr[t + 1]; ++q) {
        const int32_t pk = mpf[q];
        const int64_t f = pk >> 6;
        const int sa = (pk >> 3) & 7, sb = pk & 7;
        const double A = area[f];
        for (int c = 0; c < NFN; ++c) {
            const int64_t mvc = fmv[f * NFN + c];
            const double W = A * T.ftriple[c][sa][sb];
            for (int k = 0; k < KI; ++k) {
                vi[k] += W * mf[(1 + k) * nmv + mvc];
                ve[k] += W * mf[(4 + k) * nmv + mvc];
            }
        }
    }
    const int32_t* tg = tgt + 4 * t;
    for (int k = 0; k < KI; ++k) {
        e[k * n_entries + tg[0]] += vi[k];
        e[k * n_entries + tg[1]] += ve[k];
        xe[k * n_cross + tg[2]] = -vi[k];
        xe[k * n_cross + tg[3]] = -ve[k];
    }
}

// -int_Gamma g_r^k v and -int_Gamma h_r w at the P2 membrane nodes (cf. k_membrane_rhs)
template <int D>
__global__ void k_membrane_rhs_p2(StepParams sp, int64_t nmv, int32_t pin, const int32_t* __restrict__ mv_g,
                                  const int32_t* __restrict__ mvf_ptr, const int32_t* __restrict__ mvf,
                                  const int32_t* __restrict__ fmv, const double* __restrict__ area,
                                  const int32_t* __restrict__ fmodel, const double* __restrict__ fgleak,
                                  const uint8_t* __restrict__ fmask, const double* __restrict__ mf,
                                  double* __restrict__ f) {
    constexpr int NFN = D * (D + 1) / 2;
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= nmv) return;
    const P2Dev& T = c_p2[D - 2];
    double intI[KI] = {0, 0, 0}, cphi_i[KI] = {0, 0, 0}, cphi_e[KI] = {0, 0, 0}, intPhi = 0;
    for (int q = mvf_ptr[a]; q < mvf_ptr[a + 1]; ++q) {
        const int64_t fid = mvf[q] >> 3;
        const int s = mvf[q] & 7;
        const double A = area[fid];
        const bool hh = fmodel[fid] == KNP_MODEL_HH, kir = fmodel[fid] == KNP_MODEL_KIR;
        const double gst = fmask[fid] ? sp.g_stim : 0.0;
        double gl[KI];
        for (int k = 0; k < KI; ++k) gl[k] = fgleak[fid * KI + k];
        for (int c = 0; c < NFN; ++c) {
            const int64_t mc = fmv[fid * NFN + c];
            const double Mcs = A * T.fmass[c][s];
            double I[KI];
            for (int k = 0; k < KI; ++k) I[k] = gl[k] * mf[(7 + k) * nmv + mc];
            I[sp.ion_na] += gst * mf[(7 + sp.ion_na) * nmv + mc];
            if (hh) {
                I[sp.ion_na] += sp.gbar_na * mf[10 * nmv + mc];
                I[sp.ion_k] += sp.gbar_k * mf[11 * nmv + mc];
            }
            if (kir) {
                const double j = mf[13 * nmv + mc];
                I[sp.ion_k] = gl[sp.ion_k] * mf[12 * nmv + mc] - 2.0 * sp.F * sp.z[sp.ion_k] * j;
                I[sp.ion_na] += 3.0 * sp.F * sp.z[sp.ion_na] * j;
            }
            for (int k = 0; k < KI; ++k) intI[k] += Mcs * I[k];
            intPhi += Mcs * mf[mc];
            for (int b = 0; b < NFN; ++b) {
                const int64_t mb = fmv[fid * NFN + b];
                const double W = A * T.ftriple[c][b][s] * mf[mb];
                for (int k = 0; k < KI; ++k) {
                    cphi_i[k] += W * mf[(1 + k) * nmv + mc];
                    cphi_e[k] += W * mf[(4 + k) * nmv + mc];
                }
            }
        }
    }
    const int64_t gi = mv_g[a], ge = mv_g[nmv + a];
    double Itot = 0;
    for (int k = 0; k < KI; ++k) {
        const double jk = sp.dt * intI[k] / (sp.F * sp.z[k]);
        f[4 * gi + k] -= jk - cphi_i[k];
        f[4 * ge + k] += jk - cphi_e[k];
        Itot += intI[k];
    }
    const double hphi = (sp.dt * Itot - sp.Cm * intPhi) / sp.F;
    f[4 * gi + 3] -= hphi;
    if (ge != pin) f[4 * ge + 3] += hphi;
}

template <int D>
void launch_assembly_p2_dim(knp_problem* P, const StepParams& sp, const double* src) {
    cudaStream_t st = P->stream;
    const int64_t n = P->n_nodes, nmv = P->n_mv, ne = P->n_elem;
    constexpr int NPE = (D + 1) * (D + 2) / 2;
    const int64_t nslot = ne * (NPE * (NPE - 1) / 2);
    count_launch(2 + (nmv ? 2 : 0) + (P->n_edges ? 1 : 0) + (P->n_pairs ? 1 : 0));
    if (nmv) k_membrane_nodes<<<nblk(nmv, 128), 128, 0, st>>>(sp, nmv, P->mv_g.p, P->u.p, P->gates.p, P->gates_new.p,
                                                         P->mfield.p);
    k_p2_elem_pairs<D><<<nblk(ne, 128), 128, 0, st>>>(ne, P->el_nodes.p, P->el_g.p, P->u.p, P->cbar.p);
    if (P->n_edges)
        k_edge_values<<<nblk(P->n_edges), 256, 0, st>>>(P->n_edges, nslot, P->eptr.p, P->einc.p, P->ecoef.p,
                                                        P->cbar.p, P->ak.p);
    k_row_assemble<<<nblk(n, 128), 128, 0, st>>>(sp, n, P->N_i, P->pin, P->sell.n_entries, P->n_edges,
                                            P->sell.slice_ptr.p, P->sell.col.p, P->sell_edge.p, P->sell_m.p,
                                            P->ak.p, P->u.p, src, sp.dt, P->sell_e.p, P->f.p);
    if (P->n_pairs)
        k_membrane_pairs_p2<D><<<nblk(P->n_pairs, 128), 128, 0, st>>>(
            P->n_pairs, nmv, P->sell.n_entries, (int64_t)P->h_xcol.size(), P->mp_ptr.p, P->mpf.p, P->mp_tgt.p,
            P->f_mv.p, P->f_area.p, P->mfield.p, P->sell_e.p, P->xe.p);
    if (nmv)
        k_membrane_rhs_p2<D><<<nblk(nmv, 128), 128, 0, st>>>(sp, nmv, P->pin, P->mv_g.p, P->mvf_ptr.p, P->mvf.p,
                                                        P->f_mv.p, P->f_area.p, P->f_model.p, P->f_gleak.p,
                                                        P->f_mask.p, P->mfield.p, P->f.p);
}

}  // namespace

void p2_upload_tables(cudaStream_t st) {
    static P2Dev host[2];
    static std::once_flag once;
    std::call_once(once, [] {
        host[0] = p2_dev(2);
        host[1] = p2_dev(3);
    });
    KNP_CUDA(cudaMemcpyToSymbolAsync(c_p2, host, sizeof(host), 0, cudaMemcpyHostToDevice, st));
}

namespace {

void launch_assembly_p2(knp_problem* P) {
    StepParams sp = P->sp;
    sp.g_stim = stimulus_at(P->desc, P->t);
    const double t_n = P->t + sp.dt;
    const double* src =
        (P->src.p && P->desc.source_t0 < t_n && t_n <= P->desc.source_t1) ? P->src.p : nullptr;
    ProfScope ps(&P->prof, KC_ASSEMBLY, P->stream);
    if (P->dim == 2)
        launch_assembly_p2_dim<2>(P, sp, src);
    else
        launch_assembly_p2_dim<3>(P, sp, src);
    KNP_CUDA(cudaGetLastError());
    P->assembled = true;
}

}  // namespace

double stimulus_at(const knp_problem_desc& d, double t) {
    switch (d.stim_kind) {
        case KNP_STIM_WINDOW:
            return (t >= d.stim_t0 && t < d.stim_t1) ? d.stim_gbar : 0.0;
        case KNP_STIM_PERIODIC_EXP:
            return d.stim_gbar * std::exp(-std::fmod(t, d.stim_tau) / d.stim_a);
        default:
            return 0.0;
    }
}

void launch_assembly(knp_problem* P) {
    P->assembly_id++;
    if (P->degree == 2) {
        launch_assembly_p2(P);
        return;
    }
    cudaStream_t st = P->stream;
    StepParams sp = P->sp;
    sp.g_stim = stimulus_at(P->desc, P->t);
    const int64_t n = P->n_nodes, nmv = P->n_mv;
    const int nvpe = P->dim + 1;
    ProfScope ps(&P->prof, KC_ASSEMBLY, st);
    count_launch(2 + (nmv ? 2 : 0) + (P->n_edges ? 1 : 0) + (P->n_pairs ? 1 : 0));
    if (nmv) k_membrane_nodes<<<nblk(nmv, 128), 128, 0, st>>>(sp, nmv, P->mv_g.p, P->u.p, P->gates.p, P->gates_new.p,
                                                         P->mfield.p);
    k_elem_means<<<nblk(P->n_elem), 256, 0, st>>>(P->n_elem, nvpe, P->el_nodes.p, P->u.p, P->cbar.p);
    if (P->n_edges)
        k_edge_values<<<nblk(P->n_edges), 256, 0, st>>>(P->n_edges, P->n_elem, P->eptr.p, P->einc.p, P->ecoef.p,
                                                        P->cbar.p, P->ak.p);
    // the bulk source of the step's end time t_n, if any
    const double t_n = P->t + sp.dt;
    const double* src =
        (P->src.p && P->desc.source_t0 < t_n && t_n <= P->desc.source_t1) ? P->src.p : nullptr;
    k_row_assemble<<<nblk(n, 128), 128, 0, st>>>(sp, n, P->N_i, P->pin, P->sell.n_entries, P->n_edges,
                                            P->sell.slice_ptr.p, P->sell.col.p, P->sell_edge.p, P->sell_m.p,
                                            P->ak.p, P->u.p, src, sp.dt, P->sell_e.p, P->f.p);
    if (P->n_pairs)
        k_membrane_pairs<<<nblk(P->n_pairs, 128), 128, 0, st>>>(P->n_pairs, nmv, P->dim, P->pin, P->sell.n_entries,
                                                           (int64_t)P->h_xcol.size(), P->mp_ptr.p, P->mpf.p,
                                                           P->mp_tgt.p, P->mv_g.p, P->f_mv.p, P->f_area.p,
                                                           P->mfield.p, P->sell_e.p, P->xe.p);
    if (nmv)
        k_membrane_rhs<<<nblk(nmv, 128), 128, 0, st>>>(sp, nmv, P->dim, P->pin, P->mv_g.p, P->mvf_ptr.p, P->mvf.p,
                                                  P->f_mv.p, P->f_area.p, P->f_model.p, P->f_gleak.p, P->f_mask.p,
                                                  P->mfield.p, P->f.p);
    KNP_CUDA(cudaGetLastError());
    P->assembled = true;
}

}  // namespace knp
