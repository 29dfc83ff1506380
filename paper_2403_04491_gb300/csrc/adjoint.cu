// Adjoint of one time step (an addition to the method: the paper has no adjoint).
//
// For step n the equations are A_{n-1} u_n = f_n with A_{n-1}, f_n built from (u_{n-1}, w_n,
// g_leak) and w_n = G(w_{n-1}, phi_M(u_{n-1})) (Rush-Larsen, Section 3.2). With
// Phi_n = lambda_n^T (f_n - A_{n-1} u_n) the reverse sweep is
//     A_{n-1}^T lambda_n = dL/du_n + rho_n,
//     gamma_n   = dPhi_n/dw_n + dw_n,                  (dw_n carried from step n+1)
//     rho_{n-1} = dPhi_n/du_{n-1} + (dG_n/dphi_M)^T gamma_n,
//     dw_{n-1}  = (dG_n/dw_{n-1})^T gamma_n,   grad_g += dPhi_n/dg_leak.
// The transposed solve reuses the FGMRES and the P_0 hierarchy (P_0 is symmetric). The
// explicit partials of Phi_n are hand-derived:
//   bulk      d/dc^k:  M lambda^k - tau~^k/(d+1) sum_{T ni v} lambda~^k_T^T A^T phi_T,
//             lambda~^k = lambda^k + z_k lambda^phi (the weighted stiffness uses element means);
//   membrane  through C_r^k(c) = alpha_r^k C_m/(F z_k), E_k(c), phi_M^{n-1} and the gates in
//             the channel driving terms q, per membrane vertex from facet moments;
//   facets    dPhi/dg_leak^k_f = -(dt/F) int_f P1(q_leak^k) Psi_k,
//             Psi_k = sum_r +-_r (Lambda_r^k / z_k + Lambda_r^phi) on Gamma.
#include <algorithm>
#include <cmath>

#include "gmres.h"
#include "problem.h"

namespace knp {

namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ double moment3(int m, int a, int b, int c) {
    int eq = (a == b) + (a == c) + (b == c);
    if (m == 1) return eq == 3 ? 0.25 : 1.0 / 12.0;
    return eq == 3 ? 0.1 : (eq == 1 ? 1.0 / 30.0 : 1.0 / 60.0);
}

__device__ __forceinline__ double moment2(int m, int a, int b) {
    double den = (double)((m + 1) * (m + 2));
    return (a == b ? 2.0 : 1.0) / den;
}

// x / (exp(x) - 1) and its derivative
__device__ __forceinline__ void vtrap_d(double x, double& v, double& dv) {
    if (fabs(x) < 1e-6) {
        v = 1.0 - 0.5 * x + x * x / 12.0;
        dv = -0.5 + x / 6.0;
        return;
    }
    double em = expm1(x), ex = em + 1.0;
    v = x / em;
    dv = (em - x * ex) / (em * em);
}

// HH rates (1/ms) and their V-derivatives, V in mV relative to rest; gates (n, m, h)
__device__ __forceinline__ void hh_rates_d(double V, double a[3], double b[3], double da[3], double db[3]) {
    double v, dv;
    vtrap_d((10.0 - V) / 10.0, v, dv);
    a[0] = 0.1 * v;
    da[0] = 0.1 * dv * (-0.1);
    b[0] = 0.125 * exp(-V / 80.0);
    db[0] = -b[0] / 80.0;
    vtrap_d((25.0 - V) / 10.0, v, dv);
    a[1] = v;
    da[1] = dv * (-0.1);
    b[1] = 4.0 * exp(-V / 18.0);
    db[1] = -b[1] / 18.0;
    a[2] = 0.07 * exp(-V / 20.0);
    da[2] = -a[2] / 20.0;
    double ex = exp((30.0 - V) / 10.0);
    b[2] = 1.0 / (ex + 1.0);
    db[2] = b[2] * b[2] * ex / 10.0;
}

__device__ __forceinline__ double lam_phi(const double* lam, int64_t g, int32_t pin) {
    return g == pin ? 0.0 : lam[4 * g + 3];
}

__global__ void k_adj_elem(int64_t ne, int nvpe, const int32_t* __restrict__ eln, const double* __restrict__ elA,
                           const double* __restrict__ lam, const double* __restrict__ unew, int32_t pin, double z0,
                           double z1, double z2, double* __restrict__ sk) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const double z[3] = {z0, z1, z2};
    double Aphi[4] = {0, 0, 0, 0};
    int64_t g[4];
    for (int j = 0; j < nvpe; ++j) g[j] = eln[e * nvpe + j];
    for (int j = 0; j < nvpe; ++j)
        for (int l = 0; l < nvpe; ++l) {
            double phi = g[l] == pin ? 0.0 : unew[4 * g[l] + 3];
            Aphi[j] += elA[e * 16 + j * 4 + l] * phi;
        }
    for (int k = 0; k < KI; ++k) {
        double s = 0;
        for (int j = 0; j < nvpe; ++j) s += (lam[4 * g[j] + k] + z[k] * lam_phi(lam, g[j], pin)) * Aphi[j];
        sk[k * ne + e] = s;
    }
}

__global__ void k_adj_node(StepParams sp, int64_t n, int64_t N_i, int nvpe, int64_t ne,
                           const int64_t* __restrict__ slice_ptr, const int32_t* __restrict__ col,
                           const int32_t* __restrict__ edge, const double* __restrict__ msv,
                           const int32_t* __restrict__ neptr, const int32_t* __restrict__ nelist,
                           const double* __restrict__ sk, const double* __restrict__ lam, double* __restrict__ rho) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const RegionCoef rc = sp.reg[r < N_i ? 0 : 1];
    int64_t s = r / SELL_C, base = slice_ptr[s] + r % SELL_C, w = (slice_ptr[s + 1] - slice_ptr[s]) / SELL_C;
    double ml[KI] = {0, 0, 0};
    for (int64_t k = 0; k < w; ++k) {
        int64_t pos = base + k * SELL_C;
        if (edge[pos] == -2) continue;
        int64_t c = col[pos];
        double mv = msv[pos];
        for (int q = 0; q < KI; ++q) ml[q] += mv * lam[4 * c + q];
    }
    double ss[KI] = {0, 0, 0};
    for (int t = neptr[r]; t < neptr[r + 1]; ++t)
        for (int q = 0; q < KI; ++q) ss[q] += sk[q * ne + nelist[t]];
    for (int q = 0; q < KI; ++q) rho[4 * r + q] = ml[q] - rc.taut[q] / nvpe * ss[q];
    rho[4 * r + 3] = 0.0;
}

__global__ void k_adj_mem(StepParams sp, int64_t nmv, int dim, int32_t pin, const int32_t* __restrict__ mv_g,
                          const int32_t* __restrict__ mvf_ptr, const int32_t* __restrict__ mvf,
                          const int32_t* __restrict__ fmv, const double* __restrict__ area,
                          const int32_t* __restrict__ fmodel, const double* __restrict__ fgleak,
                          const uint8_t* __restrict__ fmask, const double* __restrict__ u,
                          const double* __restrict__ unew, const double* __restrict__ lam,
                          const double* __restrict__ w_old, const double* __restrict__ w_new,
                          const double* __restrict__ mf, double* __restrict__ rho, double* __restrict__ gam) {
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= nmv) return;
    const int m = dim - 1;
    const int na = sp.ion_na, nk = sp.ion_k;
    int64_t gi = mv_g[a], ge = mv_g[nmv + a];
    double ci[KI], ce[KI], E[KI], wi[KI], we[KI], si = 0, se = 0;
    for (int k = 0; k < KI; ++k) {
        ci[k] = u[4 * gi + k];
        ce[k] = u[4 * ge + k];
        E[k] = sp.R * sp.T / (sp.F * sp.z[k]) * log(ce[k] / ci[k]);
        wi[k] = sp.reg[0].tau[k] * sp.z[k] * sp.z[k];
        we[k] = sp.reg[1].tau[k] * sp.z[k] * sp.z[k];
        si += wi[k] * ci[k];
        se += we[k] * ce[k];
    }
    const double phiMo = mf[a];
    double wn[3], wo[3];
    for (int g = 0; g < 3; ++g) {
        wn[g] = w_new[g * nmv + a];
        wo[g] = w_old[g * nmv + a];
    }
    double wL[KI] = {0, 0, 0}, wS = 0, wHNa = 0, wHK = 0, dphiM = 0;
    double dCi[KI] = {0, 0, 0}, dCe[KI] = {0, 0, 0};
    for (int q = mvf_ptr[a]; q < mvf_ptr[a + 1]; ++q) {
        int64_t f = mvf[q] >> 2;
        int s = mvf[q] & 3;
        double A = area[f];
        bool hh = fmodel[f] == KNP_MODEL_HH;
        double gst = fmask[f] ? sp.g_stim : 0.0;
        for (int cc = 0; cc < dim; ++cc) {
            int64_t mc = fmv[f * dim + cc];
            int64_t gic = mv_g[mc], gec = mv_g[nmv + mc];
            double Mcs = A * moment2(m, cc, s);
            double Lpi = lam[4 * gic + 3], Lpe = lam_phi(lam, gec, pin);
            double Psi[KI];
            for (int k = 0; k < KI; ++k) Psi[k] = (lam[4 * gic + k] / sp.z[k] + Lpi) - (lam[4 * gec + k] / sp.z[k] + Lpe);
            for (int k = 0; k < KI; ++k) wL[k] += fgleak[f * KI + k] * Mcs * Psi[k];
            wS += gst * Mcs * Psi[na];
            if (hh) {
                wHNa += sp.gbar_na * Mcs * Psi[na];
                wHK += sp.gbar_k * Mcs * Psi[nk];
            }
            // capacitive phi_M^{n-1} term of f^phi
            dphiM += (sp.Cm / sp.F) * Mcs * (Lpi - Lpe);
            for (int bb = 0; bb < dim; ++bb) {
                int64_t mb = fmv[f * dim + bb];
                double W = A * moment3(m, s, bb, cc);
                int64_t gib = mv_g[mb], geb = mv_g[nmv + mb];
                double dphi_b = mf[mb] - (unew[4 * gib + 3] - (geb == pin ? 0.0 : unew[4 * geb + 3]));
                for (int k = 0; k < KI; ++k) {
                    // d/dC_r^k(a) of +-_r int C (phi_M^{n-1} - phi_M^n) Lambda_r^k
                    dCi[k] += W * dphi_b * lam[4 * gic + k];
                    dCe[k] -= W * dphi_b * lam[4 * gec + k];
                    // d/dphi_M^{n-1}(a) of +-_r int C_r^k phi_M^{n-1} Lambda_r^k
                    dphiM += W * (mf[(1 + k) * nmv + mb] * lam[4 * gic + k] - mf[(4 + k) * nmv + mb] * lam[4 * gec + k]);
                }
            }
        }
    }
    // channel terms: Phi contains -(dt/F) sum_k int I^k Psi_k, I^k = sum_c g_c P1(q_c)
    const double fac = -sp.dt / sp.F;
    double dE[KI] = {0, 0, 0}, dw[3] = {0, 0, 0};
    for (int k = 0; k < KI; ++k) {
        dphiM += fac * wL[k];
        dE[k] -= fac * wL[k];
    }
    dphiM += fac * wS;
    dE[na] -= fac * wS;
    {
        double dr = phiMo - E[na];
        double G = wn[1] * wn[1] * wn[1] * wn[2];
        dphiM += fac * wHNa * G;
        dE[na] -= fac * wHNa * G;
        dw[1] += fac * wHNa * 3.0 * wn[1] * wn[1] * wn[2] * dr;
        dw[2] += fac * wHNa * wn[1] * wn[1] * wn[1] * dr;
    }
    {
        double dr = phiMo - E[nk];
        double n2 = wn[0] * wn[0];
        dphiM += fac * wHK * n2 * n2;
        dE[nk] -= fac * wHK * n2 * n2;
        dw[0] += fac * wHK * 4.0 * n2 * wn[0] * dr;
    }
    // gates: w_n = winf + (w_{n-1} - winf) D^N, D = exp(-(a+b) h), rates at V = 1e3 (phi_M^{n-1} - phi_rest)
    {
        double V = 1e3 * (phiMo - sp.phi_rest);
        double al[3], be[3], dal[3], dbe[3];
        hh_rates_d(V, al, be, dal, dbe);
        const double h = 1e3 * sp.dt / sp.n_ode;
        for (int g = 0; g < 3; ++g) {
            double gamma = dw[g] + gam[g * nmv + a];
            double sab = al[g] + be[g];
            double winf = al[g] / sab;
            double dwinf = (dal[g] * be[g] - al[g] * dbe[g]) / (sab * sab);
            double DN = exp(-sab * h * sp.n_ode);
            double dwn_dV = dwinf * (1.0 - DN) - (wo[g] - winf) * sp.n_ode * h * DN * (dal[g] + dbe[g]);
            dphiM += gamma * 1e3 * dwn_dV;
            gam[g * nmv + a] = DN * gamma;
        }
    }
    // E_k = RT/(F z_k) ln(c_e / c_i); C_r^k = C_m/(F z_k) w_k c_k / sum_l w_l c_l
    double dci[KI], dce[KI];
    for (int k = 0; k < KI; ++k) {
        double rt = sp.R * sp.T / (sp.F * sp.z[k]);
        dci[k] = -dE[k] * rt / ci[k];
        dce[k] = dE[k] * rt / ce[k];
    }
    for (int mm = 0; mm < KI; ++mm)
        for (int k = 0; k < KI; ++k) {
            double cfac = sp.Cm / (sp.F * sp.z[k]);
            double ai = wi[k] * ci[k] / si, ae = we[k] * ce[k] / se;
            dci[mm] += dCi[k] * cfac * (wi[mm] / si) * ((k == mm ? 1.0 : 0.0) - ai);
            dce[mm] += dCe[k] * cfac * (we[mm] / se) * ((k == mm ? 1.0 : 0.0) - ae);
        }
    for (int k = 0; k < KI; ++k) {
        rho[4 * gi + k] += dci[k];
        rho[4 * ge + k] += dce[k];
    }
    rho[4 * gi + 3] += dphiM;
    rho[4 * ge + 3] -= dphiM;
}

__global__ void k_adj_facet(StepParams sp, int64_t nf, int64_t nmv, int dim, int32_t pin,
                            const int32_t* __restrict__ mv_g, const int32_t* __restrict__ fmv,
                            const double* __restrict__ area, const double* __restrict__ lam,
                            const double* __restrict__ mf, double* __restrict__ grad) {
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const int m = dim - 1;
    const double fac = -sp.dt / sp.F;
    double acc[KI] = {0, 0, 0};
    for (int cc = 0; cc < dim; ++cc) {
        int64_t mc = fmv[f * dim + cc];
        int64_t gic = mv_g[mc], gec = mv_g[nmv + mc];
        double Lpi = lam[4 * gic + 3], Lpe = lam_phi(lam, gec, pin);
        for (int s = 0; s < dim; ++s) {
            int64_t ms = fmv[f * dim + s];
            double M = area[f] * moment2(m, s, cc);
            for (int k = 0; k < KI; ++k) {
                double Psi = (lam[4 * gic + k] / sp.z[k] + Lpi) - (lam[4 * gec + k] / sp.z[k] + Lpe);
                acc[k] += mf[(7 + k) * nmv + ms] * M * Psi;
            }
        }
    }
    for (int k = 0; k < KI; ++k) grad[f * KI + k] += fac * acc[k];
}

__global__ void k_eq42_in(int64_t Ni, int64_t Ne, const double* __restrict__ a, double* __restrict__ out, int add) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= Ni + Ne) return;
    for (int k = 0; k < 4; ++k) {
        double v = g < Ni ? a[(int64_t)k * Ni + g] : a[4 * Ni + (int64_t)k * Ne + (g - Ni)];
        out[4 * g + k] = add ? out[4 * g + k] + v : v;
    }
}

__global__ void k_eq42_out(int64_t Ni, int64_t Ne, const double* __restrict__ in, double* __restrict__ a) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= Ni + Ne) return;
    for (int k = 0; k < 4; ++k) {
        if (g < Ni)
            a[(int64_t)k * Ni + g] = in[4 * g + k];
        else
            a[4 * Ni + (int64_t)k * Ne + (g - Ni)] = in[4 * g + k];
    }
}

}  // namespace

struct AdjointWork {
    DArray<double> elA;       // [n_elem][16] element stiffness
    DArray<int32_t> neptr, nelist;
    DArray<double> sk;        // [3][n_elem]
    DArray<double> rho, lam, rhs, unew, gam, grad, tmp;
    int64_t steps = 0;
    knp_solve_stats last{};
};

void adjoint_free(AdjointWork* w) { delete w; }

void build_problem_stiffness(knp_problem* P, std::vector<double>& elA, std::vector<int32_t>& neptr,
                             std::vector<int32_t>& nelist);

void adjoint_begin(knp_problem* P) {
    KNP_REQUIRE(P->degree == 1, KNP_ERR_INVALID_ARG, "the adjoint step covers P1 elements; this problem is P2");
    for (int32_t v : P->facet_model)
        KNP_REQUIRE(v != KNP_MODEL_KIR, KNP_ERR_INVALID_ARG,
                    "the adjoint step covers leak and HH facets; this problem has Kir-Na/K facets");
    if (!P->adj) {
        auto* W = new AdjointWork();
        P->adj = W;
        std::vector<double> elA;
        std::vector<int32_t> neptr, nelist;
        build_problem_stiffness(P, elA, neptr, nelist);
        cudaStream_t st = P->stream;
        W->elA.upload(elA, st);
        W->neptr.upload(neptr, st);
        W->nelist.upload(nelist, st);
        W->sk.alloc(3 * P->n_elem);
        for (DArray<double>* v : {&W->rho, &W->lam, &W->rhs, &W->unew, &W->tmp}) v->alloc(4 * P->n_nodes);
        W->gam.alloc(std::max<int64_t>(1, 3 * P->n_mv));
        W->grad.alloc(std::max<int64_t>(1, 3 * P->nf));
    }
    AdjointWork* W = P->adj;
    for (DArray<double>* v : {&W->rho, &W->lam, &W->gam, &W->grad}) v->zero(P->stream);
    W->steps = 0;
}

void adjoint_step(knp_problem* P, bool device, const double* u_n, const double* dLdu, const knp_solve_opts& o,
                  knp_solve_stats& stats) {
    KNP_REQUIRE(P->adj, KNP_ERR_STATE, "knp_adjoint_begin has not been called");
    KNP_REQUIRE(P->amg, KNP_ERR_STATE, "knp_amg_setup has not been called");
    AdjointWork& W = *P->adj;
    cudaStream_t st = P->stream;
    const int64_t n = P->n_nodes, Ni = P->N_i, Ne = P->N_e;
    const double *du = u_n, *dg = dLdu;
    DArray<double> hu, hg;
    if (!device) {
        std::vector<double> a(u_n, u_n + 4 * n), b(dLdu, dLdu + 4 * n);
        hu.upload(a, st);
        hg.upload(b, st);
        du = hu.p;
        dg = hg.p;
    }
    count_launch(2);
    k_eq42_in<<<nblk(n, 256), 256, 0, st>>>(Ni, Ne, du, W.unew.p, 0);
    KNP_CUDA(cudaMemcpyAsync(W.rhs.p, W.rho.p, 4 * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    k_eq42_in<<<nblk(n, 256), 256, 0, st>>>(Ni, Ne, dg, W.rhs.p, 1);
    // A_{n-1}, f_n and w_n from the current state (u_{n-1}, w_{n-1}, t_{n-1})
    launch_assembly(P);
    knp_status_detail det = fgmres(P, o, stats, W.lam.p, W.rhs.p, true);
    KNP_REQUIRE(det.code == KNP_OK, det.code, "transposed GMRES did not converge (%d iterations)", det.iterations);
    StepParams sp = P->sp;
    sp.g_stim = stimulus_at(P->desc, P->t);
    const int nvpe = P->dim + 1;
    count_launch(2 + (P->n_mv ? 1 : 0) + (P->nf ? 1 : 0));
    k_adj_elem<<<nblk(P->n_elem, 256), 256, 0, st>>>(P->n_elem, nvpe, P->el_nodes.p, W.elA.p, W.lam.p, W.unew.p,
                                                     P->pin, sp.z[0], sp.z[1], sp.z[2], W.sk.p);
    k_adj_node<<<nblk(n, 128), 128, 0, st>>>(sp, n, Ni, nvpe, P->n_elem, P->sell.slice_ptr.p, P->sell.col.p,
                                             P->sell_edge.p, P->sell_m.p, W.neptr.p, W.nelist.p, W.sk.p, W.lam.p,
                                             W.rho.p);
    if (P->n_mv)
        k_adj_mem<<<nblk(P->n_mv, 128), 128, 0, st>>>(sp, P->n_mv, P->dim, P->pin, P->mv_g.p, P->mvf_ptr.p,
                                                      P->mvf.p, P->f_mv.p, P->f_area.p, P->f_model.p, P->f_gleak.p,
                                                      P->f_mask.p, P->u.p, W.unew.p, W.lam.p, P->gates.p,
                                                      P->gates_new.p, P->mfield.p, W.rho.p, W.gam.p);
    if (P->nf)
        k_adj_facet<<<nblk(P->nf, 128), 128, 0, st>>>(sp, P->nf, P->n_mv, P->dim, P->pin, P->mv_g.p, P->f_mv.p,
                                                      P->f_area.p, W.lam.p, P->mfield.p, W.grad.p);
    KNP_CUDA(cudaGetLastError());
    if (!device) KNP_CUDA(cudaStreamSynchronize(st));
    W.steps++;
    W.last = stats;
}

void adjoint_get(knp_problem* P, bool device, double* dLdu0, double* dLdw0, double* grad, double* lambda) {
    KNP_REQUIRE(P->adj, KNP_ERR_STATE, "knp_adjoint_begin has not been called");
    AdjointWork& W = *P->adj;
    cudaStream_t st = P->stream;
    const int64_t n = P->n_nodes;
    auto out_vec = [&](const DArray<double>& v, double* dst) {
        if (!dst) return;
        if (device) {
            count_launch();
            k_eq42_out<<<nblk(n, 256), 256, 0, st>>>(P->N_i, P->N_e, v.p, dst);
        } else {
            DArray<double> tmp;
            tmp.alloc(4 * n);
            count_launch();
            k_eq42_out<<<nblk(n, 256), 256, 0, st>>>(P->N_i, P->N_e, v.p, tmp.p);
            KNP_CUDA(cudaMemcpyAsync(dst, tmp.p, 4 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
            KNP_CUDA(cudaStreamSynchronize(st));
        }
    };
    out_vec(W.rho, dLdu0);
    out_vec(W.lam, lambda);
    auto kind = device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (dLdw0 && P->n_mv) KNP_CUDA(cudaMemcpyAsync(dLdw0, W.gam.p, 3 * P->n_mv * sizeof(double), kind, st));
    if (grad && P->nf) KNP_CUDA(cudaMemcpyAsync(grad, W.grad.p, 3 * P->nf * sizeof(double), kind, st));
    KNP_CUDA(cudaStreamSynchronize(st));
}

}  // namespace knp
