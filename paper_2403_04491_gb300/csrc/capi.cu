// C ABI of the problem object: creation, assembly, AMG setup, solve, stepping,
// state access and the inspection entry points (see include/knp.h).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "amg.h"
#include "amg_gpu.h"
#include "deflate.h"
#include "gmres.h"
#include "problem.h"
#include "vcycle.h"

namespace knp {
void build_problem(knp_problem* P);
void state_copy_out(const knp_problem* p, bool device, double* c_i, double* phi_i, double* c_e, double* phi_e);
void state_copy_in(knp_problem* p, bool device, const double* c_i, const double* phi_i, const double* c_e,
                   const double* phi_e);

namespace {

// Eq. 4.3 order <-> interleaved node-major layout
int64_t eq42_index(const knp_problem* p, int64_t g, int k) {
    if (g < p->N_i) return (int64_t)k * p->N_i + g;
    return 4 * p->N_i + (int64_t)k * p->N_e + (g - p->N_i);
}

void to_interleaved(const knp_problem* p, const double* a, std::vector<double>& out) {
    out.assign(4 * p->n_nodes, 0.0);
    for (int64_t g = 0; g < p->n_nodes; ++g)
        for (int k = 0; k < 4; ++k) out[4 * g + k] = a[eq42_index(p, g, k)];
}

void from_interleaved(const knp_problem* p, const std::vector<double>& in, double* a) {
    for (int64_t g = 0; g < p->n_nodes; ++g)
        for (int k = 0; k < 4; ++k) a[eq42_index(p, g, k)] = in[4 * g + k];
}

void check_desc(const knp_mesh* m, const knp_problem_desc* d) {
    KNP_REQUIRE(d->n_ions == KI, KNP_ERR_INVALID_ARG, "this build handles exactly %d ions (got %d)", KI, d->n_ions);
    KNP_REQUIRE(d->dt > 0 && std::isfinite(d->dt), KNP_ERR_INVALID_ARG, "dt must be positive");
    KNP_REQUIRE(d->R > 0 && d->T > 0 && d->F > 0 && d->Cm > 0, KNP_ERR_INVALID_ARG, "R, T, F, Cm must be positive");
    for (int k = 0; k < KI; ++k) {
        KNP_REQUIRE(d->z[k] != 0.0, KNP_ERR_INVALID_ARG, "valence z[%d] is zero", k);
        KNP_REQUIRE(d->D_i[k] > 0 && d->D_e[k] > 0, KNP_ERR_INVALID_ARG, "diffusion coefficients must be positive");
        KNP_REQUIRE(d->c_i0[k] > 0 && d->c_e0[k] > 0, KNP_ERR_INVALID_ARG, "initial concentrations must be positive");
    }
    KNP_REQUIRE(d->ion_na >= 0 && d->ion_na < KI && d->ion_k >= 0 && d->ion_k < KI, KNP_ERR_INVALID_ARG,
                "ion_na / ion_k out of range");
    KNP_REQUIRE(d->n_ode >= 1, KNP_ERR_INVALID_ARG, "n_ode must be >= 1");
    KNP_REQUIRE(m->nf() == 0 || (d->facet_model && d->facet_gleak), KNP_ERR_INVALID_ARG,
                "facet_model and facet_gleak are required");
    KNP_REQUIRE(d->stim_kind >= 0 && d->stim_kind <= 2, KNP_ERR_INVALID_ARG, "unknown stimulus kind");
    if (d->stim_kind == KNP_STIM_PERIODIC_EXP)
        KNP_REQUIRE(d->stim_a > 0 && d->stim_tau > 0, KNP_ERR_INVALID_ARG, "stimulus a and tau must be positive");
}

}  // namespace
}  // namespace knp

using namespace knp;

knp_problem::~knp_problem() {
    delete amg;
    gmres_free(gw);
    adjoint_free(adj);
    pcg_free(pcg);
    deflation_free(defl);
}

extern "C" {

knp_status knp_problem_create(const knp_mesh* mesh, const knp_problem_desc* desc, void* stream, knp_problem** out) {
    return guarded([&] {
        KNP_REQUIRE(mesh && desc && out, KNP_ERR_INVALID_ARG, "NULL argument");
        *out = nullptr;
        check_desc(mesh, desc);
        KNP_REQUIRE(desc->degree >= 0 && desc->degree <= 2, KNP_ERR_INVALID_ARG, "degree must be 0, 1 or 2 (got %d)",
                    desc->degree);
        const int32_t degree = desc->degree == 2 ? 2 : 1;
        auto P = std::make_unique<knp_problem>();
        P->mesh = mesh;
        P->stream = (cudaStream_t)stream;
        P->desc = *desc;
        const int64_t nf = mesh->nf();
        P->facet_model.assign(desc->facet_model, desc->facet_model + nf);
        P->facet_gleak.assign(desc->facet_gleak, desc->facet_gleak + nf * KI);
        bool kir = false;
        for (int32_t v : P->facet_model) {
            KNP_REQUIRE(v == KNP_MODEL_LEAK || v == KNP_MODEL_HH || v == KNP_MODEL_KIR, KNP_ERR_INVALID_ARG,
                        "unknown membrane model %d", v);
            kir |= v == KNP_MODEL_KIR;
        }
        if (kir)
            KNP_REQUIRE(desc->rho_pump >= 0 && desc->P_na > 0 && desc->P_k > 0 && desc->c_i0[desc->ion_k] > 0 &&
                            desc->c_e0[desc->ion_k] > 0,
                        KNP_ERR_INVALID_ARG, "Kir-Na/K facets need rho_pump >= 0, P_na, P_k > 0 and positive K "
                                             "initial concentrations");
        // source arrays: per vertex (P1) or per global P2 node (P2)
        const int64_t nv = degree == 2 ? mesh->nv + p2_nodes(*mesh).n_edges : mesh->nv;
        const double* srcs[2] = {desc->source_i, desc->source_e};
        for (int r = 0; r < 2; ++r) {
            if (!srcs[r]) continue;
            P->source_v[r].assign(srcs[r], srcs[r] + nv * KI);
            for (double v : P->source_v[r])
                KNP_REQUIRE(std::isfinite(v), KNP_ERR_INVALID_ARG, "bulk source is not finite");
        }
        KNP_REQUIRE(!(srcs[0] || srcs[1]) || desc->source_t1 >= desc->source_t0, KNP_ERR_INVALID_ARG,
                    "source_t1 < source_t0");
        if (desc->stim_mask)
            P->stim_mask.assign(desc->stim_mask, desc->stim_mask + nf);
        else
            P->stim_mask.assign(nf, 1);
        P->desc.facet_model = nullptr;
        P->desc.facet_gleak = nullptr;
        P->desc.stim_mask = nullptr;
        P->desc.source_i = nullptr;
        P->desc.source_e = nullptr;
        StepParams& sp = P->sp;
        for (int k = 0; k < KI; ++k) sp.z[k] = desc->z[k];
        sp.R = desc->R;
        sp.T = desc->T;
        sp.F = desc->F;
        sp.Cm = desc->Cm;
        sp.dt = desc->dt;
        sp.psi = desc->R * desc->T / desc->F;
        for (int k = 0; k < KI; ++k) {
            sp.reg[0].tau[k] = desc->dt * desc->D_i[k];
            sp.reg[1].tau[k] = desc->dt * desc->D_e[k];
            sp.reg[0].taut[k] = sp.reg[0].tau[k] * desc->z[k] / sp.psi;
            sp.reg[1].taut[k] = sp.reg[1].tau[k] * desc->z[k] / sp.psi;
        }
        sp.ion_na = desc->ion_na;
        sp.ion_k = desc->ion_k;
        sp.gbar_na = desc->gbar_na;
        sp.gbar_k = desc->gbar_k;
        sp.phi_rest = desc->phi_rest;
        sp.n_ode = desc->n_ode;
        sp.rho_pump = desc->rho_pump;
        sp.P_na = desc->P_na;
        sp.P_k = desc->P_k;
        sp.cKe0 = desc->c_e0[desc->ion_k];
        sp.EK0 = (kir) ? desc->R * desc->T / (desc->F * desc->z[desc->ion_k]) *
                             std::log(desc->c_e0[desc->ion_k] / desc->c_i0[desc->ion_k])
                       : 0.0;
        P->degree = degree;
        if (degree == 2)
            build_problem_p2(P.get());
        else
            build_problem(P.get());
        *out = P.release();
    });
}

void knp_problem_destroy(knp_problem* p) {
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    delete p;
}

knp_status knp_sync(knp_problem* p) {
    return guarded([&] {
        KNP_REQUIRE(p, KNP_ERR_INVALID_ARG, "NULL problem");
        KNP_CUDA(cudaStreamSynchronize(p->stream));
    });
}

knp_status knp_assemble_step(knp_problem* p) {
    return guarded([&] {
        KNP_REQUIRE(p, KNP_ERR_INVALID_ARG, "NULL problem");
        launch_assembly(p);
    });
}

knp_status knp_amg_setup(knp_problem* p, const knp_amg_opts* o) {
    return guarded([&] {
        KNP_REQUIRE(p && o, KNP_ERR_INVALID_ARG, "NULL argument");
        KNP_REQUIRE(o->precision == KNP_PREC_FP64 || o->precision == KNP_PREC_FP32, KNP_ERR_INVALID_ARG,
                    "unknown precision");
        KNP_REQUIRE(o->theta >= 0 && o->theta < 1 && o->coarse_max >= 1 && o->max_levels >= 1 &&
                        o->cheb_degree >= 1 && o->cheb_degree <= 8 && o->cheb_ratio > 1 && o->theta_coarse < 1 &&
                        o->p_drop >= 0 && o->p_drop < 1,
                    KNP_ERR_INVALID_ARG, "AMG options out of range");
        KNP_REQUIRE(o->cheb_degree_pre <= 8, KNP_ERR_INVALID_ARG, "AMG options out of range");
        // CG(P_0) needs a symmetric preconditioner: as many steps before the correction as after
        const int pre = o->inner_cg_max_it > 0 ? o->cheb_degree : (o->cheb_degree_pre >= 1 ? o->cheb_degree_pre : 1);
        KNP_REQUIRE(o->inner_cg_max_it >= 0 && (o->inner_cg_max_it == 0 || (o->inner_cg_rtol > 0 && o->inner_cg_rtol < 1)),
                    KNP_ERR_INVALID_ARG, "inner CG options out of range");
        KNP_REQUIRE(o->inner_cg_max_it == 0 || o->precision == KNP_PREC_FP64, KNP_ERR_INVALID_ARG,
                    "CG(P_0) needs the FP64 hierarchy");
        if (!p->assembled) launch_assembly(p);
        cudaStream_t st = p->stream;
        const auto t0 = std::chrono::steady_clock::now();
        // P_0: the field-diagonal blocks of A_0 (Eq. 4.4) on the region-internal pattern, with the
        // pin; also the solver's diagonal scaling S = sqrt(diag P_0)
        DevCsr4d A0;
        DArray<double> strength;
        p0_extract(p, A0, strength);
        AmgSetupOpts so{o->theta, o->coarse_max, o->max_levels, o->cheb_ratio, o->theta_coarse, o->p_drop};
        if (o->host_setup) {
            // the host C++ build of the same algorithm: a reference for the GPU build
            HostCsr4 A0h;
            std::vector<double> sh;
            download(A0, A0h, st);
            strength.download(sh, st);
            KNP_CUDA(cudaStreamSynchronize(st));
            sh.resize(A0.nnz);
            A0 = DevCsr4d();
            strength.release();
            HostHierarchy H;
            amg_build(A0h, sh, p->pin, so, H);
            amg_upload(p, H, o->precision, o->cheb_degree, pre);
        } else {
            const char* cap = std::getenv("KNP_AMG_SHORT_ROW_MAX");
            GpuHierarchy G;
            amg_build_gpu(A0, strength, p->pin, so, G, st, cap ? std::atoi(cap) : 0);
            amg_take_gpu(p, G, o->precision, o->cheb_degree, pre);
        }
        p->amg->inner_cg_max_it = o->inner_cg_max_it;
        p->amg->inner_cg_rtol = o->inner_cg_rtol;
        KNP_CUDA(cudaStreamSynchronize(st));
        p->amg->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    });
}

knp_status knp_amg_setup_info(const knp_problem* p, knp_amg_setup_record* rec) {
    return guarded([&] {
        KNP_REQUIRE(p && rec, KNP_ERR_INVALID_ARG, "NULL argument");
        KNP_REQUIRE(p->amg, KNP_ERR_STATE, "knp_amg_setup has not been called");
        rec->on_gpu = p->amg->setup_on_gpu;
        rec->long_rows_p = p->amg->long_rows_p;
        rec->long_rows_rap = p->amg->long_rows_rap;
        rec->setup_ms = p->amg->setup_ms;
    });
}

knp_status knp_solve(knp_problem* p, const knp_solve_opts* o, knp_solve_stats* stats) {
    knp_status_detail det{KNP_OK, 0, 0, 0};
    knp_status st = guarded([&] {
        KNP_REQUIRE(p && o, KNP_ERR_INVALID_ARG, "NULL argument");
        KNP_REQUIRE(p->assembled, KNP_ERR_STATE, "knp_solve called before knp_assemble_step");
        KNP_REQUIRE(p->amg, KNP_ERR_STATE, "knp_solve called before knp_amg_setup");
        KNP_REQUIRE(o->rtol > 0 && o->restart >= 1 && o->max_it >= 1, KNP_ERR_INVALID_ARG, "solve options out of range");
        knp_solve_stats s{};
        const bool extrapolate = o->x0_extrapolate != 0;
        if (extrapolate) initial_guess(p, p->hist_valid);
        p->hist_valid = false;
        det = fgmres(p, *o, s, p->u.p, p->f.p, false);
        if (stats) *stats = s;
        if (det.code == KNP_OK) {
            // commit the step: gates w_n, t_n
            std::swap(p->gates.p, p->gates_new.p);
            p->t += p->sp.dt;
            p->step_index++;
            p->assembled = false;
            p->hist_valid = extrapolate;
        }
    });
    if (st == KNP_OK && det.code != KNP_OK) {
        set_error("GMRES did not reach rtol within max_it");
        return det.code;
    }
    return st;
}

knp_status knp_step(knp_problem* p, int32_t nsteps, const knp_solve_opts* o, knp_step_stats* per_step) {
    if (!p || !o || nsteps < 0) {
        set_error("NULL argument or negative step count");
        return KNP_ERR_INVALID_ARG;
    }
    for (int32_t s = 0; s < nsteps; ++s) {
        knp_status st = knp_assemble_step(p);
        if (st != KNP_OK) return st;
        knp_solve_stats ss{};
        st = knp_solve(p, o, &ss);
        if (per_step) {
            per_step[s].iterations = ss.iterations;
            per_step[s].true_relres = ss.true_relres;
        }
        if (st != KNP_OK) return st;
    }
    return KNP_OK;
}

knp_status knp_state_get(const knp_problem* p, knp_memspace space, double* c_i, double* phi_i, double* c_e,
                         double* phi_e, double* gates, double* t) {
    return guarded([&] {
        KNP_REQUIRE(p, KNP_ERR_INVALID_ARG, "NULL problem");
        state_copy_out(p, space == KNP_DEVICE, c_i, phi_i, c_e, phi_e);
        if (gates && p->n_mv)
            KNP_CUDA(cudaMemcpyAsync(gates, p->gates.p, 3 * p->n_mv * sizeof(double),
                                     space == KNP_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                     p->stream));
        KNP_CUDA(cudaStreamSynchronize(p->stream));
        if (t) *t = p->t;
    });
}

knp_status knp_state_set(knp_problem* p, knp_memspace space, const double* c_i, const double* phi_i,
                         const double* c_e, const double* phi_e, const double* gates, double t) {
    return guarded([&] {
        KNP_REQUIRE(p, KNP_ERR_INVALID_ARG, "NULL problem");
        state_copy_in(p, space == KNP_DEVICE, c_i, phi_i, c_e, phi_e);
        if (gates && p->n_mv)
            KNP_CUDA(cudaMemcpyAsync(p->gates.p, gates, 3 * p->n_mv * sizeof(double),
                                     space == KNP_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                     p->stream));
        KNP_CUDA(cudaStreamSynchronize(p->stream));
        p->t = t;
        p->assembled = false;
        p->hist_valid = false;
    });
}

knp_status knp_rhs_get(const knp_problem* p, double* rhs) {
    return guarded([&] {
        KNP_REQUIRE(p && rhs, KNP_ERR_INVALID_ARG, "NULL argument");
        KNP_REQUIRE(p->assembled, KNP_ERR_STATE, "no assembled step");
        std::vector<double> f;
        p->f.download(f, p->stream);
        KNP_CUDA(cudaStreamSynchronize(p->stream));
        from_interleaved(p, f, rhs);
    });
}

knp_status knp_apply_operator(knp_problem* p, const double* x, double* y) {
    return guarded([&] {
        KNP_REQUIRE(p && x && y, KNP_ERR_INVALID_ARG, "NULL argument");
        KNP_REQUIRE(p->assembled, KNP_ERR_STATE, "no assembled step");
        std::vector<double> xi, yi(4 * p->n_nodes);
        to_interleaved(p, x, xi);
        DArray<double> dx, dy;
        dx.upload(xi, p->stream);
        dy.alloc(xi.size());
        op_apply(p, dx.p, dy.p, nullptr, nullptr);
        dy.download(yi, p->stream);
        KNP_CUDA(cudaStreamSynchronize(p->stream));
        from_interleaved(p, yi, y);
    });
}

knp_status knp_operator_entries(knp_problem* p, int64_t count, const int64_t* rows, const int64_t* cols,
                                double* vals) {
    return guarded([&] {
        KNP_REQUIRE(p && (count == 0 || (rows && cols && vals)), KNP_ERR_INVALID_ARG, "NULL argument");
        KNP_REQUIRE(p->assembled, KNP_ERR_STATE, "no assembled step");
        std::vector<double> m, a, e, xe;
        p->sell_m.download(m, p->stream);
        p->sell_a.download(a, p->stream);
        p->sell_e.download(e, p->stream);
        p->xe.download(xe, p->stream);
        KNP_CUDA(cudaStreamSynchronize(p->stream));
        const int64_t Ni = p->N_i, Ne = p->N_e, ne = p->sell.n_entries, nx = (int64_t)p->h_xcol.size();
        auto split = [&](int64_t idx, int64_t& g, int& k) {
            KNP_REQUIRE(idx >= 0 && idx < 4 * (Ni + Ne), KNP_ERR_INVALID_ARG, "index %lld out of range", (long long)idx);
            if (idx < 4 * Ni) {
                k = (int)(idx / Ni);
                g = idx % Ni;
            } else {
                idx -= 4 * Ni;
                k = (int)(idx / Ne);
                g = Ni + idx % Ne;
            }
        };
        const SellPattern& S = p->sell;
        for (int64_t q = 0; q < count; ++q) {
            int64_t r, c;
            int kr, kc;
            split(rows[q], r, kr);
            split(cols[q], c, kc);
            const int reg = r < Ni ? 0 : 1;
            const RegionCoef& rc = p->sp.reg[reg];
            double v = 0.0;
            if (r == p->pin && kr == 3) {
                v = (c == r && kc == 3) ? 1.0 : 0.0;
            } else if (c == p->pin && kc == 3) {
                v = 0.0;   // the pinned column
            } else if ((r < Ni) == (c < Ni)) {
                int64_t s = r / SELL_C, base = S.h_slice_ptr[s] + r % SELL_C;
                int64_t w = (S.h_slice_ptr[s + 1] - S.h_slice_ptr[s]) / SELL_C;
                int64_t pos = -1;
                int32_t prev = -1;
                for (int64_t k = 0; k < w; ++k) {
                    int32_t cc = S.h_col[base + k * SELL_C];
                    if (cc <= prev) break;
                    prev = cc;
                    if (cc == c) pos = base + k * SELL_C;
                }
                if (pos >= 0) {
                    if (kr < 3 && kc < 3)
                        v = (kr == kc) ? m[pos] + rc.tau[kr] * a[pos] : 0.0;
                    else if (kr < 3 && kc == 3)
                        v = e[kr * ne + pos];
                    else if (kr == 3 && kc < 3)
                        v = p->sp.z[kc] * rc.tau[kc] * a[pos];
                    else
                        for (int i = 0; i < KI; ++i) v += p->sp.z[i] * e[i * ne + pos];
                }
            } else if (kc == 3) {
                for (int t = p->h_xptr[r]; t < p->h_xptr[r + 1]; ++t)
                    if (p->h_xcol[t] == c) {
                        if (kr < 3)
                            v = xe[kr * nx + t];
                        else
                            for (int i = 0; i < KI; ++i) v += p->sp.z[i] * xe[i * nx + t];
                    }
            }
            vals[q] = v;
        }
    });
}

knp_status knp_apply_preconditioner(knp_problem* p, const double* r, double* z) {
    return guarded([&] {
        KNP_REQUIRE(p && r && z, KNP_ERR_INVALID_ARG, "NULL argument");
        KNP_REQUIRE(p->amg, KNP_ERR_STATE, "knp_amg_setup has not been called");
        std::vector<double> ri, zi(4 * p->n_nodes), ones(4 * p->n_nodes, 1.0);
        to_interleaved(p, r, ri);
        DArray<double> dr, dz, d1;
        dr.upload(ri, p->stream);
        d1.upload(ones, p->stream);
        dz.alloc(ri.size());
        vcycle_apply(p, dr.p, d1.p, dz.p);
        dz.download(zi, p->stream);
        KNP_CUDA(cudaStreamSynchronize(p->stream));
        from_interleaved(p, zi, z);
    });
}

knp_status knp_apply_deflated_preconditioner(knp_problem* p, const double* r, double* z, int32_t transpose) {
    return guarded([&] {
        KNP_REQUIRE(p && r && z, KNP_ERR_INVALID_ARG, "NULL argument");
        KNP_REQUIRE(p->amg, KNP_ERR_STATE, "knp_amg_setup has not been called");
        KNP_REQUIRE(p->assembled, KNP_ERR_STATE, "no assembled step");
        std::vector<double> ri, zi(4 * p->n_nodes), ones(4 * p->n_nodes, 1.0);
        to_interleaved(p, r, ri);
        DArray<double> dr, dz, d1;
        dr.upload(ri, p->stream);
        d1.upload(ones, p->stream);
        dz.alloc(ri.size());
        deflation_prepare(p);
        deflated_precond_apply(p, dr.p, d1.p, dz.p, transpose != 0);
        dz.download(zi, p->stream);
        KNP_CUDA(cudaStreamSynchronize(p->stream));
        from_interleaved(p, zi, z);
    });
}

knp_status knp_problem_set_facet_gleak(knp_problem* p, knp_memspace space, const double* gleak) {
    return guarded([&] {
        KNP_REQUIRE(p && gleak, KNP_ERR_INVALID_ARG, "NULL argument");
        const int64_t nf = p->nf;
        if (nf == 0) return;
        KNP_CUDA(cudaMemcpyAsync(p->f_gleak.p, gleak, nf * KI * sizeof(double),
                                 space == KNP_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p->stream));
        KNP_CUDA(cudaStreamSynchronize(p->stream));
        p->assembled = false;
    });
}

knp_status knp_adjoint_begin(knp_problem* p) {
    return guarded([&] {
        KNP_REQUIRE(p, KNP_ERR_INVALID_ARG, "NULL problem");
        adjoint_begin(p);
    });
}

knp_status knp_adjoint_step(knp_problem* p, knp_memspace space, const double* u_n, const double* dLdu_n,
                            const knp_solve_opts* o, knp_solve_stats* stats) {
    return guarded([&] {
        KNP_REQUIRE(p && u_n && dLdu_n && o, KNP_ERR_INVALID_ARG, "NULL argument");
        KNP_REQUIRE(o->rtol > 0 && o->restart >= 1 && o->max_it >= 1, KNP_ERR_INVALID_ARG, "solve options out of range");
        knp_solve_stats s{};
        adjoint_step(p, space == KNP_DEVICE, u_n, dLdu_n, *o, s);
        if (stats) *stats = s;
    });
}

knp_status knp_adjoint_get(knp_problem* p, knp_memspace space, double* dLdu0, double* dLdw0, double* grad_gleak,
                           double* lambda) {
    return guarded([&] {
        KNP_REQUIRE(p, KNP_ERR_INVALID_ARG, "NULL problem");
        adjoint_get(p, space == KNP_DEVICE, dLdu0, dLdw0, grad_gleak, lambda);
    });
}

knp_status knp_apply_operator_transpose(knp_problem* p, const double* x, double* y) {
    return guarded([&] {
        KNP_REQUIRE(p && x && y, KNP_ERR_INVALID_ARG, "NULL argument");
        KNP_REQUIRE(p->assembled, KNP_ERR_STATE, "no assembled step");
        std::vector<double> xi, yi(4 * p->n_nodes);
        to_interleaved(p, x, xi);
        DArray<double> dx, dy;
        dx.upload(xi, p->stream);
        dy.alloc(xi.size());
        op_apply(p, dx.p, dy.p, nullptr, nullptr, true);
        dy.download(yi, p->stream);
        KNP_CUDA(cudaStreamSynchronize(p->stream));
        from_interleaved(p, yi, y);
    });
}

knp_status knp_amg_info(const knp_problem* p, int32_t* levels, int64_t* nodes, int64_t* nnz, double* op_complexity) {
    return guarded([&] {
        KNP_REQUIRE(p, KNP_ERR_INVALID_ARG, "NULL problem");
        KNP_REQUIRE(p->amg, KNP_ERR_STATE, "knp_amg_setup has not been called");
        if (levels) *levels = p->amg->levels;
        double tot = 0;
        for (int l = 0; l < p->amg->levels; ++l) {
            if (nodes) nodes[l] = p->amg->nodes[l];
            if (nnz) nnz[l] = p->amg->nnz[l];
            tot += (double)p->amg->nnz[l];
        }
        if (op_complexity) *op_complexity = tot / (double)p->amg->nnz[0];
    });
}

}  // extern "C"
