// Device-side problem state and the kernels' parameter blocks.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <vector>

#include "common.h"
#include "profile.h"

namespace knp {

#define KNP_CUDA(call)                                                                            \
    do {                                                                                          \
        cudaError_t _e = (call);                                                                  \
        if (_e != cudaSuccess)                                                                    \
            KNP_FAIL(_e == cudaErrorMemoryAllocation ? KNP_ERR_OOM : KNP_ERR_CUDA, "%s: %s (%s:%d)", #call, \
                     cudaGetErrorString(_e), __FILE__, __LINE__);                                 \
    } while (0)

// Owning device array.
template <class T>
struct DArray {
    T* p = nullptr;
    size_t n = 0;
    DArray() = default;
    DArray(const DArray&) = delete;
    DArray& operator=(const DArray&) = delete;
    DArray(DArray&& o) noexcept : p(o.p), n(o.n) {
        o.p = nullptr;
        o.n = 0;
    }
    DArray& operator=(DArray&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            n = o.n;
            o.p = nullptr;
            o.n = 0;
        }
        return *this;
    }
    ~DArray() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void alloc(size_t count) {
        release();
        if (count == 0) return;
        KNP_CUDA(cudaMalloc((void**)&p, count * sizeof(T)));
        n = count;
    }
    void upload(const std::vector<T>& h, cudaStream_t s) {
        alloc(h.size());
        if (n) KNP_CUDA(cudaMemcpyAsync(p, h.data(), n * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    void download(std::vector<T>& h, cudaStream_t s) const {
        h.resize(n);
        if (n) KNP_CUDA(cudaMemcpyAsync(h.data(), p, n * sizeof(T), cudaMemcpyDeviceToHost, s));
    }
    void zero(cudaStream_t s) {
        if (n) KNP_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
    }
};

constexpr int KI = 3;          // ions handled by the kernels
constexpr int NF = KI + 1;     // fields per node
constexpr int SELL_C = 32;     // rows per slice of the sliced-ELL layout

// Sliced ELLPACK pattern (slice height 32, column-major inside a slice).
// Entry k of row r sits at slice_ptr[r/32] + k*32 + r%32. Padding entries
// point at their own row and carry zero values.
struct SellPattern {
    int64_t n_rows = 0, n_slices = 0, n_entries = 0;
    std::vector<int64_t> h_slice_ptr;
    std::vector<int32_t> h_col;
    DArray<int64_t> slice_ptr;
    DArray<int32_t> col;
};

// Physical constants of one region as the kernels see them.
struct RegionCoef {
    double tau[KI];    // tau_r^k = dt D_r^k
    double taut[KI];   // tau~_r^k = tau_r^k z_k / psi
};

struct StepParams {
    double z[KI];
    double R, T, F, Cm, dt, psi;
    RegionCoef reg[2];     // 0 = i, 1 = e
    int32_t ion_na, ion_k;
    double gbar_na, gbar_k, phi_rest;
    int32_t n_ode;
    double g_stim;         // stimulus conductance at t_{n-1}
    // Kir-Na/K (Section 2.4.2): pump constants, E_K^0 and [K]_e^0
    double rho_pump, P_na, P_k, EK0, cKe0;
};

struct AmgHierarchy;        // vcycle.cu
struct GmresWork;           // gmres.cu
struct AdjointWork;         // adjoint.cu
struct PcgWork;             // pcg.cu
struct Deflation;           // deflate.cu

}  // namespace knp

struct knp_problem {
    const knp_mesh* mesh = nullptr;
    cudaStream_t stream = nullptr;
    knp::StepParams sp{};
    knp_problem_desc desc{};
    std::vector<int32_t> facet_model;
    std::vector<double> facet_gleak;
    std::vector<uint8_t> stim_mask;
    std::vector<double> source_v[2];     // bulk source per vertex [n_vertices][n_ions] (i, e); empty = none
    int32_t dim = 0;
    int64_t N_i = 0, N_e = 0, n_nodes = 0, n_mv = 0, nf = 0, n_elem = 0, n_edges = 0, n_pairs = 0, n_edge_inc = 0;
    int32_t pin = -1;               // global node of the pinned phi_e
    int32_t degree = 1;             // polynomial degree p of the Lagrange spaces (1 or 2)
    int32_t npe = 0;                // nodes per element: d+1 (P1) or (d+1)(d+2)/2 (P2)
    int32_t nfn = 0;                // nodes per membrane facet: d (P1) or d(d+1)/2 (P2)
    double t = 0.0;
    int64_t step_index = 0;
    bool assembled = false;

    // operator A (region-internal part in SELL; cross-region membrane part in CSR)
    knp::SellPattern sell;
    knp::DArray<int32_t> sell_edge;      // undirected edge id, -1 diagonal, -2 padding
    knp::DArray<double> sell_m, sell_a;  // static mass and stiffness
    knp::DArray<double> sell_e;          // [3][n_entries] c^k-row phi-col coefficients (per step)
    knp::DArray<double> sell_g;          // [3][n_entries] m + tau_r^k a (static, for the forward product)
    knp::DArray<double> op_w;            // [n] sum_k z_k tau_r^k x^k of the forward product's input
    std::vector<int32_t> h_xptr, h_xcol;
    knp::DArray<int32_t> xptr, xcol;     // cross-region entries, CSR over rows
    knp::DArray<double> xe;              // [3][n_cross]
    knp::DArray<int32_t> xtptr, xtrow, xtidx;   // the cross entries by column: (row, value index)

    // bulk assembly data
    knp::DArray<int32_t> el_nodes;       // [n_elem][dim+1] global node ids
    knp::DArray<double> cbar;            // [3][n_elem] element means of c^k
    knp::DArray<int32_t> eptr, einc;     // edge -> incident elements (CSR)
    knp::DArray<double> ecoef;           // element stiffness entry a^T_jl per incidence
    knp::DArray<double> ak;              // [3][n_edges] weighted stiffness per edge
    // P2 (degree 2): cbar holds [3][n_elem * n_pairs] element pair values of A_r^{k}, einc the
    // (element, local pair) slot of each incidence and ecoef 1
    knp::DArray<double> el_g;            // P2: [n_elem][16] |T| grad lambda_a . grad lambda_b

    // membrane data
    knp::DArray<int32_t> mv_g;           // [2][n_mv] global i-node and e-node of each membrane vertex
    knp::DArray<double> gates;           // [3][n_mv] (n, m, h) of the committed state w_{n-1}
    knp::DArray<double> gates_new;       // [3][n_mv] w_n computed by the last assembly
    knp::DArray<double> mfield;          // [14][n_mv]: phiM, C_i(3), C_e(3), q_leak(3), q_hhna, q_hhk,
                                         // q_kir (Kir-rectified K drive), j_pump
    knp::DArray<int32_t> f_mv;           // [nf][dim] membrane-vertex index of facet vertices
    knp::DArray<double> f_area;
    knp::DArray<int32_t> f_model;
    knp::DArray<double> f_gleak;         // [nf][3]
    knp::DArray<uint8_t> f_mask;
    knp::DArray<int32_t> mvf_ptr, mvf;   // membrane vertex -> incident facets, packed (facet << 2 | local)
    knp::DArray<int32_t> mp_ptr, mpf;    // membrane vertex pair -> shared facets, packed (f << 4 | sa << 2 | sb)
    knp::DArray<int32_t> mp_tgt;         // [n_pairs][4]: SELL pos (i), SELL pos (e), cross pos (i row), cross pos (e row)

    // vectors [n_nodes][4]
    knp::DArray<double> u;               // state u_{n-1} / u_n
    knp::DArray<double> u_hist;          // u_{n-2} for an extrapolated x_0 (allocated on first use)
    bool hist_valid = false;             // u_hist holds the state one step before u
    knp::DArray<double> f;               // right-hand side f_n
    knp::DArray<double> sinv;            // 1/sqrt(diag P_0) (set by knp_amg_setup)
    knp::DArray<double> svec;            // sqrt(diag P_0)
    knp::DArray<double> swt;             // weights of the stopping test: svec, 0 on the pinned phi_e
    mutable knp::DArray<double> stage;   // [4 n] staging copy of host state buffers (Eq. 4.3 layout)
    knp::DArray<double> src;             // bulk source f_r^k at the nodes [n_nodes][4] (empty = none)

    knp::Profiler prof;
    knp::AmgHierarchy* amg = nullptr;
    knp::GmresWork* gw = nullptr;
    knp::AdjointWork* adj = nullptr;
    knp::PcgWork* pcg = nullptr;
    knp::Deflation* defl = nullptr;   // coarse correction of the potentials' near-null modes
    int64_t assembly_id = 0;          // assemblies so far (the correction's data follow the operator)
    ~knp_problem();
};

namespace knp {
// problem.cu
void build_problem_p2(knp_problem* P);
// assemble.cu
void launch_assembly(knp_problem* p);
void p2_upload_tables(cudaStream_t st);
double stimulus_at(const knp_problem_desc& d, double t);
// adjoint.cu
void adjoint_free(AdjointWork* w);
void pcg_free(PcgWork* w);
void adjoint_begin(knp_problem* P);
void adjoint_step(knp_problem* P, bool device, const double* u_n, const double* dLdu, const knp_solve_opts& o,
                  knp_solve_stats& stats);
void adjoint_get(knp_problem* P, bool device, double* dLdu0, double* dLdw0, double* grad, double* lambda);
// spmv.cu
// y = A x (unscaled), or with row scaling / residual; see spmv.cu
// stands for "the problem's own stream" in stream arguments
inline const cudaStream_t kProblemStream = reinterpret_cast<cudaStream_t>(~uintptr_t(0));
// (on `st`, or on the problem's stream when st is the default argument)
void op_apply(knp_problem* p, const double* x, double* y, const double* rowscale, const double* b,
              bool transpose = false, cudaStream_t st = kProblemStream);
// the static per-ion values of the forward product (after the pattern and m, a are on the device)
void op_prepare(knp_problem* p, cudaStream_t st);
void download_state(const knp_problem* p, std::vector<double>& u);
// x_0 of the next solve in u: 2 u_{n-1} - u_{n-2} when extrapolating from a valid history,
// u_{n-1} otherwise; u_hist becomes u_{n-1}
void initial_guess(knp_problem* p, bool extrapolate);
}  // namespace knp
