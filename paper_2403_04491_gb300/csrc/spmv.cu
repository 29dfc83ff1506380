// y = A_{n-1} x on the node-block structure of Section 4.1.
//
// Per directed same-region entry (j, l) the operator stores five numbers: the mass
// m_jl and stiffness a_jl (static) and e^k_jl = tau~_r^k A_r^{k,n-1}_jl + [C_r^k M_{r,Gamma}]_jl
// (per step). The 4x4 node block of A_r^n is then
//     c^k row:  (m + tau_r^k a) on c^k,   e^k on phi_r
//     phi row:  z_k tau_r^k a on c^k,     sum_k z_k e^k on phi_r
// because sum_k z_k C_r^k = C_m/F (sum_k alpha_r^k = 1). Cross-region membrane entries
// (B_rq) carry -[C_r^k M_{rq,Gamma}] in the same e^k slot with m = a = 0.
//
// GB300 issues FP64 at 1/64 of its FP32 rate, so the forward product is bound by FP64 FMAs, not
// by bytes. It therefore reads the static per-ion sums g^k = m + tau_r^k a (folded once at
// problem creation) and, for the potential row, a per-node w = sum_k z_k tau_r^k x^k made by a
// small pass over the nodes first:
//     c^k row:  sum g^k x^k + sum e^k phi,     phi row:  sum a w + sum_k z_k (sum e^k phi),
// seven FMAs per stored entry (g^k x^k, e^k phi, a w) for 60 bytes, where m, a with the
// per-row tau take nine for 44 bytes. The transposed product keeps the m, a form.
// One thread per row; the sliced-ELL layout makes the value loads of a warp contiguous.
//
// Point pin (Remark 4.1): the stored values keep the phi_e column of the pinned node (so the
// same-region values stay symmetric and serve the transpose too); both kernels treat that
// column as zero and give the pinned phi_e row the identity.
#include <algorithm>

#include "problem.h"

namespace knp {

namespace {

struct OpArgs {
    int64_t n, N_i, n_entries;
    int32_t pin;
    const int64_t* slice_ptr;
    const int32_t* col;
    const double* m;
    const double* a;
    const double* e;
    const double* g;        // [3][n_entries] g^k = m + tau_r^k a of the entry's region (static)
    const double* w;        // [n] sum_k z_k tau_r^k x^k per node (made by k_op_w)
    const int32_t* xptr;
    const int32_t* xcol;
    const double* xe;
    int64_t n_cross;
    const int32_t* xtptr;   // transposed cross-region entries: row -> (source row, value index)
    const int32_t* xtrow;
    const int32_t* xtidx;
    double tau[2][KI];
    double z[KI];
};

// w[c] = sum_k z_k tau_r^k x^k[c], r the region of node c
__global__ void k_op_w(OpArgs A, const double* __restrict__ x, double* __restrict__ w) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= A.n) return;
    const int reg = c < A.N_i ? 0 : 1;
    const double2* xp = reinterpret_cast<const double2*>(x + 4 * c);
    const double2 x01 = xp[0], x23 = xp[1];
    w[c] = A.z[0] * A.tau[reg][0] * x01.x + A.z[1] * A.tau[reg][1] * x01.y + A.z[2] * A.tau[reg][2] * x23.x;
}

// y = rowscale .* (b - A x)  (b, rowscale optional); needs w = k_op_w(x)
__global__ void __launch_bounds__(128) k_op_apply(OpArgs A, const double* __restrict__ x, double* __restrict__ y,
                                                  const double* __restrict__ rowscale, const double* __restrict__ b) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= A.n) return;
    int64_t s = r / SELL_C;
    int64_t base = A.slice_ptr[s] + r % SELL_C;
    int64_t w = (A.slice_ptr[s + 1] - A.slice_ptr[s]) / SELL_C;
    double ag[KI] = {0, 0, 0}, ae[KI] = {0, 0, 0}, aw = 0.0;
    for (int64_t k = 0; k < w; ++k) {
        int64_t pos = base + k * SELL_C;
        int64_t c = A.col[pos];
        const double2* xp = reinterpret_cast<const double2*>(x + 4 * c);
        double2 x01 = xp[0], x23 = xp[1];
        double phi = (c == A.pin) ? 0.0 : x23.y;
        ag[0] += A.g[pos] * x01.x;
        ag[1] += A.g[A.n_entries + pos] * x01.y;
        ag[2] += A.g[2 * A.n_entries + pos] * x23.x;
        aw += A.a[pos] * A.w[c];
        ae[0] += A.e[pos] * phi;
        ae[1] += A.e[A.n_entries + pos] * phi;
        ae[2] += A.e[2 * A.n_entries + pos] * phi;
    }
    for (int t = A.xptr[r]; t < A.xptr[r + 1]; ++t) {
        int64_t c = A.xcol[t];
        double phi = (c == A.pin) ? 0.0 : x[4 * c + 3];
        for (int k = 0; k < KI; ++k) ae[k] += A.xe[k * A.n_cross + t] * phi;
    }
    double out[4];
    out[3] = aw;
    for (int k = 0; k < KI; ++k) {
        out[k] = ag[k] + ae[k];
        out[3] += A.z[k] * ae[k];
    }
    if (r == A.pin) out[3] = x[4 * r + 3];
    if (b) {
        for (int k = 0; k < 4; ++k) out[k] = b[4 * r + k] - out[k];
    }
    if (rowscale) {
        for (int k = 0; k < 4; ++k) out[k] *= rowscale[4 * r + k];
    }
    double2* yp = reinterpret_cast<double2*>(y + 4 * r);
    yp[0] = make_double2(out[0], out[1]);
    yp[1] = make_double2(out[2], out[3]);
}

// g^k = m + tau_r^k a per stored entry (padding included, where m = a = 0)
__global__ void k_fold_g(int64_t n, int64_t N_i, int64_t ne, const int64_t* __restrict__ slice_ptr,
                         const double* __restrict__ m, const double* __restrict__ a, double ti0, double ti1, double ti2,
                         double te0, double te1, double te2, double* __restrict__ g) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const bool in = r < N_i;
    const double t[3] = {in ? ti0 : te0, in ? ti1 : te1, in ? ti2 : te2};
    const int64_t s = r / SELL_C, base = slice_ptr[s] + r % SELL_C;
    const int64_t w = (slice_ptr[s + 1] - slice_ptr[s]) / SELL_C;
    for (int64_t k = 0; k < w; ++k) {
        const int64_t pos = base + k * SELL_C;
        for (int q = 0; q < KI; ++q) g[q * ne + pos] = m[pos] + t[q] * a[pos];
    }
}

// y = rowscale .* (b - A^T x): the transposed node block of entry (j, l) is
//     c^k row:  (m + tau^k a) x^k_j + z_k tau^k a x^phi_j,   phi row:  sum_k e^k (x^k_j + z_k x^phi_j)
// with m, a, e symmetric on same-region entries; the cross-region part uses the transposed list.
__global__ void __launch_bounds__(128) k_op_apply_t(OpArgs A, const double* __restrict__ x, double* __restrict__ y,
                                                    const double* __restrict__ rowscale,
                                                    const double* __restrict__ b) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= A.n) return;
    const int reg = r < A.N_i ? 0 : 1;
    int64_t s = r / SELL_C;
    int64_t base = A.slice_ptr[s] + r % SELL_C;
    int64_t w = (A.slice_ptr[s + 1] - A.slice_ptr[s]) / SELL_C;
    double am[KI] = {0, 0, 0}, aa[KI] = {0, 0, 0}, ap = 0.0, ae = 0.0;
    for (int64_t k = 0; k < w; ++k) {
        int64_t pos = base + k * SELL_C;
        int64_t c = A.col[pos];
        const double2* xp = reinterpret_cast<const double2*>(x + 4 * c);
        double2 x01 = xp[0], x23 = xp[1];
        double xc[KI] = {x01.x, x01.y, x23.x};
        double phi = (c == A.pin) ? 0.0 : x23.y;
        double mv = A.m[pos], av = A.a[pos];
        for (int q = 0; q < KI; ++q) {
            am[q] += mv * xc[q];
            aa[q] += av * xc[q];
            ae += A.e[q * A.n_entries + pos] * (xc[q] + A.z[q] * phi);
        }
        ap += av * phi;
    }
    for (int t = A.xtptr[r]; t < A.xtptr[r + 1]; ++t) {
        int64_t j = A.xtrow[t];
        int64_t idx = A.xtidx[t];
        double phi = (j == A.pin) ? 0.0 : x[4 * j + 3];
        for (int q = 0; q < KI; ++q) ae += A.xe[q * A.n_cross + idx] * (x[4 * j + q] + A.z[q] * phi);
    }
    double out[4];
    for (int q = 0; q < KI; ++q) out[q] = am[q] + A.tau[reg][q] * (aa[q] + A.z[q] * ap);
    out[3] = ae;
    if (r == A.pin) out[3] = x[4 * r + 3];
    if (b) {
        for (int q = 0; q < 4; ++q) out[q] = b[4 * r + q] - out[q];
    }
    if (rowscale) {
        for (int q = 0; q < 4; ++q) out[q] *= rowscale[4 * r + q];
    }
    double2* yp = reinterpret_cast<double2*>(y + 4 * r);
    yp[0] = make_double2(out[0], out[1]);
    yp[1] = make_double2(out[2], out[3]);
}

}  // namespace

void op_apply(knp_problem* p, const double* x, double* y, const double* rowscale, const double* b, bool transpose,
              cudaStream_t st) {
    if (st == kProblemStream) st = p->stream;
    OpArgs A;
    A.n = p->n_nodes;
    A.N_i = p->N_i;
    A.n_entries = p->sell.n_entries;
    A.pin = p->pin;
    A.slice_ptr = p->sell.slice_ptr.p;
    A.col = p->sell.col.p;
    A.m = p->sell_m.p;
    A.a = p->sell_a.p;
    A.e = p->sell_e.p;
    A.g = p->sell_g.p;
    A.w = p->op_w.p;
    A.xptr = p->xptr.p;
    A.xcol = p->xcol.p;
    A.xe = p->xe.p;
    A.n_cross = (int64_t)p->h_xcol.size();
    A.xtptr = p->xtptr.p;
    A.xtrow = p->xtrow.p;
    A.xtidx = p->xtidx.p;
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < KI; ++k) A.tau[r][k] = p->sp.reg[r].tau[k];
    for (int k = 0; k < KI; ++k) A.z[k] = p->sp.z[k];
    unsigned blocks = (unsigned)((A.n + 127) / 128);
    ProfScope ps(&p->prof, KC_SPMV, st);
    if (transpose) {
        count_launch();
        k_op_apply_t<<<blocks, 128, 0, st>>>(A, x, y, rowscale, b);
    } else {
        count_launch(2);
        k_op_w<<<(unsigned)((A.n + 255) / 256), 256, 0, st>>>(A, x, p->op_w.p);
        k_op_apply<<<blocks, 128, 0, st>>>(A, x, y, rowscale, b);
    }
    KNP_CUDA(cudaGetLastError());
}

void op_prepare(knp_problem* p, cudaStream_t st) {
    const int64_t n = p->n_nodes, ne = p->sell.n_entries;
    p->sell_g.alloc(std::max<int64_t>(1, 3 * ne));
    p->op_w.alloc(std::max<int64_t>(1, n));
    const RegionCoef& ri = p->sp.reg[0];
    const RegionCoef& re = p->sp.reg[1];
    count_launch();
    k_fold_g<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, p->N_i, ne, p->sell.slice_ptr.p, p->sell_m.p, p->sell_a.p,
                                                          ri.tau[0], ri.tau[1], ri.tau[2], re.tau[0], re.tau[1],
                                                          re.tau[2], p->sell_g.p);
    KNP_CUDA(cudaGetLastError());
}

}  // namespace knp
