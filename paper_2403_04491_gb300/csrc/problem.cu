// Problem creation: node numbering, the fixed sparsity pattern of A_{n-1} in
// sliced-ELL form, static mass/stiffness values, edge-element incidences for the
// per-step weighted stiffness, membrane tables, and the state accessors.
// (Section 3.3 discretisation; Section 4.1 matrices M_r, A_r, A_r^{k,n},
// M_{r,Gamma}, M_{rq,Gamma}; Section 2.3 initial state.)
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>

#include "p2_pairs.cuh"
#include "problem.h"

namespace knp {

namespace {

// Position of column c in row r of the sliced-ELL pattern (rows sorted by column), -1 if absent.
int64_t sell_find(const SellPattern& S, const std::vector<int32_t>& row_len, int64_t r, int32_t c) {
    int64_t s = r / SELL_C, lane = r % SELL_C;
    int64_t base = S.h_slice_ptr[s] + lane;
    int32_t lo = 0, hi = row_len[r] - 1;
    while (lo <= hi) {
        int32_t mid = (lo + hi) / 2;
        int32_t v = S.h_col[base + (int64_t)mid * SELL_C];
        if (v == c) return base + (int64_t)mid * SELL_C;
        if (v < c)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

double facet_area(const double* x, int dim, const int32_t* v) {
    if (dim == 2) {
        double dx = x[2 * (int64_t)v[1]] - x[2 * (int64_t)v[0]];
        double dy = x[2 * (int64_t)v[1] + 1] - x[2 * (int64_t)v[0] + 1];
        return std::sqrt(dx * dx + dy * dy);
    }
    double a[3], b[3];
    for (int d = 0; d < 3; ++d) {
        a[d] = x[3 * (int64_t)v[1] + d] - x[3 * (int64_t)v[0] + d];
        b[d] = x[3 * (int64_t)v[2] + d] - x[3 * (int64_t)v[0] + d];
    }
    double c0 = a[1] * b[2] - a[2] * b[1], c1 = a[2] * b[0] - a[0] * b[2], c2 = a[0] * b[1] - a[1] * b[0];
    return 0.5 * std::sqrt(c0 * c0 + c1 * c1 + c2 * c2);
}

// |T| and barycentric gradients of a simplex (G[j][d] = d lambda_j / dx_d).
void simplex_geometry(const double* x, int dim, const int32_t* el, double& vol, double G[4][3]) {
    double J[3][3] = {{0}};
    for (int j = 0; j < dim; ++j)
        for (int d = 0; d < dim; ++d) J[d][j] = x[(int64_t)el[j + 1] * dim + d] - x[(int64_t)el[0] * dim + d];
    double inv[3][3];
    double det;
    if (dim == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        inv[0][0] = J[1][1] / det;
        inv[0][1] = -J[0][1] / det;
        inv[1][0] = -J[1][0] / det;
        inv[1][1] = J[0][0] / det;
        vol = std::fabs(det) / 2.0;
    } else {
        det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
              J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
        inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
        inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
        inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
        vol = std::fabs(det) / 6.0;
    }
    // lambda_{1..dim} = rows of J^{-1} applied to (x - x0)
    for (int d = 0; d < dim; ++d) {
        G[0][d] = 0.0;
        for (int j = 0; j < dim; ++j) {
            G[j + 1][d] = inv[j][d];
            G[0][d] -= inv[j][d];
        }
    }
}

__global__ void k_init_state(double* u, int64_t N_i, int64_t n, double ci0, double ci1, double ci2, double ce0,
                             double ce1, double ce2, double phiM0) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= n) return;
    bool in_i = g < N_i;
    u[4 * g + 0] = in_i ? ci0 : ce0;
    u[4 * g + 1] = in_i ? ci1 : ce1;
    u[4 * g + 2] = in_i ? ci2 : ce2;
    u[4 * g + 3] = in_i ? phiM0 : 0.0;
}

__global__ void k_init_gates(double* w, int64_t n_mv, double w0, double w1, double w2) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_mv) return;
    w[i] = w0;
    w[n_mv + i] = w1;
    w[2 * n_mv + i] = w2;
}

// Between the interleaved node-major layout and the API's region, ion-major arrays.
__global__ void k_state_out(const double* u, int64_t N_i, int64_t N_e, double* c_i, double* phi_i, double* c_e,
                            double* phi_e) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= N_i + N_e) return;
    if (g < N_i) {
        if (c_i)
            for (int k = 0; k < KI; ++k) c_i[k * N_i + g] = u[4 * g + k];
        if (phi_i) phi_i[g] = u[4 * g + 3];
    } else {
        int64_t j = g - N_i;
        if (c_e)
            for (int k = 0; k < KI; ++k) c_e[k * N_e + j] = u[4 * g + k];
        if (phi_e) phi_e[j] = u[4 * g + 3];
    }
}

__global__ void k_state_in(double* u, int64_t N_i, int64_t N_e, const double* c_i, const double* phi_i,
                           const double* c_e, const double* phi_e) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= N_i + N_e) return;
    if (g < N_i) {
        if (c_i)
            for (int k = 0; k < KI; ++k) u[4 * g + k] = c_i[k * N_i + g];
        if (phi_i) u[4 * g + 3] = phi_i[g];
    } else {
        int64_t j = g - N_i;
        if (c_e)
            for (int k = 0; k < KI; ++k) u[4 * g + k] = c_e[k * N_e + j];
        if (phi_e) u[4 * g + 3] = phi_e[j];
    }
}

// x_0 of a solve: u <- 2 u_{n-1} - u_{n-2} (extrapolate) or u_{n-1}; h <- u_{n-1}
__global__ void k_initial_guess(int64_t n4, double* __restrict__ u, double* __restrict__ h, int extrapolate) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n4) return;
    const double o = u[i];
    if (extrapolate) u[i] = 2.0 * o - h[i];
    h[i] = o;
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

namespace {

// The region-internal pattern: node -> element incidence, sorted neighbour lists per row, the
// sliced-ELL layout (padding points at its own row), and the undirected entry id of every
// directed entry (-1 diagonal, -2 padding). eln holds npe global node ids per element.
int64_t build_pattern(const std::vector<int32_t>& eln, int npe, int64_t ne, int64_t n, SellPattern& S,
                      std::vector<int32_t>& row_len, std::vector<int32_t>& h_edge) {
    std::vector<int64_t> ne_ptr(n + 1, 0);
    for (int64_t e = 0; e < ne; ++e)
        for (int j = 0; j < npe; ++j) ne_ptr[eln[e * npe + j] + 1]++;
    for (int64_t i = 0; i < n; ++i) ne_ptr[i + 1] += ne_ptr[i];
    std::vector<int32_t> ne_list(ne_ptr[n]);
    {
        std::vector<int64_t> fill(ne_ptr.begin(), ne_ptr.end() - 1);
        for (int64_t e = 0; e < ne; ++e)
            for (int j = 0; j < npe; ++j) ne_list[fill[eln[e * npe + j]]++] = (int32_t)e;
    }
    row_len.assign(n, 0);
    std::vector<std::vector<int32_t>> rows(n);
    for (int64_t r = 0; r < n; ++r) {
        auto& v = rows[r];
        for (int64_t t = ne_ptr[r]; t < ne_ptr[r + 1]; ++t)
            for (int j = 0; j < npe; ++j) v.push_back(eln[(int64_t)ne_list[t] * npe + j]);
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        row_len[r] = (int32_t)v.size();
    }
    S.n_rows = n;
    S.n_slices = (n + SELL_C - 1) / SELL_C;
    S.h_slice_ptr.assign(S.n_slices + 1, 0);
    for (int64_t s = 0; s < S.n_slices; ++s) {
        int32_t w = 0;
        for (int64_t r = s * SELL_C; r < std::min<int64_t>(n, (s + 1) * SELL_C); ++r) w = std::max(w, row_len[r]);
        S.h_slice_ptr[s + 1] = S.h_slice_ptr[s] + (int64_t)w * SELL_C;
    }
    S.n_entries = S.h_slice_ptr[S.n_slices];
    KNP_REQUIRE(S.n_entries < INT32_MAX, KNP_ERR_INVALID_ARG, "pattern too large for 32-bit positions");
    S.h_col.assign(S.n_entries, 0);
    h_edge.assign(S.n_entries, -2);
    for (int64_t s = 0; s < S.n_slices; ++s) {
        int64_t w = (S.h_slice_ptr[s + 1] - S.h_slice_ptr[s]) / SELL_C;
        for (int64_t lane = 0; lane < SELL_C; ++lane) {
            int64_t r = s * SELL_C + lane;
            for (int64_t k = 0; k < w; ++k) {
                int64_t pos = S.h_slice_ptr[s] + k * SELL_C + lane;
                S.h_col[pos] = (r < n && k < row_len[r]) ? rows[r][k] : (int32_t)std::min<int64_t>(r, n - 1);
            }
        }
    }
    int64_t n_edges = 0;
    for (int64_t r = 0; r < n; ++r)
        for (int32_t k = 0; k < row_len[r]; ++k) {
            int32_t c = rows[r][k];
            int64_t pos = S.h_slice_ptr[r / SELL_C] + (int64_t)k * SELL_C + r % SELL_C;
            if (c == r)
                h_edge[pos] = -1;
            else if (c > r)
                h_edge[pos] = (int32_t)n_edges++;
        }
    for (int64_t r = 0; r < n; ++r)
        for (int32_t k = 0; k < row_len[r]; ++k) {
            int32_t c = rows[r][k];
            if (c < r) {
                int64_t pos = S.h_slice_ptr[r / SELL_C] + (int64_t)k * SELL_C + r % SELL_C;
                h_edge[pos] = h_edge[sell_find(S, row_len, c, (int32_t)r)];
            }
        }
    return n_edges;
}

// Membrane tables on the host: the region nodes of each membrane node, the facet node ->
// membrane node map, facet areas, node -> (facet, slot) and pair -> (facet, slot, slot)
// incidences (slots packed with `bits` bits each), and the cross-region CSR with its transpose.
struct MembraneHost {
    std::vector<int32_t> mvg, fmv, mvf_ptr, mvf, mp_ptr, mpf, tgt, xtp, xtr, xti;
    std::vector<double> farea;
    int64_t npairs = 0;
};

void build_membrane(knp_problem* P, const SellPattern& S, const std::vector<int32_t>& row_len,
                    const std::vector<int32_t>& fnodes, int nfn, const std::vector<int32_t>& mnodes,
                    const std::vector<int32_t>& loc_i, const std::vector<int32_t>& loc_e, int bits, MembraneHost& M) {
    const knp_mesh& m = *P->mesh;
    const int dim = m.dim;
    const int64_t n = P->n_nodes, Ni = P->N_i, nmv = (int64_t)mnodes.size(), nf = m.nf();
    M.mvg.resize(2 * nmv);
    for (int64_t a = 0; a < nmv; ++a) {
        int32_t x = mnodes[a];
        M.mvg[a] = loc_i[x];
        M.mvg[nmv + a] = (int32_t)(Ni + loc_e[x]);
    }
    M.fmv.resize(nf * nfn);
    M.farea.resize(nf);
    for (int64_t f = 0; f < nf; ++f) {
        for (int s = 0; s < nfn; ++s) {
            int32_t x = fnodes[f * nfn + s];
            M.fmv[f * nfn + s] = (int32_t)(std::lower_bound(mnodes.begin(), mnodes.end(), x) - mnodes.begin());
        }
        M.farea[f] = facet_area(m.coords.data(), dim, &m.facets[f * dim]);
    }
    M.mvf_ptr.assign(nmv + 1, 0);
    for (int64_t f = 0; f < nf; ++f)
        for (int s = 0; s < nfn; ++s) M.mvf_ptr[M.fmv[f * nfn + s] + 1]++;
    for (int64_t a = 0; a < nmv; ++a) M.mvf_ptr[a + 1] += M.mvf_ptr[a];
    M.mvf.resize(M.mvf_ptr[nmv]);
    {
        std::vector<int32_t> fill(M.mvf_ptr.begin(), M.mvf_ptr.end() - 1);
        for (int64_t f = 0; f < nf; ++f)
            for (int s = 0; s < nfn; ++s) M.mvf[fill[M.fmv[f * nfn + s]]++] = (int32_t)((f << bits) | s);
    }
    // membrane node pairs (a, b) sharing a facet, with the shared facets
    struct PairInc {
        int64_t key;
        int32_t packed;
    };
    std::vector<PairInc> pinc;
    pinc.reserve(nf * nfn * nfn);
    for (int64_t f = 0; f < nf; ++f)
        for (int sa = 0; sa < nfn; ++sa)
            for (int sb = 0; sb < nfn; ++sb) {
                int64_t a = M.fmv[f * nfn + sa], b = M.fmv[f * nfn + sb];
                pinc.push_back({a * nmv + b, (int32_t)((f << (2 * bits)) | (sa << bits) | sb)});
            }
    std::sort(pinc.begin(), pinc.end(), [](const PairInc& x, const PairInc& y) {
        return x.key < y.key || (x.key == y.key && x.packed < y.packed);
    });
    std::vector<int64_t> pair_key;
    M.mp_ptr.assign(1, 0);
    M.mpf.clear();
    for (size_t i = 0; i < pinc.size(); ++i) {
        if (i == 0 || pinc[i].key != pinc[i - 1].key) {
            pair_key.push_back(pinc[i].key);
            M.mp_ptr.push_back(M.mp_ptr.back());
        }
        M.mpf.push_back(pinc[i].packed);
        M.mp_ptr.back()++;
    }
    const int64_t npairs = (int64_t)pair_key.size();
    M.npairs = npairs;
    // cross-region CSR: row gi(a) -> col ge(b) and row ge(a) -> col gi(b)
    std::vector<int32_t>& xp = P->h_xptr;
    std::vector<int32_t>& xc = P->h_xcol;
    xp.assign(n + 1, 0);
    for (int64_t t = 0; t < npairs; ++t) {
        int64_t a = pair_key[t] / nmv;
        xp[M.mvg[a] + 1]++;
        xp[M.mvg[nmv + a] + 1]++;
    }
    for (int64_t r = 0; r < n; ++r) xp[r + 1] += xp[r];
    xc.assign(xp[n], 0);
    M.tgt.resize(4 * npairs);
    {
        std::vector<int32_t> fill(xp.begin(), xp.end() - 1);
        // pairs are sorted by (a, b), so columns within a row come out sorted by b
        for (int64_t t = 0; t < npairs; ++t) {
            int64_t a = pair_key[t] / nmv, b = pair_key[t] % nmv;
            int32_t gia = M.mvg[a], gea = M.mvg[nmv + a], gib = M.mvg[b], geb = M.mvg[nmv + b];
            M.tgt[4 * t + 0] = (int32_t)sell_find(S, row_len, gia, gib);
            M.tgt[4 * t + 1] = (int32_t)sell_find(S, row_len, gea, geb);
            KNP_REQUIRE(M.tgt[4 * t] >= 0 && M.tgt[4 * t + 1] >= 0, KNP_ERR_INVALID_MESH,
                        "membrane facet node pair missing from the region pattern");
            xc[fill[gia]] = geb;
            M.tgt[4 * t + 2] = fill[gia]++;
            xc[fill[gea]] = gib;
            M.tgt[4 * t + 3] = fill[gea]++;
        }
    }
    // transposed cross-region list (used by the transposed operator)
    M.xtp.assign(n + 1, 0);
    M.xtr.resize(xc.size());
    M.xti.resize(xc.size());
    for (size_t t = 0; t < xc.size(); ++t) M.xtp[xc[t] + 1]++;
    for (int64_t r = 0; r < n; ++r) M.xtp[r + 1] += M.xtp[r];
    {
        std::vector<int32_t> fill(M.xtp.begin(), M.xtp.end() - 1);
        for (int64_t r = 0; r < n; ++r)
            for (int32_t t = xp[r]; t < xp[r + 1]; ++t) {
                int32_t q = fill[xc[t]]++;
                M.xtr[q] = (int32_t)r;
                M.xti[q] = t;
            }
    }
}

// The bulk source at the region nodes (source_v indexed by the ids in nodes_i / nodes_e), empty
// without a source.
std::vector<double> node_source(const knp_problem* P, const std::vector<int32_t>& nodes_i,
                                const std::vector<int32_t>& nodes_e) {
    std::vector<double> hs;
    if (P->source_v[0].empty() && P->source_v[1].empty()) return hs;
    hs.assign(4 * P->n_nodes, 0.0);
    for (int r = 0; r < 2; ++r) {
        if (P->source_v[r].empty()) continue;
        const std::vector<int32_t>& ids = r == 0 ? nodes_i : nodes_e;
        const int64_t off = r == 0 ? 0 : P->N_i;
        for (size_t j = 0; j < ids.size(); ++j)
            for (int k = 0; k < KI; ++k) hs[4 * (off + j) + k] = P->source_v[r][(size_t)ids[j] * KI + k];
    }
    return hs;
}

// KNP_DRY_RUN_TABLES=<file>: write the host tables instead of uploading them (see knp.h).
class TableWriter {
  public:
    explicit TableWriter(const char* path) : f_(std::fopen(path, "ab")) {
        KNP_REQUIRE(f_, KNP_ERR_INVALID_ARG, "cannot open %s", path);
    }
    ~TableWriter() { std::fclose(f_); }
    template <class T>
    void put(const char* name, const std::vector<T>& v) {
        const int64_t head[3] = {(int64_t)std::strlen(name), (int64_t)v.size(), (int64_t)sizeof(T)};
        std::fwrite(head, sizeof(head), 1, f_);
        std::fwrite(name, 1, std::strlen(name), f_);
        if (!v.empty()) std::fwrite(v.data(), sizeof(T), v.size(), f_);
    }

  private:
    std::FILE* f_;
};

// Uploads of the operator, assembly and membrane tables, the bulk source, the state vectors and
// u_0, w_0 (and, for P2, the reference tables in constant memory).
void upload_problem(knp_problem* P, const std::vector<int32_t>& h_edge, const std::vector<double>& hm,
                    const std::vector<double>& ha, const std::vector<int32_t>& eln, const std::vector<double>* hg,
                    int64_t cbar_len, const std::vector<int32_t>& e_cnt, const std::vector<int32_t>& h_einc,
                    const std::vector<double>& h_ecoef, const MembraneHost& M, const std::vector<int32_t>& nodes_i,
                    const std::vector<int32_t>& nodes_e) {
    cudaStream_t st = P->stream;
    SellPattern& S = P->sell;
    const int64_t n = P->n_nodes, Ni = P->N_i, nmv = P->n_mv;
    const std::vector<double> hs = node_source(P, nodes_i, nodes_e);
    if (const char* path = std::getenv("KNP_DRY_RUN_TABLES")) {
        {
            TableWriter w(path);
            w.put("info", std::vector<int64_t>{P->degree, P->dim, P->N_i, P->N_e, P->pin, P->n_mv, P->n_elem});
            w.put("slice_ptr", S.h_slice_ptr);
            w.put("col", S.h_col);
            w.put("sell_edge", h_edge);
            w.put("sell_m", hm);
            w.put("sell_a", ha);
            w.put("xptr", P->h_xptr);
            w.put("xcol", P->h_xcol);
            w.put("el_nodes", eln);
            if (hg) w.put("el_g", *hg);
            w.put("eptr", e_cnt);
            w.put("einc", h_einc);
            w.put("ecoef", h_ecoef);
            w.put("mv_g", M.mvg);
            w.put("f_mv", M.fmv);
            w.put("f_area", M.farea);
            w.put("f_model", P->facet_model);
            w.put("f_gleak", P->facet_gleak);
            w.put("f_mask", P->stim_mask);
            w.put("mvf_ptr", M.mvf_ptr);
            w.put("mvf", M.mvf);
            w.put("mp_ptr", M.mp_ptr);
            w.put("mpf", M.mpf);
            w.put("mp_tgt", M.tgt);
            w.put("src", hs);
        }
        KNP_FAIL(KNP_ERR_STATE, "dry run: the problem's host tables were written to %s; no device work", path);
    }
    if (P->degree == 2) p2_upload_tables(st);
    S.slice_ptr.upload(S.h_slice_ptr, st);
    S.col.upload(S.h_col, st);
    P->sell_edge.upload(h_edge, st);
    P->sell_m.upload(hm, st);
    P->sell_a.upload(ha, st);
    op_prepare(P, st);
    P->sell_e.alloc(3 * S.n_entries);
    P->sell_e.zero(st);
    P->xptr.upload(P->h_xptr, st);
    P->xcol.upload(P->h_xcol, st);
    P->xtptr.upload(M.xtp, st);
    P->xtrow.upload(M.xtr, st);
    P->xtidx.upload(M.xti, st);
    P->xe.alloc(std::max<int64_t>(1, 3 * (int64_t)P->h_xcol.size()));
    P->xe.zero(st);
    P->el_nodes.upload(eln, st);
    if (hg) P->el_g.upload(*hg, st);
    P->cbar.alloc(cbar_len);
    P->eptr.upload(e_cnt, st);
    P->einc.upload(h_einc, st);
    P->ecoef.upload(h_ecoef, st);
    P->ak.alloc(std::max<int64_t>(1, 3 * P->n_edges));
    P->mv_g.upload(M.mvg, st);
    P->gates.alloc(3 * nmv);
    P->gates_new.alloc(3 * nmv);
    P->mfield.alloc(14 * nmv);
    P->f_mv.upload(M.fmv, st);
    P->f_area.upload(M.farea, st);
    P->f_model.upload(P->facet_model, st);
    P->f_gleak.upload(P->facet_gleak, st);
    P->f_mask.upload(P->stim_mask, st);
    P->mvf_ptr.upload(M.mvf_ptr, st);
    P->mvf.upload(M.mvf, st);
    P->mp_ptr.upload(M.mp_ptr, st);
    P->mpf.upload(M.mpf, st);
    P->mp_tgt.upload(M.tgt, st);
    if (!hs.empty()) P->src.upload(hs, st);
    P->u.alloc(4 * n);
    P->f.alloc(4 * n);
    P->f.zero(st);
    P->sinv.alloc(4 * n);
    P->svec.alloc(4 * n);
    P->swt.alloc(4 * n);
    const knp_problem_desc& d = P->desc;
    count_launch(nmv ? 2 : 1);
    k_init_state<<<nblk(n), 256, 0, st>>>(P->u.p, Ni, n, d.c_i0[0], d.c_i0[1], d.c_i0[2], d.c_e0[0], d.c_e0[1],
                                          d.c_e0[2], d.phi_M0);
    if (nmv) k_init_gates<<<nblk(nmv), 256, 0, st>>>(P->gates.p, nmv, d.w0[0], d.w0[1], d.w0[2]);
    KNP_CUDA(cudaGetLastError());
    KNP_CUDA(cudaStreamSynchronize(st));
}

}  // namespace

void build_problem(knp_problem* P) {
    const knp_mesh& m = *P->mesh;
    const int dim = m.dim, nvpe = dim + 1;
    const int64_t Ni = (int64_t)m.nodes_i.size(), Ne = (int64_t)m.nodes_e.size();
    const int64_t n = Ni + Ne;
    P->dim = dim;
    P->npe = nvpe;
    P->nfn = dim;
    P->N_i = Ni;
    P->N_e = Ne;
    P->n_nodes = n;
    P->n_mv = (int64_t)m.mverts.size();
    P->nf = m.nf();
    P->n_elem = m.ne;
    P->pin = (int32_t)(Ni + m.loc_e[m.pin_vertex]);

    // ---- elements with global node ids (intracellular first, then extracellular)
    std::vector<int32_t> eln((size_t)m.ne * nvpe);
    std::vector<int32_t> elem_src(m.ne);
    {
        int64_t k = 0;
        for (int32_t e : m.elems_i) {
            for (int j = 0; j < nvpe; ++j) eln[k * nvpe + j] = m.loc_i[m.elems[(int64_t)e * nvpe + j]];
            elem_src[k++] = e;
        }
        for (int32_t e : m.elems_e) {
            for (int j = 0; j < nvpe; ++j) eln[k * nvpe + j] = (int32_t)(Ni + m.loc_e[m.elems[(int64_t)e * nvpe + j]]);
            elem_src[k++] = e;
        }
    }
    SellPattern& S = P->sell;
    std::vector<int32_t> row_len, h_edge;
    const int64_t n_edges = build_pattern(eln, nvpe, m.ne, n, S, row_len, h_edge);
    P->n_edges = n_edges;
    // ---- static M and A, and the edge incidence (element, a^T_jl)
    std::vector<double> hm(S.n_entries, 0.0), ha(S.n_entries, 0.0);
    std::vector<int32_t> e_cnt(n_edges + 1, 0);
    std::vector<double> vol(m.ne);
    std::vector<double> Ael((size_t)m.ne * 16);
    for (int64_t e = 0; e < m.ne; ++e) {
        double G[4][3];
        simplex_geometry(m.coords.data(), dim, &m.elems[(int64_t)elem_src[e] * nvpe], vol[e], G);
        for (int j = 0; j < nvpe; ++j)
            for (int l = 0; l < nvpe; ++l) {
                double s = 0;
                for (int d = 0; d < dim; ++d) s += G[j][d] * G[l][d];
                Ael[e * 16 + j * 4 + l] = vol[e] * s;
            }
    }
    const double mdiag = (dim == 2) ? 1.0 / 6.0 : 1.0 / 10.0;   // (1+1)/((d+1)(d+2))
    const double moff = (dim == 2) ? 1.0 / 12.0 : 1.0 / 20.0;
    for (int64_t e = 0; e < m.ne; ++e) {
        for (int j = 0; j < nvpe; ++j)
            for (int l = 0; l < nvpe; ++l) {
                int32_t r = eln[e * nvpe + j], c = eln[e * nvpe + l];
                int64_t pos = sell_find(S, row_len, r, c);
                hm[pos] += vol[e] * (j == l ? mdiag : moff);
                ha[pos] += Ael[e * 16 + j * 4 + l];
                if (j < l) {
                    int32_t id = h_edge[pos];
                    e_cnt[id + 1]++;
                }
            }
    }
    for (int64_t i = 0; i < n_edges; ++i) e_cnt[i + 1] += e_cnt[i];
    P->n_edge_inc = e_cnt[n_edges];
    std::vector<int32_t> h_einc(e_cnt[n_edges]);
    std::vector<double> h_ecoef(e_cnt[n_edges]);
    {
        std::vector<int32_t> fill(e_cnt.begin(), e_cnt.end() - 1);
        for (int64_t e = 0; e < m.ne; ++e)
            for (int j = 0; j < nvpe; ++j)
                for (int l = j + 1; l < nvpe; ++l) {
                    int32_t r = eln[e * nvpe + j], c = eln[e * nvpe + l];
                    int32_t id = h_edge[sell_find(S, row_len, r, c)];
                    h_einc[fill[id]] = (int32_t)e;
                    h_ecoef[fill[id]] = Ael[e * 16 + j * 4 + l];
                    fill[id]++;
                }
    }
    // ---- membrane (P1: the facet's vertices are its nodes)
    MembraneHost M;
    build_membrane(P, S, row_len, m.facets, dim, m.mverts, m.loc_i, m.loc_e, 2, M);
    P->n_pairs = M.npairs;
    upload_problem(P, h_edge, hm, ha, eln, nullptr, 3 * m.ne, e_cnt, h_einc, h_ecoef, M, m.nodes_i, m.nodes_e);
}

// ---- P2 elements (Section 3.3 with p = 2) ---------------------------------------------------

namespace {

// |T| grad lambda_a . grad lambda_b, and the P2 element mass and stiffness (Section 4.1).
void p2_element(const double* x, int dim, const int32_t* el, const P2Ref& R, double Gm[4][4],
                double Me[P2_NPE_MAX][P2_NPE_MAX], double Ae[P2_NPE_MAX][P2_NPE_MAX]) {
    double vol, G[4][3];
    simplex_geometry(x, dim, el, vol, G);
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            double s = 0.0;
            if (a <= dim && b <= dim)
                for (int d = 0; d < dim; ++d) s += G[a][d] * G[b][d];
            Gm[a][b] = vol * s;
        }
    for (int j = 0; j < R.npe; ++j)
        for (int l = 0; l < R.npe; ++l) {
            double s = 0.0;
            for (int a = 0; a <= dim; ++a)
                for (int b = 0; b <= dim; ++b) s += R.stiff[j][l][a][b] * Gm[a][b];
            Me[j][l] = vol * R.mass[j][l];
            Ae[j][l] = s;
        }
}

}  // namespace

// Problem creation for P2 elements: the same operator layout as build_problem (sliced-ELL
// region pattern with static m, a per entry; cross-region membrane CSR; node-major vectors),
// with P2 nodes. The per-step weighted stiffness comes from element pair values (one per
// element and off-diagonal local pair) summed over the incidences of each undirected entry.
void build_problem_p2(knp_problem* P) {
    const knp_mesh& m = *P->mesh;
    const knp_p2_nodes& t2 = p2_nodes(m);
    const int dim = m.dim, nvpe = dim + 1;
    const P2Ref& R = p2_ref(dim);
    const int npe = R.npe, nfn = R.nfn, npairs = R.npairs;
    const int64_t Ni = (int64_t)t2.nodes_i.size(), Ne = (int64_t)t2.nodes_e.size();
    const int64_t n = Ni + Ne;
    P->dim = dim;
    P->degree = 2;
    P->npe = npe;
    P->nfn = nfn;
    P->N_i = Ni;
    P->N_e = Ne;
    P->n_nodes = n;
    P->n_mv = (int64_t)t2.mnodes.size();
    P->nf = m.nf();
    P->n_elem = m.ne;
    P->pin = (int32_t)(Ni + t2.loc_e[t2.pin_node]);
    KNP_REQUIRE(m.ne * npairs < INT32_MAX, KNP_ERR_INVALID_ARG, "too many P2 element pairs for 32-bit slots");
    KNP_REQUIRE(P->nf < (1 << 25), KNP_ERR_INVALID_ARG, "too many membrane facets for the P2 tables");

    // ---- elements with global node ids (intracellular first, then extracellular)
    std::vector<int32_t> eln((size_t)m.ne * npe);
    std::vector<int32_t> elem_src(m.ne);
    {
        int64_t k = 0;
        for (int32_t e : m.elems_i) {
            for (int j = 0; j < npe; ++j) eln[k * npe + j] = t2.loc_i[t2.elem_nodes[(int64_t)e * npe + j]];
            elem_src[k++] = e;
        }
        for (int32_t e : m.elems_e) {
            for (int j = 0; j < npe; ++j)
                eln[k * npe + j] = (int32_t)(Ni + t2.loc_e[t2.elem_nodes[(int64_t)e * npe + j]]);
            elem_src[k++] = e;
        }
    }
    SellPattern& S = P->sell;
    std::vector<int32_t> row_len, h_edge;
    const int64_t n_edges = build_pattern(eln, npe, m.ne, n, S, row_len, h_edge);
    P->n_edges = n_edges;
    // ---- static M and A; |T| G per element; the (element, pair) incidences of each undirected entry
    std::vector<double> hm(S.n_entries, 0.0), ha(S.n_entries, 0.0), hg((size_t)m.ne * 16);
    std::vector<int32_t> e_cnt(n_edges + 1, 0);
    for (int64_t e = 0; e < m.ne; ++e) {
        double Gm[4][4], Me[P2_NPE_MAX][P2_NPE_MAX], Ae[P2_NPE_MAX][P2_NPE_MAX];
        p2_element(m.coords.data(), dim, &m.elems[(int64_t)elem_src[e] * nvpe], R, Gm, Me, Ae);
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) hg[e * 16 + a * 4 + b] = Gm[a][b];
        for (int j = 0; j < npe; ++j)
            for (int l = 0; l < npe; ++l) {
                int64_t pos = sell_find(S, row_len, eln[e * npe + j], eln[e * npe + l]);
                hm[pos] += Me[j][l];
                ha[pos] += Ae[j][l];
            }
        for (int p = 0; p < npairs; ++p) {
            int64_t pos = sell_find(S, row_len, eln[e * npe + R.pj[p]], eln[e * npe + R.pl[p]]);
            e_cnt[h_edge[pos] + 1]++;
        }
    }
    for (int64_t i = 0; i < n_edges; ++i) e_cnt[i + 1] += e_cnt[i];
    P->n_edge_inc = e_cnt[n_edges];
    std::vector<int32_t> h_einc(e_cnt[n_edges]);
    std::vector<double> h_ecoef(e_cnt[n_edges], 1.0);
    {
        std::vector<int32_t> fill(e_cnt.begin(), e_cnt.end() - 1);
        for (int64_t e = 0; e < m.ne; ++e)
            for (int p = 0; p < npairs; ++p) {
                int32_t id = h_edge[sell_find(S, row_len, eln[e * npe + R.pj[p]], eln[e * npe + R.pl[p]])];
                h_einc[fill[id]++] = (int32_t)(e * npairs + p);
            }
    }
    // ---- membrane: the P2 nodes of Gamma (slots of up to 6 facet nodes: 3 bits)
    MembraneHost M;
    build_membrane(P, S, row_len, t2.facet_nodes, nfn, t2.mnodes, t2.loc_i, t2.loc_e, 3, M);
    P->n_pairs = M.npairs;
    upload_problem(P, h_edge, hm, ha, eln, &hg, 3 * m.ne * npairs, e_cnt, h_einc, h_ecoef, M, t2.nodes_i,
                   t2.nodes_e);
}

// Element contributions to the P2 matrices M_r, A_r and A_r^{c} of one region (host only). The
// weighted stiffness uses the per-step kernel's pair values (p2_pair_values), with each element
// diagonal entry minus its row's off-diagonal sum, as the row pass does for the assembled matrix.
void p2_region_triplets(const knp_mesh& m, int region, const double* c, int32_t* rows, int32_t* cols, double* M,
                        double* A, double* Ac) {
    const knp_p2_nodes& t2 = p2_nodes(m);
    const int dim = m.dim;
    const P2Ref& R = p2_ref(dim);
    const P2Dev& T = p2_dev(dim);
    const int npe = R.npe;
    const std::vector<int32_t>& els = region == 0 ? m.elems_i : m.elems_e;
    const std::vector<int32_t>& loc = region == 0 ? t2.loc_i : t2.loc_e;
    int64_t k = 0;
    for (int32_t e : els) {
        double Gm[4][4], Me[P2_NPE_MAX][P2_NPE_MAX], Ae[P2_NPE_MAX][P2_NPE_MAX];
        p2_element(m.coords.data(), dim, &m.elems[(int64_t)e * (dim + 1)], R, Gm, Me, Ae);
        double Ce[P2_NPE_MAX][P2_NPE_MAX] = {};
        if (Ac) {
            double ce[P2_NPE_MAX], pv[P2_NPAIR_MAX];
            for (int j = 0; j < npe; ++j) ce[j] = c[loc[t2.elem_nodes[(int64_t)e * npe + j]]];
            if (dim == 2)
                p2_pair_values<2>(T, &Gm[0][0], ce, pv);
            else
                p2_pair_values<3>(T, &Gm[0][0], ce, pv);
            for (int p = 0; p < R.npairs; ++p) {
                Ce[R.pj[p]][R.pl[p]] = Ce[R.pl[p]][R.pj[p]] = pv[p];
                Ce[R.pj[p]][R.pj[p]] -= pv[p];
                Ce[R.pl[p]][R.pl[p]] -= pv[p];
            }
        }
        for (int j = 0; j < npe; ++j)
            for (int l = 0; l < npe; ++l, ++k) {
                if (rows) rows[k] = loc[t2.elem_nodes[(int64_t)e * npe + j]];
                if (cols) cols[k] = loc[t2.elem_nodes[(int64_t)e * npe + l]];
                if (M) M[k] = Me[j][l];
                if (A) A[k] = Ae[j][l];
                if (Ac) Ac[k] = Ce[j][l];
            }
    }
}

// Element stiffness matrices [n_elem][4][4] (elements in el_nodes order) and the node -> element
// incidence, for the adjoint of the weighted stiffness A_r^{k}(c).
void build_problem_stiffness(knp_problem* P, std::vector<double>& elA, std::vector<int32_t>& neptr,
                             std::vector<int32_t>& nelist) {
    const knp_mesh& m = *P->mesh;
    const int dim = m.dim, nvpe = dim + 1;
    const int64_t n = P->n_nodes;
    std::vector<int32_t> src;
    src.insert(src.end(), m.elems_i.begin(), m.elems_i.end());
    src.insert(src.end(), m.elems_e.begin(), m.elems_e.end());
    elA.assign(src.size() * 16, 0.0);
    neptr.assign(n + 1, 0);
    std::vector<int32_t> gl(src.size() * nvpe);
    for (size_t e = 0; e < src.size(); ++e) {
        double vol, G[4][3];
        simplex_geometry(m.coords.data(), dim, &m.elems[(int64_t)src[e] * nvpe], vol, G);
        for (int j = 0; j < nvpe; ++j) {
            for (int l = 0; l < nvpe; ++l) {
                double s = 0;
                for (int d = 0; d < dim; ++d) s += G[j][d] * G[l][d];
                elA[e * 16 + j * 4 + l] = vol * s;
            }
            int32_t v = m.elems[(int64_t)src[e] * nvpe + j];
            int32_t g = e < m.elems_i.size() ? m.loc_i[v] : (int32_t)(P->N_i + m.loc_e[v]);
            gl[e * nvpe + j] = g;
            neptr[g + 1]++;
        }
    }
    for (int64_t i = 0; i < n; ++i) neptr[i + 1] += neptr[i];
    nelist.assign(neptr[n], 0);
    std::vector<int32_t> fill(neptr.begin(), neptr.end() - 1);
    for (size_t e = 0; e < src.size(); ++e)
        for (int j = 0; j < nvpe; ++j) nelist[fill[gl[e * nvpe + j]]++] = (int32_t)e;
}

void download_state(const knp_problem* p, std::vector<double>& u) {
    p->u.download(u, p->stream);
    KNP_CUDA(cudaStreamSynchronize(p->stream));
}

void initial_guess(knp_problem* p, bool extrapolate) {
    const int64_t n4 = 4 * (p->N_i + p->N_e);
    if ((int64_t)p->u_hist.n < n4) {
        p->u_hist.alloc(n4);
        extrapolate = false;
    }
    count_launch();
    k_initial_guess<<<nblk(n4), 256, 0, p->stream>>>(n4, p->u.p, p->u_hist.p, extrapolate ? 1 : 0);
    KNP_CUDA(cudaGetLastError());
}

// Host buffers go through a device staging copy in the Eq. 4.3 layout ([c_i (3 N_i), phi_i (N_i),
// c_e (3 N_e), phi_e (N_e)]): one DMA per array (direct from pinned memory) and the same reorder
// kernels as for device buffers, instead of reordering on the host.
static double* state_stage(const knp_problem* p) {
    const int64_t n4 = 4 * (p->N_i + p->N_e);
    if ((int64_t)p->stage.n < n4) p->stage.alloc(n4);
    return p->stage.p;
}

void state_copy_out(const knp_problem* p, bool device, double* c_i, double* phi_i, double* c_e, double* phi_e) {
    const int64_t Ni = p->N_i, Ne = p->N_e, n = Ni + Ne;
    if (device) {
        count_launch();
        k_state_out<<<nblk(n), 256, 0, p->stream>>>(p->u.p, Ni, Ne, c_i, phi_i, c_e, phi_e);
        KNP_CUDA(cudaGetLastError());
        KNP_CUDA(cudaStreamSynchronize(p->stream));
        return;
    }
    double* s = state_stage(p);
    double* seg[4] = {s, s + 3 * Ni, s + 4 * Ni, s + 4 * Ni + 3 * Ne};
    double* dst[4] = {c_i, phi_i, c_e, phi_e};
    const int64_t len[4] = {3 * Ni, Ni, 3 * Ne, Ne};
    count_launch();
    k_state_out<<<nblk(n), 256, 0, p->stream>>>(p->u.p, Ni, Ne, c_i ? seg[0] : nullptr, phi_i ? seg[1] : nullptr,
                                                c_e ? seg[2] : nullptr, phi_e ? seg[3] : nullptr);
    KNP_CUDA(cudaGetLastError());
    for (int a = 0; a < 4; ++a)
        if (dst[a] && len[a])
            KNP_CUDA(cudaMemcpyAsync(dst[a], seg[a], len[a] * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    KNP_CUDA(cudaStreamSynchronize(p->stream));
}

void state_copy_in(knp_problem* p, bool device, const double* c_i, const double* phi_i, const double* c_e,
                   const double* phi_e) {
    const int64_t Ni = p->N_i, Ne = p->N_e, n = Ni + Ne;
    if (device) {
        count_launch();
        k_state_in<<<nblk(n), 256, 0, p->stream>>>(p->u.p, Ni, Ne, c_i, phi_i, c_e, phi_e);
        KNP_CUDA(cudaGetLastError());
        return;
    }
    double* s = state_stage(p);
    double* seg[4] = {s, s + 3 * Ni, s + 4 * Ni, s + 4 * Ni + 3 * Ne};
    const double* src[4] = {c_i, phi_i, c_e, phi_e};
    const int64_t len[4] = {3 * Ni, Ni, 3 * Ne, Ne};
    for (int a = 0; a < 4; ++a)
        if (src[a] && len[a])
            KNP_CUDA(cudaMemcpyAsync(seg[a], src[a], len[a] * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    count_launch();
    k_state_in<<<nblk(n), 256, 0, p->stream>>>(p->u.p, Ni, Ne, c_i ? seg[0] : nullptr, phi_i ? seg[1] : nullptr,
                                               c_e ? seg[2] : nullptr, phi_e ? seg[3] : nullptr);
    KNP_CUDA(cudaGetLastError());
    // the caller's host buffers may be reused as soon as this returns
    KNP_CUDA(cudaStreamSynchronize(p->stream));
}

}  // namespace knp

extern "C" knp_status knp_mesh_p2_region_matrices(const knp_mesh* mesh, int32_t region, const double* c,
                                                  int64_t* count, int32_t* rows, int32_t* cols, double* M, double* A,
                                                  double* Ac) {
    return knp::guarded([&] {
        KNP_REQUIRE(mesh && count, KNP_ERR_INVALID_ARG, "NULL argument");
        KNP_REQUIRE(region == 0 || region == 1, KNP_ERR_INVALID_ARG, "region must be 0 or 1 (got %d)", region);
        KNP_REQUIRE(!Ac || c, KNP_ERR_INVALID_ARG, "the weighted stiffness needs the coefficient c");
        const int64_t npe = (int64_t)(mesh->dim + 1) * (mesh->dim + 2) / 2;
        const int64_t ne = (int64_t)(region == 0 ? mesh->elems_i.size() : mesh->elems_e.size());
        *count = ne * npe * npe;
        if (rows || cols || M || A || Ac) knp::p2_region_triplets(*mesh, region, c, rows, cols, M, A, Ac);
    });
}

