// Coarse correction of the potentials' near-null modes, wrapped around P_0^{-1} (Section 4.2).
//
// The potential blocks of P_0 are nearly singular: the intracellular potential of each cell is held
// only by the membrane capacitance (C_m/F M_Gamma, small against the stiffness of the cell's
// interior) and the extracellular potential only by the point pin of Remark 4.1. One V-cycle
// applies P_0^{-1} to these modes correctly, but a residual component along them is amplified by
// about 1/lambda_min. The paper's left-preconditioned GMRES minimises the preconditioned residual
// and so works on exactly that amplified quantity; the right-preconditioned FGMRES used here
// minimises the residual, which barely sees these modes, while its stopping test measures the
// preconditioned residual: without help the test stagnates far above its threshold (on the paper's
// 1 um Model A as well as at 100 um).
//
// The remedy is a two-level preconditioner with the coarse space Z = the per-cell constants of
// phi_i and the constant of phi_e (the pinned node left out), on the true operator:
//     E = Z^T A Z,   y = E^{-1} Z^T r,   M_D^{-1} r = P_0^{-1} (r - A Z y) + Z y.
// The V-cycle then sees a residual orthogonal to Z (nothing left to amplify) and Z y is the exact
// correction of those modes. FGMRES tolerates any preconditioner, so the iterate's accuracy is
// still set by the stopping test alone. The adjoint's A^T solve uses the same coarse space with
// Z^T A^T Z = E^T.
//
// Costs. A applied to a piecewise-constant potential is nonzero only through the membrane and
// pin terms: per row, the sum of its same-region e^k coefficients times the constant of its own
// region, plus its cross-region entries times the constants of their cells. Those row sums are
// formed once per step (RS, three values per node), E is an arrowhead matrix (cells couple only
// to the extracellular space) solved by its Schur complement on the device, and each application
// adds a gather and a small solve; the right-hand-side pass and the update run inside the
// V-cycle's first and last kernels (the transposed form and CG(P_0) keep them as separate passes,
// about 0.2 KB per node).
// Sums are taken in a fixed order (no atomics), so the result is reproducible bit for bit.
#include <algorithm>
#include <map>
#include <vector>

#include "deflate.h"
#include "problem.h"
#include "vcycle.h"

namespace knp {

namespace {

constexpr int DT = 256;          // threads of the deflation kernels
constexpr int EXT_BLOCKS = 304;  // partial-sum blocks over the extracellular nodes

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    return s;   // valid in thread 0
}

// RS[r][k] = sum of the same-region e^k values of row r over phi columns other than the pin;
// RSa[r] the same sum of the static stiffness a (for the transposed operator's concentration rows)
__global__ void k_defl_rowsums(int64_t n, int32_t pin, const int64_t* __restrict__ slice_ptr,
                               const int32_t* __restrict__ col, const double* __restrict__ e, int64_t ne,
                               const double* __restrict__ a, double* __restrict__ RS, double* __restrict__ RSa) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t s = r / SELL_C, base = slice_ptr[s] + r % SELL_C;
    const int64_t w = (slice_ptr[s + 1] - slice_ptr[s]) / SELL_C;
    double acc[KI] = {0, 0, 0}, sa = 0.0;
    for (int64_t k = 0; k < w; ++k) {
        const int64_t pos = base + k * SELL_C;
        if (col[pos] == pin) continue;
        for (int q = 0; q < KI; ++q) acc[q] += e[q * ne + pos];
        sa += a[pos];
    }
    for (int q = 0; q < KI; ++q) RS[3 * r + q] = acc[q];
    RSa[r] = sa;
}

// group of the source row of every transposed cross entry (-1: the pinned node)
__global__ void k_defl_xtg(int64_t nx, int64_t N_i, int32_t pin, const int32_t* __restrict__ xtrow,
                           const int32_t* __restrict__ rgrp, int32_t ext_group, int32_t* __restrict__ xtg) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nx) return;
    const int32_t j = xtrow[t];
    xtg[t] = j == pin ? -1 : (j < N_i ? rgrp[j] : ext_group);
}

// Per cell group j (one block): E_jj, E_je and E_ej of E = Z^T A Z. Potential-row coefficient of a
// stored entry: sum_k z_k e^k (same region) or sum_k z_k xe^k (cross region).
__global__ void __launch_bounds__(DT) k_defl_E_cells(const int64_t* __restrict__ cptr, const int32_t* __restrict__ cnodes,
                                                     const double* __restrict__ RS, const int32_t* __restrict__ xptr,
                                                     const int32_t* __restrict__ xg, const int32_t* __restrict__ xtptr,
                                                     const int32_t* __restrict__ xtrow, const int32_t* __restrict__ xtidx,
                                                     const double* __restrict__ xe, int64_t n_cross, int32_t pin,
                                                     double z0, double z1, double z2, int32_t ext_group,
                                                     double* __restrict__ Ejj, double* __restrict__ Eje,
                                                     double* __restrict__ Eej) {
    __shared__ double sh[DT / 32];
    const int j = blockIdx.x;
    double djj = 0.0, dje = 0.0, dej = 0.0;
    for (int64_t q = cptr[j] + threadIdx.x; q < cptr[j + 1]; q += blockDim.x) {
        const int64_t r = cnodes[q];
        djj += z0 * RS[3 * r] + z1 * RS[3 * r + 1] + z2 * RS[3 * r + 2];
        for (int t = xptr[r]; t < xptr[r + 1]; ++t)
            if (xg[t] == ext_group)
                dje += z0 * xe[t] + z1 * xe[n_cross + t] + z2 * xe[2 * n_cross + t];
        // column r of the cross part: rows of the extracellular space (the pinned one left out)
        for (int t = xtptr[r]; t < xtptr[r + 1]; ++t) {
            if (xtrow[t] == pin) continue;
            const int64_t idx = xtidx[t];
            dej += z0 * xe[idx] + z1 * xe[n_cross + idx] + z2 * xe[2 * n_cross + idx];
        }
    }
    double a = block_sum(djj, sh);
    if (threadIdx.x == 0) Ejj[j] = a;
    a = block_sum(dje, sh);
    if (threadIdx.x == 0) Eje[j] = a;
    a = block_sum(dej, sh);
    if (threadIdx.x == 0) Eej[j] = a;
}

// partial sums of E_ee over the extracellular rows (the pinned one left out)
__global__ void __launch_bounds__(DT) k_defl_E_ext(int64_t N_i, int64_t n, int32_t pin, const double* __restrict__ RS,
                                                   double z0, double z1, double z2, double* __restrict__ part) {
    __shared__ double sh[DT / 32];
    double acc = 0.0;
    for (int64_t r = N_i + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        if (r != pin) acc += z0 * RS[3 * r] + z1 * RS[3 * r + 1] + z2 * RS[3 * r + 2];
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// E_ee and the Schur complement S_e = E_ee - sum_j E_ej E_je / E_jj (one block)
__global__ void __launch_bounds__(DT) k_defl_schur(int nc, int nparts, const double* __restrict__ part,
                                                   const double* __restrict__ Ejj, const double* __restrict__ Eje,
                                                   const double* __restrict__ Eej, double* __restrict__ Ee) {
    __shared__ double sh[DT / 32];
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < nparts; q += blockDim.x) a += part[q];
    for (int j = threadIdx.x; j < nc; j += blockDim.x) b += Eej[j] * Eje[j] / Ejj[j];
    const double eee = block_sum(a, sh);
    const double red = block_sum(b, sh);
    if (threadIdx.x == 0) {
        Ee[0] = eee;
        Ee[1] = eee - red;
    }
}

// g = Z^T r with r = s .* v: blocks [0, nc) sum the potentials of one cell each, blocks
// [nc, nc + EXT_BLOCKS) partial sums over the extracellular potentials (pin left out)
__global__ void __launch_bounds__(DT) k_defl_gather(int nc, const int64_t* __restrict__ cptr,
                                                    const int32_t* __restrict__ cnodes, int64_t N_i, int64_t n,
                                                    int32_t pin, const double* __restrict__ v,
                                                    const double* __restrict__ s, double* __restrict__ g,
                                                    double* __restrict__ part) {
    __shared__ double sh[DT / 32];
    double acc = 0.0;
    if ((int)blockIdx.x < nc) {
        const int j = blockIdx.x;
        for (int64_t q = cptr[j] + threadIdx.x; q < cptr[j + 1]; q += blockDim.x) {
            const int64_t i = 4 * (int64_t)cnodes[q] + 3;
            acc += s[i] * v[i];
        }
        const double t = block_sum(acc, sh);
        if (threadIdx.x == 0) g[j] = t;
    } else {
        const int b = blockIdx.x - nc;
        for (int64_t r = N_i + b * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)EXT_BLOCKS * blockDim.x)
            if (r != pin) acc += s[4 * r + 3] * v[4 * r + 3];
        const double t = block_sum(acc, sh);
        if (threadIdx.x == 0) part[b] = t;
    }
}

// y = E^{-1} g for the arrowhead E (one block): y_e = (g_e - sum_j E_ej g_j / E_jj) / S_e,
// y_j = (g_j - E_je y_e) / E_jj; y[nc] = y_e
__global__ void __launch_bounds__(DT) k_defl_solve(int nc, const double* __restrict__ part, const double* __restrict__ g,
                                                   const double* __restrict__ Ejj, const double* __restrict__ Eje,
                                                   const double* __restrict__ Eej, const double* __restrict__ Ee,
                                                   double* __restrict__ y) {
    __shared__ double sh[DT / 32];
    __shared__ double ye_s;
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < EXT_BLOCKS; q += blockDim.x) a += part[q];
    for (int j = threadIdx.x; j < nc; j += blockDim.x) b += Eej[j] * g[j] / Ejj[j];
    const double ge = block_sum(a, sh);
    const double red = block_sum(b, sh);
    if (threadIdx.x == 0) {
        ye_s = (ge - red) / Ee[1];
        y[nc] = ye_s;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nc; j += blockDim.x) y[j] = (g[j] - Eje[j] * ye_s) / Ejj[j];
}

// t = s .* v - A Z y. Row r of A Z y: its same-region phi columns hold its own region's constant
// (RS), its cross-region entries their cells' constants; the potential row is sum_k z_k of the
// concentration rows' terms; the pinned potential row (the identity) gives 0.
__global__ void k_defl_rhs(int64_t n, int64_t N_i, int32_t pin, const int32_t* __restrict__ rgrp,
                           const double* __restrict__ RS, const int32_t* __restrict__ xptr,
                           const int32_t* __restrict__ xg, const double* __restrict__ xe, int64_t n_cross, double z0,
                           double z1, double z2, const double* __restrict__ y, int32_t ext_group,
                           const double* __restrict__ v, const double* __restrict__ s, double* __restrict__ t) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const double yr = y[r < N_i ? rgrp[r] : ext_group];
    double ae[KI];
    for (int q = 0; q < KI; ++q) ae[q] = RS[3 * r + q] * yr;
    for (int u = xptr[r]; u < xptr[r + 1]; ++u) {
        const int gq = xg[u];
        if (gq < 0) continue;
        const double yc = y[gq];
        for (int q = 0; q < KI; ++q) ae[q] += xe[q * n_cross + u] * yc;
    }
    double out3 = z0 * ae[0] + z1 * ae[1] + z2 * ae[2];
    if (r == pin) out3 = 0.0;
    const int64_t b = 4 * r;
    t[b] = s[b] * v[b] - ae[0];
    t[b + 1] = s[b + 1] * v[b + 1] - ae[1];
    t[b + 2] = s[b + 2] * v[b + 2] - ae[2];
    t[b + 3] = s[b + 3] * v[b + 3] - out3;
}

// t = s .* v - A^T Z y (the transposed operator's node block, cf. the transposed product): the
// concentration rows see tau_r^k z_k (sum of a over the row's phi columns) times the row's own
// constant; the potential row sum_k z_k e^k times it plus, through the transposed cross-region
// list, sum_k z_k xe^k times the source rows' constants; the pinned potential row gives 0.
__global__ void k_defl_rhs_t(int64_t n, int64_t N_i, int32_t pin, const int32_t* __restrict__ rgrp,
                             const double* __restrict__ RS, const double* __restrict__ RSa,
                             const int32_t* __restrict__ xtptr, const int32_t* __restrict__ xtidx,
                             const int32_t* __restrict__ xtg, const double* __restrict__ xe, int64_t n_cross,
                             double z0, double z1, double z2, RegionCoef ri, RegionCoef re,
                             const double* __restrict__ y, int32_t ext_group, const double* __restrict__ v,
                             const double* __restrict__ s, double* __restrict__ t) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const bool in = r < N_i;
    const RegionCoef& rc = in ? ri : re;
    const double yr = y[in ? rgrp[r] : ext_group];
    const double z[KI] = {z0, z1, z2};
    double out[4];
    for (int q = 0; q < KI; ++q) out[q] = rc.tau[q] * z[q] * RSa[r] * yr;
    double o3 = (z0 * RS[3 * r] + z1 * RS[3 * r + 1] + z2 * RS[3 * r + 2]) * yr;
    for (int u = xtptr[r]; u < xtptr[r + 1]; ++u) {
        const int gq = xtg[u];
        if (gq < 0) continue;
        const int64_t idx = xtidx[u];
        o3 += (z0 * xe[idx] + z1 * xe[n_cross + idx] + z2 * xe[2 * n_cross + idx]) * y[gq];
    }
    out[3] = r == pin ? 0.0 : o3;
    const int64_t b = 4 * r;
    for (int q = 0; q < 4; ++q) t[b + q] = s[b + q] * v[b + q] - out[q];
}

// z += Z y: the potential of every node of a group takes its group's constant
__global__ void k_defl_add(int64_t n, int64_t N_i, int32_t pin, const int32_t* __restrict__ rgrp,
                           const double* __restrict__ y, int32_t ext_group, double* __restrict__ z) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n || r == pin) return;
    z[4 * r + 3] += y[r < N_i ? rgrp[r] : ext_group];
}

__global__ void k_fill_ones(int64_t n, double* __restrict__ v) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) v[i] = 1.0;
}

inline unsigned nbk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

struct Deflation {
    int nc = 0;                       // cell groups (cells with at least one intracellular node)
    DArray<int64_t> cptr;             // group -> its intracellular nodes (increasing)
    DArray<int32_t> cnodes;
    DArray<int32_t> rgrp;             // intracellular node -> its group
    DArray<int32_t> xg;               // cross entry -> group of its column (-1: the pinned node)
    DArray<double> RS;                // [n][3] row sums of e^k over phi columns (per step)
    DArray<double> RSa;               // [n] row sums of a over phi columns (the transposed operator)
    DArray<int32_t> xtg;              // transposed cross entry -> group of its source row (-1: pin)
    DArray<double> Ejj, Eje, Eej, Ee; // the arrowhead E (per step); Ee = {E_ee, Schur complement}
    DArray<double> g, y, part, t, ones;
    int64_t built_for = -1;           // assembly whose operator E was formed from
};

void deflation_free(Deflation* d) { delete d; }

static Deflation& deflation_setup(knp_problem* p) {
    if (p->defl) return *p->defl;
    auto* d = new Deflation();
    p->defl = d;
    cudaStream_t st = p->stream;
    const knp_mesh& m = *p->mesh;
    const std::vector<int32_t>& cell = p->degree == 2 ? p2_nodes(m).node_cell_i : m.node_cell_i;
    KNP_REQUIRE((int64_t)cell.size() == p->N_i, KNP_ERR_STATE, "cell map does not match the intracellular nodes");
    std::map<int32_t, int> gid;
    for (int32_t c : cell) gid.emplace(c, 0);
    int k = 0;
    for (auto& kv : gid) kv.second = k++;
    d->nc = k;
    std::vector<int32_t> rg(std::max<int64_t>(p->N_i, 1), 0);
    std::vector<int64_t> cptr(d->nc + 1, 0);
    for (int64_t r = 0; r < p->N_i; ++r) {
        rg[r] = gid[cell[r]];
        cptr[rg[r] + 1]++;
    }
    for (int j = 0; j < d->nc; ++j) cptr[j + 1] += cptr[j];
    std::vector<int32_t> cn(std::max<int64_t>(p->N_i, 1));
    {
        std::vector<int64_t> fill(cptr.begin(), cptr.end() - 1);
        for (int64_t r = 0; r < p->N_i; ++r) cn[fill[rg[r]]++] = (int32_t)r;
    }
    const int32_t ext = d->nc;
    std::vector<int32_t> xg(std::max<size_t>(p->h_xcol.size(), 1), -1);
    for (size_t t = 0; t < p->h_xcol.size(); ++t) {
        const int32_t c = p->h_xcol[t];
        xg[t] = c == p->pin ? -1 : (c < p->N_i ? rg[c] : ext);
    }
    d->cptr.upload(cptr, st);
    d->cnodes.upload(cn, st);
    d->rgrp.upload(rg, st);
    d->xg.upload(xg, st);
    const int64_t n = p->n_nodes;
    d->RS.alloc(3 * n);
    d->RSa.alloc(n);
    const int64_t nx = (int64_t)p->h_xcol.size();
    d->xtg.alloc(std::max<int64_t>(nx, 1));
    if (nx) {
        k_defl_xtg<<<nbk(nx, 256), 256, 0, st>>>(nx, p->N_i, p->pin, p->xtrow.p, d->rgrp.p, ext, d->xtg.p);
        count_launch();
    }
    for (DArray<double>* a : {&d->Ejj, &d->Eje, &d->Eej}) a->alloc(std::max(d->nc, 1));
    d->Ee.alloc(2);
    d->g.alloc(std::max(d->nc, 1));
    d->y.alloc(d->nc + 1);
    d->part.alloc(EXT_BLOCKS);
    d->t.alloc(4 * n);
    d->ones.alloc(4 * n);
    k_fill_ones<<<nbk(4 * n, 256), 256, 0, st>>>(4 * n, d->ones.p);
    count_launch();
    KNP_CUDA(cudaGetLastError());
    return *d;
}

void deflation_prepare(knp_problem* p) {
    Deflation& d = deflation_setup(p);
    if (d.built_for == p->assembly_id) return;
    cudaStream_t st = p->stream;
    const int64_t n = p->n_nodes, nx = (int64_t)p->h_xcol.size();
    const double* z = p->sp.z;
    count_launch(4);
    k_defl_rowsums<<<nbk(n, 128), 128, 0, st>>>(n, p->pin, p->sell.slice_ptr.p, p->sell.col.p, p->sell_e.p,
                                                 p->sell.n_entries, p->sell_a.p, d.RS.p, d.RSa.p);
    if (d.nc)
        k_defl_E_cells<<<d.nc, DT, 0, st>>>(d.cptr.p, d.cnodes.p, d.RS.p, p->xptr.p, d.xg.p, p->xtptr.p, p->xtrow.p,
                                            p->xtidx.p, p->xe.p, nx, p->pin, z[0], z[1], z[2], d.nc, d.Ejj.p,
                                            d.Eje.p, d.Eej.p);
    k_defl_E_ext<<<EXT_BLOCKS, DT, 0, st>>>(p->N_i, n, p->pin, d.RS.p, z[0], z[1], z[2], d.part.p);
    k_defl_schur<<<1, DT, 0, st>>>(d.nc, EXT_BLOCKS, d.part.p, d.Ejj.p, d.Eje.p, d.Eej.p, d.Ee.p);
    KNP_CUDA(cudaGetLastError());
    d.built_for = p->assembly_id;
}

void deflated_precond_apply(knp_problem* p, const double* v, const double* s, double* z, bool transpose) {
    Deflation& d = *p->defl;
    cudaStream_t st = p->stream;
    const int64_t n = p->n_nodes, nx = (int64_t)p->h_xcol.size();
    const double* zc = p->sp.z;
    count_launch(2);
    k_defl_gather<<<d.nc + EXT_BLOCKS, DT, 0, st>>>(d.nc, d.cptr.p, d.cnodes.p, p->N_i, n, p->pin, v, s, d.g.p,
                                                    d.part.p);
    // Z^T A^T Z = E^T: the same Schur complement, E_je and E_ej exchanged
    k_defl_solve<<<1, DT, 0, st>>>(d.nc, d.part.p, d.g.p, d.Ejj.p, transpose ? d.Eej.p : d.Eje.p,
                                   transpose ? d.Eje.p : d.Eej.p, d.Ee.p, d.y.p);
    if (!transpose && p->amg->inner_cg_max_it == 0) {
        // one V-cycle: its first kernel forms s .* v - A Z y and its output kernel adds Z y
        DeflFuse df;
        df.rgrp = d.rgrp.p;
        df.RS = d.RS.p;
        df.xptr = p->xptr.p;
        df.xg = d.xg.p;
        df.xe = p->xe.p;
        df.y = d.y.p;
        df.n_cross = nx;
        df.N_i = p->N_i;
        df.pin = p->pin;
        df.ext_group = d.nc;
        for (int q = 0; q < 3; ++q) df.z[q] = zc[q];
        KNP_CUDA(cudaGetLastError());
        vcycle_apply(p, v, s, z, &df);
        return;
    }
    count_launch();
    if (transpose)
        k_defl_rhs_t<<<nbk(n, 128), 128, 0, st>>>(n, p->N_i, p->pin, d.rgrp.p, d.RS.p, d.RSa.p, p->xtptr.p,
                                                  p->xtidx.p, d.xtg.p, p->xe.p, nx, zc[0], zc[1], zc[2], p->sp.reg[0],
                                                  p->sp.reg[1], d.y.p, d.nc, v, s, d.t.p);
    else
        k_defl_rhs<<<nbk(n, 128), 128, 0, st>>>(n, p->N_i, p->pin, d.rgrp.p, d.RS.p, p->xptr.p, d.xg.p, p->xe.p, nx,
                                                zc[0], zc[1], zc[2], d.y.p, d.nc, v, s, d.t.p);
    precond_apply(p, d.t.p, d.ones.p, z);
    count_launch();
    k_defl_add<<<nbk(n, 256), 256, 0, st>>>(n, p->N_i, p->pin, d.rgrp.p, d.y.p, d.nc, z);
    KNP_CUDA(cudaGetLastError());
}

}  // namespace knp
