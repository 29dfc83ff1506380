// CG(P_0): P_0^{-1} applied by the conjugate gradient method, preconditioned by one V-cycle,
// field-split into the 2(|K|+1) = 8 independent blocks of P_0 (four fields in each of the two
// regions, Eq. 4.4). This is the block-wise CG(P_0) strategy of Section 6.3, an (almost) exact
// inverse of P_0, against which the single V-cycle of AMG(P_0) is compared: with it FGMRES sees
// P_0^{-1} itself, so its iteration counts are those of the preconditioner P_0, whatever the
// quality of the V-cycle.
//
// The eight CGs run in lockstep on the interleaved [node][4] vectors; each has its own step
// lengths and its own stopping test ||r_g|| <= rtol ||b_g||. A block that has converged keeps
// its iterate (step lengths 0). P_0 and the V-cycle are symmetric positive definite (for CG(P_0)
// knp_amg_setup gives the V-cycle the same Chebyshev steps before and after, and the coarsest
// level is solved exactly), as CG needs. The dot products come to the host once per inner
// iteration.
#include <cmath>
#include <vector>

#include "problem.h"
#include "vcycle.h"

namespace knp {

namespace {

constexpr int NG = 8;            // field blocks: 4 fields x 2 regions
constexpr int DOT_BLOCKS = 304;  // 2 x 152 SMs
constexpr int DOT_THREADS = 256;

__device__ __forceinline__ int group_of(int64_t node, int f, int64_t Ni) { return f + (node >= Ni ? 4 : 0); }

// partial[b][g] and partial[b][NG + g]: block b's share of <a, b>_g and <c, d>_g (c, d may be NULL)
__global__ void __launch_bounds__(DOT_THREADS) k_group_dots(int64_t n, int64_t Ni, const double* __restrict__ a,
                                                            const double* __restrict__ b,
                                                            const double* __restrict__ c,
                                                            const double* __restrict__ d,
                                                            double* __restrict__ partial) {
    double acc[2 * NG];
    for (int k = 0; k < 2 * NG; ++k) acc[k] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int o = i >= Ni ? 4 : 0;
        for (int f = 0; f < 4; ++f) {
            acc[o + f] += a[4 * i + f] * b[4 * i + f];
            if (c) acc[NG + o + f] += c[4 * i + f] * d[4 * i + f];
        }
    }
    __shared__ double sh[DOT_THREADS / 32][2 * NG];
    const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
    for (int k = 0; k < 2 * NG; ++k) {
        double v = acc[k];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) sh[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2 * NG) {
        double s = 0.0;
        for (int w = 0; w < DOT_THREADS / 32; ++w) s += sh[w][threadIdx.x];
        partial[(int64_t)blockIdx.x * 2 * NG + threadIdx.x] = s;
    }
}

// out[k] = sum_b partial[b][k], k < 2 NG (one block)
__global__ void k_group_reduce(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
    const int k = threadIdx.x;
    if (k >= 2 * NG) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partial[(int64_t)b * 2 * NG + k];
    out[k] = s;
}

struct Coefs {
    double v[NG];
};

// r = s .* v, z = 0
__global__ void k_pcg_init(int64_t n4, const double* __restrict__ v, const double* __restrict__ s,
                           double* __restrict__ r, double* __restrict__ z) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n4) return;
    r[i] = s[i] * v[i];
    z[i] = 0.0;
}

// z += alpha_g p, r -= alpha_g q
__global__ void k_pcg_step(int64_t n, int64_t Ni, Coefs alpha, const double* __restrict__ pv,
                           const double* __restrict__ q, double* __restrict__ z, double* __restrict__ r) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int f = 0; f < 4; ++f) {
        const double a = alpha.v[group_of(i, f, Ni)];
        z[4 * i + f] += a * pv[4 * i + f];
        r[4 * i + f] -= a * q[4 * i + f];
    }
}

// p = y + beta_g p
__global__ void k_pcg_dir(int64_t n, int64_t Ni, Coefs beta, const double* __restrict__ y, double* __restrict__ pv) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int f = 0; f < 4; ++f) pv[4 * i + f] = y[4 * i + f] + beta.v[group_of(i, f, Ni)] * pv[4 * i + f];
}

__global__ void k_fill_one(int64_t n4, double* __restrict__ o) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n4) o[i] = 1.0;
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

struct PcgWork {
    DArray<double> r, y, pv, q, ones, partial, dots;
    double* h_dots = nullptr;   // pinned, 2 NG
    ~PcgWork() {
        if (h_dots) cudaFreeHost(h_dots);
    }
};

void pcg_free(PcgWork* w) { delete w; }

namespace {

PcgWork& pcg_work(knp_problem* p) {
    if (!p->pcg) {
        auto* w = new PcgWork();
        p->pcg = w;
        const int64_t n4 = 4 * p->n_nodes;
        for (DArray<double>* v : {&w->r, &w->y, &w->pv, &w->q, &w->ones}) v->alloc(n4);
        w->partial.alloc(DOT_BLOCKS * 2 * NG);
        w->dots.alloc(2 * NG);
        KNP_CUDA(cudaMallocHost(&w->h_dots, 2 * NG * sizeof(double)));
        count_launch();
        k_fill_one<<<nblk(n4, 256), 256, 0, p->stream>>>(n4, w->ones.p);
    }
    return *p->pcg;
}

// the two per-group dot products <a, b>_g and <c, d>_g, on the host
void group_dots(knp_problem* p, PcgWork& w, const double* a, const double* b, const double* c, const double* d,
                double out[2 * NG]) {
    cudaStream_t st = p->stream;
    count_launch(2);
    k_group_dots<<<DOT_BLOCKS, DOT_THREADS, 0, st>>>(p->n_nodes, p->N_i, a, b, c, d, w.partial.p);
    k_group_reduce<<<1, 32, 0, st>>>(w.partial.p, DOT_BLOCKS, w.dots.p);
    KNP_CUDA(cudaMemcpyAsync(w.h_dots, w.dots.p, 2 * NG * sizeof(double), cudaMemcpyDeviceToHost, st));
    KNP_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < 2 * NG; ++k) {
        KNP_REQUIRE(std::isfinite(w.h_dots[k]), KNP_ERR_NUMERIC, "CG(P_0): dot product is not finite");
        out[k] = w.h_dots[k];
    }
}

void pcg_apply(knp_problem* p, const double* v, const double* s, double* z) {
    AmgHierarchy& H = *p->amg;
    PcgWork& w = pcg_work(p);
    cudaStream_t st = p->stream;
    const int64_t n = p->n_nodes, n4 = 4 * n, Ni = p->N_i;
    const double tol2 = H.inner_cg_rtol * H.inner_cg_rtol;
    count_launch();
    k_pcg_init<<<nblk(n4, 256), 256, 0, st>>>(n4, v, s, w.r.p, z);
    // y = M r (one V-cycle), p = y
    vcycle_apply(p, w.r.p, w.ones.p, w.y.p);
    KNP_CUDA(cudaMemcpyAsync(w.pv.p, w.y.p, n4 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    double d0[2 * NG];
    group_dots(p, w, w.r.p, w.y.p, w.r.p, w.r.p, d0);
    double rho[NG], bb[NG];
    bool done[NG];
    for (int g = 0; g < NG; ++g) {
        rho[g] = d0[g];
        bb[g] = d0[NG + g];
        done[g] = bb[g] == 0.0 || rho[g] <= 0.0;
    }
    for (int it = 0; it < H.inner_cg_max_it; ++it) {
        bool all = true;
        for (int g = 0; g < NG; ++g) all &= done[g];
        if (all) break;
        // q = P_0 p, alpha_g = rho_g / <p, q>_g
        p0_apply(p, w.pv.p, w.q.p);
        double pq[2 * NG];
        group_dots(p, w, w.pv.p, w.q.p, nullptr, nullptr, pq);
        Coefs alpha{};
        for (int g = 0; g < NG; ++g) alpha.v[g] = (done[g] || pq[g] <= 0.0) ? 0.0 : rho[g] / pq[g];
        count_launch();
        k_pcg_step<<<nblk(n, 256), 256, 0, st>>>(n, Ni, alpha, w.pv.p, w.q.p, z, w.r.p);
        H.inner_its++;
        // y = M r; rho'_g = <r, y>_g; ||r||_g
        vcycle_apply(p, w.r.p, w.ones.p, w.y.p);
        double ry[2 * NG];
        group_dots(p, w, w.r.p, w.y.p, w.r.p, w.r.p, ry);
        Coefs beta{};
        for (int g = 0; g < NG; ++g) {
            if (done[g]) continue;
            if (ry[NG + g] <= tol2 * bb[g] || ry[g] <= 0.0 || pq[g] <= 0.0) {
                done[g] = true;
                continue;
            }
            beta.v[g] = ry[g] / rho[g];
            rho[g] = ry[g];
        }
        count_launch();
        k_pcg_dir<<<nblk(n, 256), 256, 0, st>>>(n, Ni, beta, w.y.p, w.pv.p);
    }
    KNP_CUDA(cudaGetLastError());
}

}  // namespace

void precond_apply(knp_problem* p, const double* v, const double* s, double* z) {
    KNP_REQUIRE(p->amg, KNP_ERR_STATE, "knp_amg_setup has not been called");
    if (p->amg->inner_cg_max_it > 0)
        pcg_apply(p, v, s, z);
    else
        vcycle_apply(p, v, s, z);
}

}  // namespace knp
