// Flexible GMRES(m), FP64, right-preconditioned by one V-cycle on P_0 (Section 4.2,
// Section 6.2: restart 30, x_0 = u_{n-1}).
//
// The Krylov space is built for the symmetrically scaled system
// S^-1 A S^-1 (S x) = S^-1 f with S^2 = diag(P_0), which evens out the concentration and
// potential rows (their magnitudes differ by orders of magnitude); the scaling is applied
// on the fly (SpMV row scale, V-cycle input scale), so the preconditioned directions
// z_j live in the unscaled solution space and x = x_0 + Z y directly. Orthogonalisation
// is classical Gram-Schmidt with one reorthogonalisation (CGS2) in three fused passes; the
// second pass is made only when the first removed nearly all of the new vector (REORTH_KEEP).
//
// Stopping test: the preconditioned residual, as in Section 6.2, measured in the scaled
// norm and relative to the iterate x_c the current restart cycle began from (x_0 for the
// first cycle; or, if that is smaller, to the correction of the cycle, which covers a cold
// start), for the concentrations and the potentials apart:
// ||S M^-1 r_k||_g <= rtol max(||S x_c||_g, ||S (x_k - x_c)||_g) for g in {c, phi}. A residual norm
// alone is blind to the per-cell constant of phi_i (the intracellular potential block is
// singular up to the small membrane mass), while M^-1 r approximates the error. For the
// FGMRES iterate, M^-1 r_k = Z_{k+1} c with c = Q_k^T g_k e_{k+1} from the Givens rotations,
// so its group S-norms (and those of the correction Z y_k) take one pass over Z. That pass is
// made only when the test may pass: each evaluation records est_g / |g_k|, and the next is
// scheduled once that ratio times the current Givens residual |g_k| comes near the threshold.
// (Apart, because the scaled concentrations outweigh the scaled potentials by two orders.)
// The host sees one Hessenberg column per iteration.
#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <unordered_map>
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "deflate.h"
#include "gmres.h"
#include "problem.h"
#include "vcycle.h"

namespace knp {

namespace {

constexpr int RED_BLOCKS = 608;   // 4 x 152 SMs: the most blocks a reduction kernel launches
constexpr int RED_THREADS = 256;
constexpr int MAXV = 32;          // restart + 2
constexpr int MAXW = 3 * MAXV;    // partial-sum slots per block
// device scalars: [0, MAXV) first-pass dots, [MAXV, 2 MAXV) second-pass dots, [2 MAXV, 2 MAXV +
// MAXW) reference norms, 2 MAXV + MAXW the skip flag, then the six stopping-test norms
constexpr int CHK_OFF = 2 * MAXV + MAXW + 1;
constexpr int DOTS_LEN = CHK_OFF + 6;
constexpr int CHECK_EVERY = 8;         // steps between exact evaluations of the stopping test, at most
                                       // (8 against 4: 0.8-1.4% less time per step on the 3D and 2D
                                       // workloads, iteration counts equal or +2 in 290)
constexpr double CHECK_MARGIN = 10.0;  // evaluate once a prediction is within this factor of passing

// Every kernel below is instantiated for a compile-time vector count NV, so that the
// accumulators and basis values stay in registers (a runtime count put them on the stack).

// One halving step of a warp reduce-scatter of C values per lane (C even): lanes with bit O
// set keep the upper half and receive their partner's upper half, the others the lower half.
template <int C>
__device__ __forceinline__ void warp_halve(double* v, int lane, int O) {
    const bool hi = (lane & O) != 0;
#pragma unroll
    for (int k = 0; k < C / 2; ++k) {
        const double send = hi ? v[k] : v[k + C / 2];
        const double keep = hi ? v[k + C / 2] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, O);
    }
}

// Block sums of NT values per thread into partial[blockIdx.x][0..NT). Inside a warp the NT
// values (padded to C, a multiple of 32) are reduce-scattered in five halving steps, which
// leave lane L with the warp sums of values [L C/32, (L+1) C/32): about C shuffles and adds
// per lane instead of 5 NT for a butterfly per value (the adds are FP64, the scarce pipe).
template <int NT>
__device__ __forceinline__ void block_reduce_store(const double (&acc)[NT], double* __restrict__ partial) {
    constexpr int C = (NT + 31) / 32 * 32;
    constexpr int PER = C / 32;
    __shared__ double sh[RED_THREADS / 32][C];
    const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
    double v[C];
#pragma unroll
    for (int k = 0; k < C; ++k) v[k] = k < NT ? acc[k] : 0.0;
    warp_halve<C>(v, lane, 16);
    warp_halve<C / 2>(v, lane, 8);
    warp_halve<C / 4>(v, lane, 4);
    warp_halve<C / 8>(v, lane, 2);
    warp_halve<C / 16>(v, lane, 1);
#pragma unroll
    for (int m = 0; m < PER; ++m) sh[wid][lane * PER + m] = v[m];
    __syncthreads();
    if (threadIdx.x < NT) {
        double s = 0;
        for (int w = 0; w < RED_THREADS / 32; ++w) s += sh[w][threadIdx.x];
        partial[(int64_t)blockIdx.x * MAXW + threadIdx.x] = s;
    }
}

// partial[b][k] = block b's share of <V_k, w> for k < NV, and of <w, w> at k = NV
template <int NV>
__global__ void __launch_bounds__(RED_THREADS) k_mdot(int64_t n4, const double* __restrict__ V, int64_t ldv,
                                                      const double* __restrict__ w, double* __restrict__ partial) {
    double acc[NV + 1];
#pragma unroll
    for (int k = 0; k <= NV; ++k) acc[k] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        double wi = w[i];
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += V[k * ldv + i] * wi;
        acc[NV] += wi * wi;
    }
    block_reduce_store<NV + 1>(acc, partial);
}

// S^2-weighted dots split by group: slot NG*k + g holds group g's part of <V_k, w>_S and slots
// NG*NV + g hold <w, w>_S. Groups: 0 = concentrations (fields 0..2), 1 = potentials (field 3);
// with NG = 3, group 2 takes the extracellular potentials (elements at or past n4i).
template <int NV, int NG>
__global__ void __launch_bounds__(RED_THREADS) k_mdot_split(int64_t n4, const double* __restrict__ V, int64_t ldv,
                                                            const double* __restrict__ w, const double* __restrict__ s,
                                                            int64_t n4i, double* __restrict__ partial) {
    double acc[NV + 1];
    double out[NG * (NV + 1)];
#pragma unroll
    for (int k = 0; k <= NV; ++k) acc[k] = 0.0;
#pragma unroll
    for (int k = 0; k < NG * (NV + 1); ++k) out[k] = 0.0;
    // the grid stride is a multiple of 4, so every thread keeps the same field; a thread of the
    // potential field crosses the region boundary at most once, which flushes its sums
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool phi = (i0 & 3) == 3;
    int grp = phi ? ((NG == 3 && i0 >= n4i) ? 2 : 1) : 0;
    for (int64_t i = i0; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        if (NG == 3 && phi && grp == 1 && i >= n4i) {
#pragma unroll
            for (int k = 0; k <= NV; ++k) {
                out[NG * k + 1] += acc[k];
                acc[k] = 0.0;
            }
            grp = 2;
        }
        double wi = w[i] * s[i] * s[i];
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += V[k * ldv + i] * wi;
        acc[NV] += wi * w[i];
    }
#pragma unroll
    for (int k = 0; k <= NV; ++k) {
        if (grp == 0) out[NG * k] += acc[k];
        if (grp == 1) out[NG * k + 1] += acc[k];
        if (NG == 3 && grp == 2) out[NG * k + NG - 1] += acc[k];
    }
    block_reduce_store<NG * (NV + 1)>(out, partial);
}

// S^2-weighted squared norms, by group, of two combinations of the columns of Z:
// u = sum_k c[k] Z_k and v = sum_k y[k] Z_k (y[NV-1] is the newest column's, often 0).
// Slot g holds group g's part of ||u||_S^2 and slot NG + g that of ||v||_S^2 (groups as above).
// Without with_y only u is formed (v's slots stay zero): half the FP64 work.
template <int NV, int NG>
__global__ void __launch_bounds__(RED_THREADS) k_combo_norms(int64_t n4, const double* __restrict__ Z, int64_t ldz,
                                                             const double* __restrict__ cy, const double* __restrict__ s,
                                                             int64_t n4i, double* __restrict__ partial, int with_y) {
    double ck[NV > 0 ? NV : 1], yk[NV > 0 ? NV : 1];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        ck[k] = cy[k];
        yk[k] = cy[MAXV + k];
    }
    double out[2 * NG];
#pragma unroll
    for (int k = 0; k < 2 * NG; ++k) out[k] = 0.0;
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool phi = (i0 & 3) == 3;   // the grid stride is a multiple of 4
    for (int64_t i = i0; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        double u = 0.0, v = 0.0;
        if (with_y) {
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const double zk = Z[k * ldz + i];
                u += ck[k] * zk;
                v += yk[k] * zk;
            }
        } else {
#pragma unroll
            for (int k = 0; k < NV; ++k) u += ck[k] * Z[k * ldz + i];
        }
        const double w = s[i];
        u *= w;
        v *= w;
        const int grp = phi ? ((NG == 3 && i >= n4i) ? 2 : 1) : 0;
#pragma unroll
        for (int q = 0; q < NG; ++q) {
            if (grp == q) {
                out[q] += u * u;
                out[NG + q] += v * v;
            }
        }
    }
    block_reduce_store<2 * NG>(out, partial);
}

// w' = w - sum_k h[k] V_k (in place); partial sums of <V_k, w'> and <w', w'>. h holds the first
// pass's dots and, at h[NV], <w, w>. When the first pass kept at least REORTH_KEEP of w's squared
// norm (|w'|^2 = <w,w> - |h|^2 >= REORTH_KEEP <w,w>), w' is orthogonal to the basis to about
// eps / sqrt(REORTH_KEEP) and the second pass is skipped: only <w', w'> is formed, the dots stay
// zero, and k_orth_final then just normalises. This is the Daniel-Gragg-Kaufman-Stewart test with
// a looser threshold than its usual 1/2: on the FGMRES workloads here the first pass keeps
// 8-20% of |w|^2, the second pass found nothing to remove in 85-99% of the steps, and FP64 issue
// (not bandwidth) bounds these kernels on GB300.
constexpr double REORTH_KEEP = 1e-4;
template <int NV>
__global__ void __launch_bounds__(RED_THREADS) k_orth_update_dot(int64_t n4, const double* __restrict__ V, int64_t ldv,
                                                                 const double* __restrict__ h, double* __restrict__ w,
                                                                 double* __restrict__ partial) {
    double acc[NV + 1], hk[NV > 0 ? NV : 1];
    double hh = 0.0;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        hk[k] = h[k];
        hh += hk[k] * hk[k];
    }
    const double ww = h[NV];
    const bool second = ww - hh < REORTH_KEEP * ww;
#pragma unroll
    for (int k = 0; k <= NV; ++k) acc[k] = 0.0;
    if (second) {
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
            double vk[NV > 0 ? NV : 1];
            double wi = w[i];
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                vk[k] = V[k * ldv + i];
                wi -= hk[k] * vk[k];
            }
            w[i] = wi;
#pragma unroll
            for (int k = 0; k < NV; ++k) acc[k] += vk[k] * wi;
            acc[NV] += wi * wi;
        }
    } else {
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
            double wi = w[i];
#pragma unroll
            for (int k = 0; k < NV; ++k) wi -= hk[k] * V[k * ldv + i];
            w[i] = wi;
            acc[NV] += wi * wi;
        }
    }
    block_reduce_store<NV + 1>(acc, partial);
}

// v_{j+1} = (w' - sum_k h2[k] V_k) / eta with eta^2 = <w',w'> - |h2|^2 (in place). When the second
// Gram-Schmidt pass found nothing to remove (|h2| <= ORTH_SKIP * |w'|), the subtraction is skipped,
// V is not read, eta = |w'|, and flag[0] = 1 tells the host to keep h1 alone in the Hessenberg column.
constexpr double ORTH_SKIP = 1e-10;
template <int NV>
__global__ void __launch_bounds__(RED_THREADS) k_orth_final(int64_t n4, const double* __restrict__ V, int64_t ldv,
                                                            const double* __restrict__ h2, double* __restrict__ w,
                                                            double* __restrict__ flag) {
    double hk[NV > 0 ? NV : 1];
    double hh = 0.0;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        hk[k] = h2[k];
        hh += hk[k] * hk[k];
    }
    const double s2 = h2[NV];
    const bool skip = hh <= ORTH_SKIP * ORTH_SKIP * s2;
    const double e2 = skip ? s2 : s2 - hh;
    const double inv_eta = e2 > 0 ? 1.0 / sqrt(e2) : 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) flag[0] = skip ? 1.0 : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        double wi = w[i];
        if (!skip) {
#pragma unroll
            for (int k = 0; k < NV; ++k) wi -= hk[k] * V[k * ldv + i];
        }
        w[i] = wi * inv_eta;
    }
}

// out[k] = sum_b partial[b][k]
__global__ void k_reduce(const double* __restrict__ partial, int nblocks, int nv, double* __restrict__ out) {
    int k = blockIdx.x;
    if (k >= nv) return;
    double s = 0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(int64_t)b * MAXW + k];
    __shared__ double sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = sh[0];
}

// x += sum_k y[k] Z_k
template <int NZ>
__global__ void __launch_bounds__(RED_THREADS) k_update_x(int64_t n4, const double* __restrict__ Z, int64_t ldz,
                                                          const double* __restrict__ y, double* __restrict__ x) {
    double yk[NZ > 0 ? NZ : 1];
#pragma unroll
    for (int k = 0; k < NZ; ++k) yk[k] = y[k];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        double s = x[i];
#pragma unroll
        for (int k = 0; k < NZ; ++k) s += yk[k] * Z[k * ldz + i];
        x[i] = s;
    }
}

// Blocks of a grid-stride reduction kernel: one full wave, i.e. the blocks that are resident at
// once given this kernel's registers (from the occupancy calculator), at most RED_BLOCKS. A fixed
// grid that is not a multiple of the resident blocks leaves a partly filled last wave that costs
// as much as a full one (3 resident blocks per SM and 608 blocks ran these kernels 2x slower).
int red_grid(const void* fn) {
    static std::mutex mu;
    static std::unordered_map<const void*, int> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(fn);
    if (it != cache.end()) return it->second;
    int dev = 0, sms = 0, per_sm = 0;
    KNP_CUDA(cudaGetDevice(&dev));
    KNP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    KNP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, RED_THREADS, 0));
    const int g = std::max(1, std::min(RED_BLOCKS, per_sm * sms));
    cache.emplace(fn, g);
    return g;
}

#define KNP_NV_CASES(X) \
    X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(17) X(18) X(19) \
    X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30) X(31)

#define KNP_NV_CASE_k_mdot(N) \
    case N: nb_red = red_grid((const void*)&k_mdot<N>); k_mdot<N><<<nb_red, RED_THREADS, 0, st>>>(KNP_ARGS); break;
#define KNP_NV_CASE_k_mdot_split2(N) \
    case N: nb_red = red_grid((const void*)&k_mdot_split<N, 2>); k_mdot_split<N, 2><<<nb_red, RED_THREADS, 0, st>>>(KNP_ARGS); break;
#define KNP_NV_CASE_k_mdot_split3(N) \
    case N: nb_red = red_grid((const void*)&k_mdot_split<N, 3>); k_mdot_split<N, 3><<<nb_red, RED_THREADS, 0, st>>>(KNP_ARGS); break;
#define KNP_NV_CASE_k_combo_norms2(N) \
    case N: nb_red = red_grid((const void*)&k_combo_norms<N, 2>); k_combo_norms<N, 2><<<nb_red, RED_THREADS, 0, st>>>(KNP_ARGS); break;
#define KNP_NV_CASE_k_combo_norms3(N) \
    case N: nb_red = red_grid((const void*)&k_combo_norms<N, 3>); k_combo_norms<N, 3><<<nb_red, RED_THREADS, 0, st>>>(KNP_ARGS); break;
#define KNP_NV_CASE_k_orth_update_dot(N)                                                        \
    case N:                                                                                     \
        nb_red = red_grid((const void*)&k_orth_update_dot<N>);                                  \
        k_orth_update_dot<N><<<nb_red, RED_THREADS, 0, st>>>(KNP_ARGS);                         \
        break;
#define KNP_NV_CASE_k_orth_final(N) \
    case N: nb_red = red_grid((const void*)&k_orth_final<N>); k_orth_final<N><<<nb_red, RED_THREADS, 0, st>>>(KNP_ARGS); break;
#define KNP_NV_CASE_k_update_x(N) \
    case N: nb_red = red_grid((const void*)&k_update_x<N>); k_update_x<N><<<nb_red, RED_THREADS, 0, st>>>(KNP_ARGS); break;
// Launch KERNEL<nv><<<nb_red, RED_THREADS, 0, st>>>(args) for a runtime nv in [0, 31]; nb_red
// (a variable of the caller) receives the grid, which the following k_reduce sums over
#define KNP_LAUNCH_NV(nv, KERNEL)                                                                    \
    do {                                                                                             \
        switch (nv) {                                                                                \
            KNP_NV_CASES(KNP_NV_CASE_##KERNEL)                                                       \
            default: KNP_FAIL(KNP_ERR_INVALID_ARG, "vector count %d out of range", (int)(nv));        \
        }                                                                                            \
    } while (0)

__global__ void k_scale_copy(int64_t n4, const double* __restrict__ a, const double* __restrict__ s,
                             double* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n4) out[i] = a[i] * s[i];
}

__global__ void k_scale_inplace(int64_t n4, double* __restrict__ v, double s) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n4) v[i] *= s;
}

}  // namespace

struct GmresWork {
    int restart = 0;
    int64_t n4 = 0;
    DArray<double> V, Z, partial, dots, y, cy, tmp;
    DArray<double> ones;            // unit weights (the paper's unscaled stopping test), on first use
    double* hh = nullptr;           // pinned copy of dots, DOTS_LEN
    cudaEvent_t ev_dots = nullptr;  // recorded after the copy of dots to hh
    // the Arnoldi step of basis index j (SpMV, the three orthogonalisation passes with their
    // reductions, the copy of the dots to hh) as a CUDA graph per (j, transposed)
    std::map<std::pair<int, bool>, cudaGraphExec_t> arnoldi;
    cudaStream_t cap = nullptr;     // capture stream (the problem's stream may be the legacy one)
    ~GmresWork() {
        for (auto& kv : arnoldi) cudaGraphExecDestroy(kv.second);
        if (cap) cudaStreamDestroy(cap);
        if (hh) cudaFreeHost(hh);
        if (ev_dots) cudaEventDestroy(ev_dots);
    }
};

GmresWork* gmres_work(knp_problem* p, int restart) {
    if (p->gw && p->gw->restart == restart) return p->gw;
    delete p->gw;
    p->gw = nullptr;
    auto* g = new GmresWork();
    g->restart = restart;
    g->n4 = 4 * p->n_nodes;
    g->V.alloc((restart + 1) * g->n4);
    g->Z.alloc((restart + 1) * g->n4);
    g->partial.alloc(RED_BLOCKS * MAXW);
    g->dots.alloc(DOTS_LEN);
    g->y.alloc(MAXV);
    g->cy.alloc(2 * MAXV);
    g->tmp.alloc(g->n4);
    KNP_CUDA(cudaMallocHost(&g->hh, DOTS_LEN * sizeof(double)));
    KNP_CUDA(cudaEventCreateWithFlags(&g->ev_dots, cudaEventDisableTiming));
    p->gw = g;
    return g;
}

void gmres_free(GmresWork* g) { delete g; }

// squared norm of a device vector (through the multi-dot kernels)
static double norm2_dev(GmresWork& g, const double* v, cudaStream_t st) {
    count_launch(2);
    const int nb = red_grid((const void*)&k_mdot<0>);
    k_mdot<0><<<nb, RED_THREADS, 0, st>>>(g.n4, nullptr, 0, v, g.partial.p);
    k_reduce<<<1, 256, 0, st>>>(g.partial.p, nb, 1, g.dots.p);
    double s;
    KNP_CUDA(cudaMemcpyAsync(&s, g.dots.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    KNP_CUDA(cudaStreamSynchronize(st));
    return s;
}

// w = S^-1 A z_j into V_{j+1}, orthogonalised against V_0..V_j (CGS2, second pass skipped on the
// device when it has nothing to remove) and normalised; the dots of both passes land in g.dots
static void arnoldi_kernels(knp_problem* p, GmresWork& g, int j, bool transpose, cudaStream_t st) {
    const int64_t n4 = g.n4;
    const int nv = j + 1;
    int nb_red = RED_BLOCKS;
    double* zj = g.Z.p + (int64_t)j * n4;
    double* w = g.V.p + (int64_t)(j + 1) * n4;
    op_apply(p, zj, w, p->sinv.p, nullptr, transpose, st);
    ProfScope ps(&p->prof, KC_ORTHO, st);
    count_launch(5);
#define KNP_ARGS n4, g.V.p, n4, w, g.partial.p
    KNP_LAUNCH_NV(nv, k_mdot);
#undef KNP_ARGS
    k_reduce<<<nv + 1, 256, 0, st>>>(g.partial.p, nb_red, nv + 1, g.dots.p);
#define KNP_ARGS n4, g.V.p, n4, g.dots.p, w, g.partial.p
    KNP_LAUNCH_NV(nv, k_orth_update_dot);
#undef KNP_ARGS
    k_reduce<<<nv + 1, 256, 0, st>>>(g.partial.p, nb_red, nv + 1, g.dots.p + MAXV);
#define KNP_ARGS n4, g.V.p, n4, g.dots.p + MAXV, w, g.dots.p + 2 * MAXV + MAXW
    KNP_LAUNCH_NV(nv, k_orth_final);
#undef KNP_ARGS
    KNP_CUDA(cudaGetLastError());
}

// The Arnoldi step j followed by the copy of the dots to the pinned g.hh, replayed from a CUDA
// graph captured at first use (about ten launches become one).
static void arnoldi_graph_launch(knp_problem* p, GmresWork& g, int j, bool transpose) {
    auto key = std::make_pair(j, transpose);
    auto it = g.arnoldi.find(key);
    if (it == g.arnoldi.end()) {
        if (!g.cap) KNP_CUDA(cudaStreamCreateWithFlags(&g.cap, cudaStreamNonBlocking));
        const int64_t before = g_launches.load();
        KNP_CUDA(cudaStreamBeginCapture(g.cap, cudaStreamCaptureModeThreadLocal));
        try {
            arnoldi_kernels(p, g, j, transpose, g.cap);
            KNP_CUDA(cudaMemcpyAsync(g.hh, g.dots.p, DOTS_LEN * sizeof(double), cudaMemcpyDeviceToHost, g.cap));
        } catch (...) {
            cudaGraph_t tmp = nullptr;
            cudaStreamEndCapture(g.cap, &tmp);
            if (tmp) cudaGraphDestroy(tmp);
            throw;
        }
        cudaGraph_t graph = nullptr;
        KNP_CUDA(cudaStreamEndCapture(g.cap, &graph));
        g_launches.fetch_sub(g_launches.load() - before);
        cudaGraphExec_t ex = nullptr;
        cudaError_t e = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        KNP_CUDA(e);
        it = g.arnoldi.emplace(key, ex).first;
    }
    KNP_CUDA(cudaGraphLaunch(it->second, p->stream));
    count_launch(6);
}

knp_status_detail fgmres(knp_problem* p, const knp_solve_opts& o, knp_solve_stats& stats, double* x,
                         const double* fvec, bool transpose) {
    auto t0 = std::chrono::steady_clock::now();
    const int m = o.restart;
    KNP_REQUIRE(m >= 1 && m + 2 <= MAXV, KNP_ERR_INVALID_ARG, "restart must be in [1, %d]", MAXV - 2);
    GmresWork& g = *gmres_work(p, m);
    KNP_REQUIRE(p->amg, KNP_ERR_STATE, "knp_amg_setup has not been called");
    const int64_t inner0 = p->amg->inner_its;
    cudaStream_t st = p->stream;
    const int64_t n4 = g.n4;
    const unsigned nb = (unsigned)((n4 + 255) / 256);
    const bool paper_test = o.stop_test == KNP_TEST_PAPER;
    KNP_REQUIRE(o.stop_test == KNP_TEST_SCALED || paper_test, KNP_ERR_INVALID_ARG, "unknown stopping test %d",
                (int)o.stop_test);
    // the paper's test is one group over the whole vector: unit weights, no phi_e group
    const int NG = (o.phi_e_group && !paper_test) ? 3 : 2;
    const int64_t n4i = 4 * p->N_i;
    const bool defl = o.deflate != 0;
    if (defl) deflation_prepare(p);
    auto precond = [&](const double* v, const double* s, double* z) {
        if (defl)
            deflated_precond_apply(p, v, s, z, transpose);
        else
            precond_apply(p, v, s, z);
    };
    if (paper_test && !g.ones.p) {
        g.ones.alloc(n4);
        std::vector<double> h(n4, 1.0);
        KNP_CUDA(cudaMemcpyAsync(g.ones.p, h.data(), n4 * sizeof(double), cudaMemcpyHostToDevice, st));
        KNP_CUDA(cudaStreamSynchronize(st));
    }
    const double* wts = paper_test ? g.ones.p : p->swt.p;
    int nb_red = RED_BLOCKS;   // grid of the last reduction kernel (KNP_LAUNCH_NV sets it)
    // Arnoldi steps from CUDA graphs, unless a kernel class is being profiled (event pairs go
    // around single launches) or graphs are switched off for the V-cycle as well
    const bool use_graphs = p->amg->use_graphs && p->prof.active < 0;
    // reference norms of the stopping test, per group: ||S x|| of the iterate a cycle starts from
    // (the initial guess, then each restart's), taken together with the cycle's correction
    double tol[3] = {0, 0, 0};
    double paper_tol = 0.0;   // rtol ||M^-1 f||_2 (the paper's test)
    auto reference_norms = [&]() {
        if (paper_test) {
            tol[0] = tol[1] = paper_tol;
            return;
        }
        count_launch(2);
        int nb = 0;
        if (NG == 3) {
            nb = red_grid((const void*)&k_mdot_split<0, 3>);
            k_mdot_split<0, 3><<<nb, RED_THREADS, 0, st>>>(n4, nullptr, 0, x, p->swt.p, n4i, g.partial.p);
        } else {
            nb = red_grid((const void*)&k_mdot_split<0, 2>);
            k_mdot_split<0, 2><<<nb, RED_THREADS, 0, st>>>(n4, nullptr, 0, x, p->swt.p, n4i, g.partial.p);
        }
        k_reduce<<<NG, 256, 0, st>>>(g.partial.p, nb, NG, g.dots.p + 2 * MAXV);
        double xn2[3] = {0, 0, 0};
        KNP_CUDA(cudaMemcpyAsync(xn2, g.dots.p + 2 * MAXV, NG * sizeof(double), cudaMemcpyDeviceToHost, st));
        KNP_CUDA(cudaStreamSynchronize(st));
        KNP_REQUIRE(std::isfinite(xn2[0]) && std::isfinite(xn2[1]) && std::isfinite(xn2[2]), KNP_ERR_NUMERIC,
                    "iterate is not finite");
        for (int q = 0; q < NG; ++q) tol[q] = o.rtol * std::sqrt(std::max(xn2[q], 0.0));
        if (NG == 3) {
            // phi_e is some 1e-8 of phi_i: below ~1e-14 of the whole potential the rounding of the
            // coupled equations sets the floor, and a tighter request would stagnate
            const double floor_rel = o.phi_e_floor > 0 ? o.phi_e_floor : 1e-14;
            tol[2] = std::max(tol[2], floor_rel * std::sqrt(std::max(xn2[1] + xn2[2], 0.0)));
        }
    };
    if (paper_test) {
        precond(fvec, g.ones.p, g.tmp.p);
        paper_tol = o.rtol * std::sqrt(norm2_dev(g, g.tmp.p, st));
        KNP_REQUIRE(std::isfinite(paper_tol), KNP_ERR_NUMERIC, "preconditioned right-hand side is not finite");
    }
    k_scale_copy<<<nb, 256, 0, st>>>(n4, fvec, p->sinv.p, g.tmp.p);
    count_launch();
    const double bnorm = std::sqrt(norm2_dev(g, g.tmp.p, st));
    KNP_REQUIRE(std::isfinite(bnorm), KNP_ERR_NUMERIC, "right-hand side is not finite");
    knp_status_detail res{KNP_OK, 0, 0, 0.0};
    // KNP_GMRES_MONITOR set: every iteration prints the stopping test's terms to stderr
    static const bool monitor = std::getenv("KNP_GMRES_MONITOR") != nullptr;
    std::vector<double> H((m + 1) * m), cs(m), sn(m), gv(m + 1), cyh(2 * MAXV);
    int its = 0, restarts = 0;
    bool converged = false;
    double beta = 0;
    while (!converged) {
        // V_0 = S^-1 (f - A x)
        op_apply(p, x, g.V.p, p->sinv.p, fvec, transpose);
        beta = std::sqrt(norm2_dev(g, g.V.p, st));
        KNP_REQUIRE(std::isfinite(beta), KNP_ERR_NUMERIC, "residual is not finite");
        if (beta == 0.0) {
            converged = true;
            break;
        }
        if (its >= o.max_it) break;
        if (its > 0) restarts++;
        reference_norms();
        count_launch();
        k_scale_inplace<<<nb, 256, 0, st>>>(n4, g.V.p, 1.0 / beta);
        std::fill(gv.begin(), gv.end(), 0.0);
        gv[0] = beta;
        int k_done = 0;   // Arnoldi steps whose Hessenberg columns are kept
        // The stopping test is evaluated exactly (one pass over Z) at the first step of a cycle,
        // at its last, at least every CHECK_EVERY steps, and whenever the group norms predicted
        // from the last evaluation (est_g scaled by the Givens residual |g_j|) come within
        // CHECK_MARGIN of their thresholds; convergence is only ever declared from an evaluation.
        double ratio[3] = {0, 0, 0}, corr_last[3] = {0, 0, 0};
        int last_check = -1;
        bool vc_queued = false;
        for (int j = 0; j <= m; ++j) {
            double* vj = g.V.p + (int64_t)j * n4;
            double* zj = g.Z.p + (int64_t)j * n4;
            // z_j = P_0^{-1} (S v_j) (one V-cycle, or CG(P_0)), unless the previous step queued it
            if (!vc_queued) precond(vj, p->svec.p, zj);
            vc_queued = false;
            const bool arnoldi = (j < m) && (its < o.max_it);
            bool check = last_check < 0 || !arnoldi || j - last_check >= CHECK_EVERY;
            if (!check) {
                check = true;
                for (int q = 0; q < NG; ++q) {
                    const double ref = std::max(tol[q], o.rtol * corr_last[q]);
                    if (ratio[q] * std::fabs(gv[j]) > CHECK_MARGIN * ref) check = false;
                }
            }
            if (check) {
                // preconditioned residual of the iterate after j steps: M^-1 r = Z c with
                // c = Q^T (0, .., 0, g_j); the correction of this cycle, x_j - x_c = Z y_j
                const int k = j;
                std::fill(cyh.begin(), cyh.end(), 0.0);
                double* c = cyh.data();
                double* yk = cyh.data() + MAXV;
                c[k] = gv[k];
                for (int i = k - 1; i >= 0; --i) {
                    double a = c[i], b = c[i + 1];
                    c[i] = cs[i] * a - sn[i] * b;
                    c[i + 1] = sn[i] * a + cs[i] * b;
                }
                for (int i = k - 1; i >= 0; --i) {
                    double sacc = gv[i];
                    for (int q2 = i + 1; q2 < k; ++q2) sacc -= H[i * m + q2] * yk[q2];
                    yk[i] = sacc / H[i * m + i];
                }
                KNP_CUDA(cudaMemcpyAsync(g.cy.p, cyh.data(), 2 * MAXV * sizeof(double), cudaMemcpyHostToDevice,
                                         st));
                count_launch(2);
                // the correction's norm enters the reference only where a group's ||S x_c|| is zero
                // (a cold start); otherwise max(||S x_c||, ||S (x - x_c)||) is the state's norm
                // for every realistic step, so Z y is formed only in the first case
                bool with_y = false;
                for (int q = 0; q < NG; ++q) with_y |= tol[q] == 0.0;
#define KNP_ARGS n4, g.Z.p, n4, g.cy.p, wts, n4i, g.partial.p, (int)with_y
                if (NG == 3)
                    KNP_LAUNCH_NV(j + 1, k_combo_norms3);
                else
                    KNP_LAUNCH_NV(j + 1, k_combo_norms2);
#undef KNP_ARGS
                k_reduce<<<2 * NG, 256, 0, st>>>(g.partial.p, nb_red, 2 * NG, g.dots.p + CHK_OFF);
            }
            const int nv = j + 1;
            if (arnoldi && use_graphs) {
                arnoldi_graph_launch(p, g, j, transpose);   // includes the copy of the dots
            } else {
                if (arnoldi) arnoldi_kernels(p, g, j, transpose, st);
                KNP_CUDA(cudaMemcpyAsync(g.hh, g.dots.p, DOTS_LEN * sizeof(double), cudaMemcpyDeviceToHost, st));
            }
            KNP_CUDA(cudaEventRecord(g.ev_dots, st));
            if (arnoldi) {
                // v_{j+1} is already normalised on the device: queue its V-cycle before the host
                // waits for this step's dots, so the GPU works while the host does the Givens step
                precond(g.V.p + (int64_t)(j + 1) * n4, p->svec.p, g.Z.p + (int64_t)(j + 1) * n4);
                vc_queued = true;
            }
            KNP_CUDA(cudaEventSynchronize(g.ev_dots));
            KNP_CUDA(cudaGetLastError());
            if (check) {
                bool ok = true;
                if (monitor) std::fprintf(stderr, "fgmres%s it %d |g| %.3e", transpose ? "^T" : "", its, std::fabs(gv[j]));
                if (paper_test) {
                    // one group: ||M^-1 r||_2 over the whole vector against rtol ||M^-1 f||_2; the
                    // ratio predicts it from the Givens residual as for the scaled test
                    const double e0 = g.hh[CHK_OFF], e1 = g.hh[CHK_OFF + 1];
                    KNP_REQUIRE(std::isfinite(e0) && std::isfinite(e1), KNP_ERR_NUMERIC,
                                "preconditioned residual is not finite");
                    const double est = std::sqrt(std::max(e0 + e1, 0.0));
                    ok = est <= paper_tol;
                    ratio[0] = ratio[1] = gv[j] != 0.0 ? est / std::fabs(gv[j]) : 0.0;
                    corr_last[0] = corr_last[1] = 0.0;
                    if (monitor) std::fprintf(stderr, "  est %.3e tol %.3e", est, paper_tol);
                } else {
                    for (int q = 0; q < NG; ++q) {
                        const double est2 = g.hh[CHK_OFF + q], corr2 = g.hh[CHK_OFF + NG + q];
                        KNP_REQUIRE(std::isfinite(est2) && std::isfinite(corr2), KNP_ERR_NUMERIC,
                                    "preconditioned residual is not finite");
                        const double est = std::sqrt(std::max(est2, 0.0)), corr = std::sqrt(std::max(corr2, 0.0));
                        const double ref = std::max(tol[q], o.rtol * corr);
                        ok &= est <= ref;
                        ratio[q] = gv[j] != 0.0 ? est / std::fabs(gv[j]) : 0.0;
                        corr_last[q] = corr;
                        if (monitor) std::fprintf(stderr, "  [%d] est %.3e tol %.3e corr %.3e", q, est, tol[q], corr);
                    }
                }
                if (monitor) std::fprintf(stderr, "\n");
                last_check = j;
                if (ok) {
                    converged = true;
                    k_done = j;
                    break;
                }
            }
            if (!arnoldi) {
                k_done = j;
                break;
            }
            // second pass skipped on the device (flag): the column is h1 and eta = |w'|
            const bool skipped = g.hh[2 * MAXV + MAXW] != 0.0;
            if (monitor) {
                // first Gram-Schmidt pass: |w'|^2 / |w|^2 = 1 - sum h1^2 / |w|^2
                double h1 = 0.0;
                for (int k = 0; k < nv; ++k) h1 += g.hh[k] * g.hh[k];
                std::fprintf(stderr, "arnoldi j %d pass1 ratio %.3e second-pass skipped %d\n", j,
                             g.hh[nv] > 0 ? 1.0 - h1 / g.hh[nv] : 0.0, (int)skipped);
            }
            double s2 = g.hh[MAXV + nv];
            double eta2 = s2;
            for (int k = 0; k < nv; ++k) {
                H[k * m + j] = g.hh[k] + (skipped ? 0.0 : g.hh[MAXV + k]);
                if (!skipped) eta2 -= g.hh[MAXV + k] * g.hh[MAXV + k];
            }
            KNP_REQUIRE(std::isfinite(eta2), KNP_ERR_NUMERIC, "Arnoldi vector is not finite");
            double eta = eta2 > 0 ? std::sqrt(eta2) : 0.0;
            H[(j + 1) * m + j] = eta;
            for (int k = 0; k < j; ++k) {
                double a = H[k * m + j], b = H[(k + 1) * m + j];
                H[k * m + j] = cs[k] * a + sn[k] * b;
                H[(k + 1) * m + j] = -sn[k] * a + cs[k] * b;
            }
            double den = std::hypot(H[j * m + j], H[(j + 1) * m + j]);
            cs[j] = H[j * m + j] / den;
            sn[j] = H[(j + 1) * m + j] / den;
            H[j * m + j] = den;
            H[(j + 1) * m + j] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            its++;
            k_done = j + 1;
            if (eta == 0.0) {
                converged = true;   // happy breakdown: the Krylov space holds the solution
                break;
            }
        }
        if (k_done > 0) {
            // y = R^-1 g (upper triangular), x += Z y
            std::vector<double> y(k_done);
            for (int k = k_done - 1; k >= 0; --k) {
                double s = gv[k];
                for (int q = k + 1; q < k_done; ++q) s -= H[k * m + q] * y[q];
                y[k] = s / H[k * m + k];
            }
            KNP_CUDA(cudaMemcpyAsync(g.y.p, y.data(), k_done * sizeof(double), cudaMemcpyHostToDevice, st));
            count_launch();
#define KNP_ARGS n4, g.Z.p, n4, g.y.p, x
            KNP_LAUNCH_NV(k_done, k_update_x);
#undef KNP_ARGS
            KNP_CUDA(cudaGetLastError());
        }
        if (!converged && its >= o.max_it) {
            res.code = KNP_ERR_NOT_CONVERGED;
            break;
        }
    }
    // report the scaled true residual of the final iterate
    op_apply(p, x, g.tmp.p, p->sinv.p, fvec, transpose);
    double rn = std::sqrt(norm2_dev(g, g.tmp.p, st));
    double relres = bnorm > 0 ? rn / bnorm : 0.0;
    if (!converged) res.code = KNP_ERR_NOT_CONVERGED;
    res.iterations = its;
    res.restarts = restarts;
    res.relres = relres;
    stats.iterations = its;
    stats.restarts = restarts;
    stats.inner_iterations = p->amg->inner_its - inner0;
    stats.true_relres = relres;
    stats.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return res;
}

}  // namespace knp
