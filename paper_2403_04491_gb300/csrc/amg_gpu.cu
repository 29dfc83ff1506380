// GPU construction of the smoothed-aggregation hierarchy on P_0 (Section 4.2: one AMG V-cycle
// on P_0, set up once). The same algorithm as the host version in amg_setup.cpp, step for
// step, so that both give the same aggregates and operators:
//   strength graph  |s_ij| >= theta sqrt(|s_ii s_jj|)                  k_strength_count/fill
//   MIS-2           Luby-style rounds with hashed priorities: a node is a root when it holds
//                   the largest priority among undecided nodes within distance 2, and is
//                   excluded when a root lies within distance 2             k_mis2_*
//   aggregates      roots + their strong neighbours; leftovers join the first aggregated strong
//                   neighbour; what remains becomes singletons               k_agg_*
//   prolongator     P_f = (I - omega_f D_f^-1 A_f) P_tent,f, four fields on one pattern
//   Galerkin        R = P^T, A_c = R (A P) per field by a row-per-warp SpGEMM: keys through a
//                   shared-memory hash, values accumulated in the host's (Gustavson) order, so
//                   the result does not depend on thread timing               k_spgemm_*
//   Chebyshev bounds power iteration on D^-1 A per field, 20 steps             k_power_*
// The coarsest level's dense inverse is formed on the host (a few hundred unknowns).
#include <algorithm>
#include <cmath>

#include "amg_gpu.h"

namespace knp {

namespace {

inline unsigned nb(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

__host__ __device__ __forceinline__ uint32_t hash32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// ------------------------------------------------------------------ exclusive scan (int64)
__global__ void k_scan_block(int64_t n, const int64_t* __restrict__ in, int64_t* __restrict__ out,
                             int64_t* __restrict__ sums) {
    __shared__ int64_t sh[1024];
    int64_t i = blockIdx.x * 1024LL + threadIdx.x;
    int64_t v = i < n ? in[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int64_t t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = sh[threadIdx.x] - v;   // exclusive
    if (threadIdx.x == 1023) sums[blockIdx.x] = sh[1023];
}

__global__ void k_scan_add(int64_t n, int64_t* __restrict__ out, const int64_t* __restrict__ offs) {
    int64_t i = blockIdx.x * 1024LL + threadIdx.x;
    if (i < n) out[i] += offs[blockIdx.x];
}

// out[0..n] = exclusive scan of in[0..n-1] with out[n] = total; returns the total
int64_t exclusive_scan(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st) {
    if (n == 0) {
        int64_t z = 0;
        KNP_CUDA(cudaMemcpyAsync(out, &z, sizeof(int64_t), cudaMemcpyHostToDevice, st));
        KNP_CUDA(cudaStreamSynchronize(st));
        return 0;
    }
    int64_t blocks = (n + 1023) / 1024;
    DArray<int64_t> sums;
    sums.alloc(blocks);
    k_scan_block<<<(unsigned)blocks, 1024, 0, st>>>(n, in, out, sums.p);
    const int64_t* total_src = sums.p;   // one block: its sum is the total
    DArray<int64_t> offs;
    if (blocks > 1) {
        // scan of the block sums (recursion ends at one block), then the block offsets
        offs.alloc(blocks + 1);
        exclusive_scan(sums.p, offs.p, blocks, st);
        k_scan_add<<<(unsigned)blocks, 1024, 0, st>>>(n, out, offs.p);
        total_src = offs.p + blocks;
    }
    KNP_CUDA(cudaMemcpyAsync(out + n, total_src, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    int64_t total = 0;
    KNP_CUDA(cudaMemcpyAsync(&total, total_src, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    KNP_CUDA(cudaStreamSynchronize(st));
    return total;
}

// ------------------------------------------------------------------ level basics

// diagonal, D^-1 (with an empty field row given a unit diagonal, as on the host), |s_ii|
__global__ void k_diag(int64_t n, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                       double* __restrict__ val, const double* __restrict__ s, double* __restrict__ dinv,
                       double* __restrict__ sdiag, int* __restrict__ bad) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t td = -1;
    for (int64_t t = ptr[i]; t < ptr[i + 1]; ++t)
        if (col[t] == i) td = t;
    if (td < 0) {
        atomicExch(bad, 1);
        return;
    }
    sdiag[i] = fabs(s ? s[td] : val[4 * td + 3]);   // before the empty-row fix, as on the host
    for (int f = 0; f < 4; ++f) {
        double d = val[4 * td + f];
        if (d == 0.0) {
            bool empty = true;
            for (int64_t t = ptr[i]; t < ptr[i + 1]; ++t) empty &= val[4 * t + f] == 0.0;
            if (empty) val[4 * td + f] = d = 1.0;
        }
        if (!(d > 0.0) || !isfinite(d)) atomicExch(bad, 2);
        dinv[4 * i + f] = 1.0 / d;
    }
}

__global__ void k_power_init(int64_t n4, double* __restrict__ x) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n4) x[i] = 1.0 + 0.5 * ((hash32((uint32_t)i) & 1023) / 1023.0);
}

// y = D^-1 A x per field; partial sums of |y|^2 and |x|^2 per field
__global__ void k_power_step(int64_t n, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                             const double* __restrict__ val, const double* __restrict__ dinv,
                             const double* __restrict__ x, double* __restrict__ y, double* __restrict__ partial) {
    __shared__ double sh[8][256];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s[4] = {0, 0, 0, 0};
        for (int64_t t = ptr[i]; t < ptr[i + 1]; ++t)
            for (int f = 0; f < 4; ++f) s[f] += val[4 * t + f] * x[4 * (int64_t)col[t] + f];
        for (int f = 0; f < 4; ++f) {
            double v = dinv[4 * i + f] * s[f];
            y[4 * i + f] = v;
            acc[f] += v * v;
            acc[4 + f] += x[4 * i + f] * x[4 * i + f];
        }
    }
    for (int k = 0; k < 8; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int k = 0; k < 8; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 8) partial[blockIdx.x * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_power_scale(int64_t n4, int nblocks, const double* __restrict__ partial, const double* __restrict__ y,
                              double* __restrict__ x, double* __restrict__ lam) {
    __shared__ double tot[8];
    if (threadIdx.x < 8) {
        double s = 0;
        for (int b = 0; b < nblocks; ++b) s += partial[b * 8 + threadIdx.x];
        tot[threadIdx.x] = s;
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x < 4)
        lam[threadIdx.x] = sqrt(tot[threadIdx.x] / fmax(tot[4 + threadIdx.x], 1e-300));
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = y[i] * (1.0 / sqrt(fmax(tot[i & 3], 1e-300)));
}

// ------------------------------------------------------------------ strength graph
__global__ void k_strength_count(int64_t n, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                 const double* __restrict__ s, const double* __restrict__ sdiag, double theta,
                                 int64_t* __restrict__ cnt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t c = 0;
    for (int64_t t = ptr[i]; t < ptr[i + 1]; ++t) {
        int64_t j = col[t];
        if (j == i) continue;
        if (fabs(s[t]) >= theta * sqrt(sdiag[i] * sdiag[j]) && s[t] != 0.0) ++c;
    }
    cnt[i] = c;
}

__global__ void k_strength_fill(int64_t n, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                const double* __restrict__ s, const double* __restrict__ sdiag, double theta,
                                const int64_t* __restrict__ gptr, int32_t* __restrict__ gadj) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t q = gptr[i];
    for (int64_t t = ptr[i]; t < ptr[i + 1]; ++t) {
        int64_t j = col[t];
        if (j == i) continue;
        if (fabs(s[t]) >= theta * sqrt(sdiag[i] * sdiag[j]) && s[t] != 0.0) gadj[q++] = (int32_t)j;
    }
}

// ------------------------------------------------------------------ MIS-2
__device__ __forceinline__ uint64_t mis_key(uint8_t st, uint64_t prio) {
    return st == 0 ? prio : (st == 1 ? ~0ULL : 0ULL);
}

__global__ void k_mis2_init(int64_t n, int level, const int64_t* __restrict__ gptr, uint8_t* __restrict__ state,
                            uint64_t* __restrict__ prio) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    prio[i] = ((uint64_t)hash32((uint32_t)i * 2654435761u + (uint32_t)level * 97u) << 32) | (uint64_t)i;
    state[i] = (gptr[i] == gptr[i + 1]) ? 1 : 0;   // isolated nodes are singleton roots
}

__global__ void k_mis2_max1(int64_t n, const int64_t* __restrict__ gptr, const int32_t* __restrict__ gadj,
                            const uint8_t* __restrict__ state, const uint64_t* __restrict__ prio,
                            uint64_t* __restrict__ m1) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t v = mis_key(state[i], prio[i]);
    for (int64_t t = gptr[i]; t < gptr[i + 1]; ++t) {
        int64_t j = gadj[t];
        v = max(v, mis_key(state[j], prio[j]));
    }
    m1[i] = v;
}

__global__ void k_mis2_max2(int64_t n, const int64_t* __restrict__ gptr, const int32_t* __restrict__ gadj,
                            const uint64_t* __restrict__ m1, uint64_t* __restrict__ m2) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t v = m1[i];
    for (int64_t t = gptr[i]; t < gptr[i + 1]; ++t) v = max(v, m1[gadj[t]]);
    m2[i] = v;
}

__global__ void k_mis2_update(int64_t n, const uint64_t* __restrict__ m2, const uint64_t* __restrict__ prio,
                              uint8_t* __restrict__ state, unsigned long long* __restrict__ undecided) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || state[i] != 0) return;
    if (m2[i] == prio[i])
        state[i] = 1;
    else if (m2[i] == ~0ULL)
        state[i] = 2;
    else
        atomicAdd(undecided, 1ULL);
}

__global__ void k_flag(int64_t n, const uint8_t* __restrict__ state, uint8_t v, int64_t* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = state[i] == v ? 1 : 0;
}

__global__ void k_root_ids(int64_t n, const uint8_t* __restrict__ state, const int64_t* __restrict__ rank,
                           int32_t* __restrict__ agg) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) agg[i] = state[i] == 1 ? (int32_t)rank[i] : -1;
}

__global__ void k_root_neighbours(int64_t n, const int64_t* __restrict__ gptr, const int32_t* __restrict__ gadj,
                                  const uint8_t* __restrict__ state, int32_t* __restrict__ agg) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || state[i] != 1) return;
    // neighbourhoods of roots are disjoint (roots are at distance >= 3)
    for (int64_t t = gptr[i]; t < gptr[i + 1]; ++t) agg[gadj[t]] = agg[i];
}

__global__ void k_leftover(int64_t n, const int64_t* __restrict__ gptr, const int32_t* __restrict__ gadj,
                           const int32_t* __restrict__ agg_old, int32_t* __restrict__ agg_new, int* __restrict__ changed) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t a = agg_old[i];
    if (a < 0) {
        for (int64_t t = gptr[i]; t < gptr[i + 1]; ++t) {
            int32_t b = agg_old[gadj[t]];
            if (b >= 0) {
                a = b;
                *changed = 1;
                break;
            }
        }
    }
    agg_new[i] = a;
}

__global__ void k_unassigned(int64_t n, const int32_t* __restrict__ agg, int64_t* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = agg[i] < 0 ? 1 : 0;
}

__global__ void k_singletons(int64_t n, int64_t base, const int64_t* __restrict__ rank, int32_t* __restrict__ agg) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && agg[i] < 0) agg[i] = (int32_t)(base + rank[i]);
}

// ------------------------------------------------------------------ smoothed prolongator
constexpr int PMAX = 96;    // distinct aggregates in one row of P (longer rows: k_prolong_long)

// Row i of P: slots in order of first appearance (agg(i), then the aggregates of row i of A),
// accumulated in that order as on the host, then sorted by column; pass 0 counts, pass 1 writes.
// A row with more than PMAX distinct aggregates is left to k_prolong_long: pass 0 appends it to
// long_rows[*n_long] (pass 1 skips it).
__global__ void k_prolong(int64_t n, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                          const double* __restrict__ val, const double* __restrict__ dinv,
                          const double* __restrict__ B, const int32_t* __restrict__ agg, double om0, double om1,
                          double om2, double om3, double p_drop, int pass, int64_t* __restrict__ cnt,
                          const int64_t* __restrict__ pptr, int32_t* __restrict__ pcol, double* __restrict__ pval,
                          int64_t* __restrict__ long_rows, unsigned long long* __restrict__ n_long, int pmax) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double om[4] = {om0, om1, om2, om3};
    int32_t keys[PMAX];
    double acc[PMAX][4];
    int m = 0;
    auto slot = [&](int32_t c) -> int {
        for (int q = 0; q < m; ++q)
            if (keys[q] == c) return q;
        if (m >= pmax) return -1;
        keys[m] = c;
        for (int f = 0; f < 4; ++f) acc[m][f] = 0.0;
        return m++;
    };
    int q0 = slot(agg[i]);
    for (int f = 0; f < 4; ++f) acc[q0][f] += B[4 * i + f];
    for (int64_t t = ptr[i]; t < ptr[i + 1]; ++t) {
        int64_t j = col[t];
        int q = slot(agg[j]);
        if (q < 0) {
            if (!pass) {
                cnt[i] = 0;
                long_rows[atomicAdd(n_long, 1ULL)] = i;
            }
            return;
        }
        for (int f = 0; f < 4; ++f) acc[q][f] -= om[f] * dinv[4 * i + f] * val[4 * t + f] * B[4 * j + f];
    }
    // sort slots by column (insertion sort on a permutation)
    int order[PMAX];
    for (int q = 0; q < m; ++q) {
        int k = q;
        while (k > 0 && keys[order[k - 1]] > keys[q]) {
            order[k] = order[k - 1];
            --k;
        }
        order[k] = q;
    }
    double rmax[4] = {0, 0, 0, 0};
    for (int q = 0; q < m; ++q)
        for (int f = 0; f < 4; ++f) rmax[f] = fmax(rmax[f], fabs(acc[q][f]));
    int64_t w = pass ? pptr[i] : 0;
    int64_t c = 0;
    for (int k = 0; k < m; ++k) {
        int q = order[k];
        bool keep = keys[q] == agg[i] || p_drop <= 0;
        for (int f = 0; f < 4 && !keep; ++f) keep = fabs(acc[q][f]) >= p_drop * rmax[f];
        if (!keep) continue;
        if (pass) {
            pcol[w + c] = keys[q];
            for (int f = 0; f < 4; ++f) pval[4 * (w + c) + f] = acc[q][f];
        }
        ++c;
    }
    if (!pass) cnt[i] = c;
}

// ------------------------------------------------------------------ long rows
// Rows with more distinct columns than the register slots of k_prolong or the shared-memory hash
// of the SpGEMM hold are finished by one block per row with a dense accumulator over the n_cols
// output columns in global memory: acc [n_cols][4] and mark [n_cols], one such workspace per
// block, zero between rows. The terms reach each output slot in the same order as in the
// short-row kernels and on the host (one thread adds a P row's terms one after another; the
// SpGEMM adds the entries of one row of B at a time, whose columns are distinct), so the values
// are the same. Reading the marks in column order gives the row sorted.

// Ordered compaction of the marked columns of [0, n_cols): emit(c, rank) for every c with
// mark[c] != 0, rank = the number of marked columns before c. Returns the count. Called by all
// threads of the block (blockDim.x a multiple of 32, at most 1024).
template <class Emit>
__device__ int64_t block_marked_scan(int64_t n_cols, const int32_t* __restrict__ mark, Emit emit) {
    __shared__ int wcnt[32];
    __shared__ int64_t base_s, chunk_s;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) base_s = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < n_cols; c0 += blockDim.x) {
        const int64_t c = c0 + tid;
        const bool m = c < n_cols && mark[c] != 0;
        const unsigned bal = __ballot_sync(0xffffffffu, m);
        if (lane == 0) wcnt[wid] = __popc(bal);
        __syncthreads();
        if (tid == 0) {
            int s = 0;
            for (int w = 0; w < nw; ++w) {
                const int t = wcnt[w];
                wcnt[w] = s;
                s += t;
            }
            chunk_s = s;
        }
        __syncthreads();
        if (m) emit(c, base_s + wcnt[wid] + __popc(bal & ((1u << lane) - 1u)));
        __syncthreads();
        if (tid == 0) base_s += chunk_s;
        __syncthreads();
    }
    return base_s;
}

// Long rows of P (see k_prolong): pass 0 writes cnt[i], pass 1 the row at pptr[i].
__global__ void __launch_bounds__(256) k_prolong_long(int64_t n_long, const int64_t* __restrict__ rows, int64_t na,
                                                      const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                                      const double* __restrict__ val, const double* __restrict__ dinv,
                                                      const double* __restrict__ B, const int32_t* __restrict__ agg,
                                                      double om0, double om1, double om2, double om3, double p_drop,
                                                      int pass, int64_t* __restrict__ cnt,
                                                      const int64_t* __restrict__ pptr, int32_t* __restrict__ pcol,
                                                      double* __restrict__ pval, double* __restrict__ ws_acc,
                                                      int32_t* __restrict__ ws_mark) {
    double* acc = ws_acc + (int64_t)blockIdx.x * na * 4;
    int32_t* mark = ws_mark + (int64_t)blockIdx.x * na;
    __shared__ double rmax[4];
    const double om[4] = {om0, om1, om2, om3};
    for (int64_t q = blockIdx.x; q < n_long; q += gridDim.x) {
        const int64_t i = rows[q];
        const int64_t a0 = ptr[i], a1 = ptr[i + 1];
        const int64_t ai = agg[i];
        if (threadIdx.x == 0) mark[ai] = 1;
        for (int64_t t = a0 + threadIdx.x; t < a1; t += blockDim.x) mark[agg[col[t]]] = 1;
        if (threadIdx.x == 0) {
            for (int f = 0; f < 4; ++f) acc[4 * ai + f] += B[4 * i + f];
            for (int64_t t = a0; t < a1; ++t) {
                const int64_t j = col[t], aj = agg[j];
                for (int f = 0; f < 4; ++f) acc[4 * aj + f] -= om[f] * dinv[4 * i + f] * val[4 * t + f] * B[4 * j + f];
            }
        }
        __syncthreads();
        if (threadIdx.x < 4) {
            const int f = threadIdx.x;
            double r = fabs(acc[4 * ai + f]);
            for (int64_t t = a0; t < a1; ++t) r = fmax(r, fabs(acc[4 * (int64_t)agg[col[t]] + f]));
            rmax[f] = r;
        }
        __syncthreads();
        if (p_drop > 0) {
            for (int64_t t = a0 + threadIdx.x; t < a1; t += blockDim.x) {
                const int64_t c = agg[col[t]];
                bool keep = c == ai;
                for (int f = 0; f < 4 && !keep; ++f) keep = fabs(acc[4 * c + f]) >= p_drop * rmax[f];
                if (!keep) mark[c] = 0;
            }
            __syncthreads();
        }
        const int64_t w = pass ? pptr[i] : 0;
        const int64_t m = block_marked_scan(na, mark, [&](int64_t c, int64_t r) {
            if (pass) {
                pcol[w + r] = (int32_t)c;
                for (int f = 0; f < 4; ++f) pval[4 * (w + r) + f] = acc[4 * c + f];
            }
        });
        if (!pass && threadIdx.x == 0) cnt[i] = m;
        // clear the workspace for the next row
        if (threadIdx.x == 0) {
            mark[ai] = 0;
            for (int f = 0; f < 4; ++f) acc[4 * ai + f] = 0.0;
        }
        for (int64_t t = a0 + threadIdx.x; t < a1; t += blockDim.x) {
            const int64_t c = agg[col[t]];
            mark[c] = 0;
            for (int f = 0; f < 4; ++f) acc[4 * c + f] = 0.0;
        }
        __syncthreads();
    }
}

// Long rows of C = A B (see row_keys): pass 0 writes cnt[row], pass 1 the sorted row at cptr[row].
__global__ void __launch_bounds__(256) k_spgemm_long(int64_t n_long, const int64_t* __restrict__ rows, int64_t n_cols,
                                                     const int64_t* __restrict__ aptr, const int32_t* __restrict__ acol,
                                                     const double* __restrict__ aval, const int64_t* __restrict__ bptr,
                                                     const int32_t* __restrict__ bcol, const double* __restrict__ bval,
                                                     int pass, int64_t* __restrict__ cnt,
                                                     const int64_t* __restrict__ cptr, int32_t* __restrict__ ccol,
                                                     double* __restrict__ cval, double* __restrict__ ws_acc,
                                                     int32_t* __restrict__ ws_mark) {
    double* acc = ws_acc + (int64_t)blockIdx.x * n_cols * 4;
    int32_t* mark = ws_mark + (int64_t)blockIdx.x * n_cols;
    for (int64_t q = blockIdx.x; q < n_long; q += gridDim.x) {
        const int64_t row = rows[q];
        for (int64_t t = aptr[row]; t < aptr[row + 1]; ++t) {
            const int64_t k = acol[t];
            const double a[4] = {aval[4 * t], aval[4 * t + 1], aval[4 * t + 2], aval[4 * t + 3]};
            for (int64_t u = bptr[k] + threadIdx.x; u < bptr[k + 1]; u += blockDim.x) {
                const int64_t c = bcol[u];
                mark[c] = 1;
                if (pass)
                    for (int f = 0; f < 4; ++f) acc[4 * c + f] += a[f] * bval[4 * u + f];
            }
            if (pass) __syncthreads();   // the next row of B may hit the same columns
        }
        __syncthreads();
        const int64_t w = pass ? cptr[row] : 0;
        const int64_t m = block_marked_scan(n_cols, mark, [&](int64_t c, int64_t r) {
            if (pass) {
                ccol[w + r] = (int32_t)c;
                for (int f = 0; f < 4; ++f) cval[4 * (w + r) + f] = acc[4 * c + f];
            }
        });
        if (!pass && threadIdx.x == 0) cnt[row] = m;
        for (int64_t t = aptr[row]; t < aptr[row + 1]; ++t) {
            const int64_t k = acol[t];
            for (int64_t u = bptr[k] + threadIdx.x; u < bptr[k + 1]; u += blockDim.x) {
                const int64_t c = bcol[u];
                mark[c] = 0;
                for (int f = 0; f < 4; ++f) acc[4 * c + f] = 0.0;
            }
        }
        __syncthreads();
    }
}

// Workspace for the long-row kernels: as many blocks as rows, within `budget` bytes.
struct LongRowWork {
    DArray<double> acc;
    DArray<int32_t> mark;
    unsigned blocks = 0;
    void setup(int64_t n_long, int64_t n_cols, cudaStream_t st, size_t budget = size_t(1) << 30) {
        const size_t per = (size_t)std::max<int64_t>(n_cols, 1) * (4 * sizeof(double) + sizeof(int32_t));
        const int64_t fit = (int64_t)std::max<size_t>(1, budget / per);
        blocks = (unsigned)std::min<int64_t>({n_long, fit, 4096});
        acc.alloc((size_t)blocks * std::max<int64_t>(n_cols, 1) * 4);
        mark.alloc((size_t)blocks * std::max<int64_t>(n_cols, 1));
        acc.zero(st);
        mark.zero(st);
    }
};

__global__ void k_coarse_B(int64_t n, const int32_t* __restrict__ agg, const double* __restrict__ B,
                           unsigned long long* __restrict__ Bc_bits) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    // max over aggregate members; B >= 0, so the IEEE bit patterns order like the values
    for (int f = 0; f < 4; ++f)
        atomicMax(&Bc_bits[4 * (int64_t)agg[i] + f], (unsigned long long)__double_as_longlong(B[4 * i + f]));
}

// ------------------------------------------------------------------ transpose
__global__ void k_col_count(int64_t nnz, const int32_t* __restrict__ col, unsigned long long* __restrict__ cnt) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < nnz) atomicAdd(&cnt[col[t]], 1ULL);
}

__global__ void k_transpose_fill(int64_t n, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                 const double* __restrict__ val, const int64_t* __restrict__ rptr,
                                 unsigned long long* __restrict__ fill, int32_t* __restrict__ rcol,
                                 double* __restrict__ rval) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t t = ptr[i]; t < ptr[i + 1]; ++t) {
        int64_t c = col[t];
        int64_t q = rptr[c] + (int64_t)atomicAdd(&fill[c], 1ULL);
        rcol[q] = (int32_t)i;
        for (int f = 0; f < 4; ++f) rval[4 * q + f] = val[4 * t + f];
    }
}

// sort each row of a CSR4 by column with one block per row: the (column, position) pairs of a row
// of up to SORT_MAX entries are bitonic-sorted in shared memory and the four values gathered in
// that order; longer rows fall back to the serial sort above. Columns within a row are distinct,
// so the result equals that of any other sort.
constexpr int SORT_MAX = 1024;
constexpr int SORT_THREADS = 256;
__global__ void __launch_bounds__(SORT_THREADS) k_sort_rows_block(int64_t n, const int64_t* __restrict__ ptr,
                                                                  int32_t* __restrict__ col,
                                                                  double* __restrict__ val) {
    __shared__ int32_t key[SORT_MAX];
    __shared__ int32_t pos[SORT_MAX];
    __shared__ double vs[4 * SORT_MAX];
    const int64_t i = blockIdx.x;
    if (i >= n) return;
    const int64_t a0 = ptr[i];
    const int len = (int)(ptr[i + 1] - a0);
    if (len <= 1) return;
    if (len > SORT_MAX) {
        if (threadIdx.x == 0) {
            for (int64_t a = a0 + 1; a < a0 + len; ++a) {
                int32_t c = col[a];
                double v[4] = {val[4 * a], val[4 * a + 1], val[4 * a + 2], val[4 * a + 3]};
                int64_t b = a;
                while (b > a0 && col[b - 1] > c) {
                    col[b] = col[b - 1];
                    for (int f = 0; f < 4; ++f) val[4 * b + f] = val[4 * (b - 1) + f];
                    --b;
                }
                col[b] = c;
                for (int f = 0; f < 4; ++f) val[4 * b + f] = v[f];
            }
        }
        return;
    }
    int m = 1;
    while (m < len) m <<= 1;
    for (int k = threadIdx.x; k < m; k += SORT_THREADS) {
        key[k] = k < len ? col[a0 + k] : INT32_MAX;
        pos[k] = k;
    }
    for (int k = threadIdx.x; k < 4 * len; k += SORT_THREADS) vs[k] = val[4 * a0 + k];
    __syncthreads();
    for (int size = 2; size <= m; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int k = threadIdx.x; k < m; k += SORT_THREADS) {
                const int l = k ^ stride;
                if (l > k) {
                    const bool up = (k & size) == 0;
                    if ((key[k] > key[l]) == up) {
                        const int32_t tk = key[k];
                        key[k] = key[l];
                        key[l] = tk;
                        const int32_t tp = pos[k];
                        pos[k] = pos[l];
                        pos[l] = tp;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int k = threadIdx.x; k < len; k += SORT_THREADS) {
        col[a0 + k] = key[k];
        for (int f = 0; f < 4; ++f) val[4 * (a0 + k) + f] = vs[4 * pos[k] + f];
    }
}

// ------------------------------------------------------------------ SpGEMM C = A B (four fields)
// One warp per row of C. The keys of the row go through an open-addressing hash set in shared
// memory (capacity hcap, at most hcap/2 keys), are compacted and bitonic-sorted. In the value
// pass the entries of row i of A are taken one after another (the host's order) and the lanes
// share the entries of the matching row of B, whose keys are distinct, so each output slot
// receives its terms in the same order as on the host and no atomics are needed.
__device__ __forceinline__ int hash_insert(int32_t* table, int hcap, int32_t key, int* count) {
    uint32_t h = hash32((uint32_t)key) & (hcap - 1);
    while (true) {
        int32_t prev = atomicCAS(&table[h], -1, key);
        if (prev == -1) {
            atomicAdd(count, 1);
            return (int)h;
        }
        if (prev == key) return (int)h;
        h = (h + 1) & (hcap - 1);
    }
}

__device__ void warp_bitonic_sort(int32_t* a, int m, int lane) {
    // a[0..m) padded to the next power of two with INT_MAX by the caller
    for (int k = 2; k <= m; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < m; i += 32) {
                int l = i ^ j;
                if (l > i) {
                    bool up = (i & k) == 0;
                    int32_t x = a[i], y = a[l];
                    if ((x > y) == up) {
                        a[i] = y;
                        a[l] = x;
                    }
                }
            }
            __syncwarp();
        }
}

// keys of row `row` of C into sorted[0..count); returns count, or -1 when the row has kcap keys or
// more (kcap <= hcap / 2 keeps the table at most half full)
__device__ int row_keys(int64_t row, const int64_t* __restrict__ aptr, const int32_t* __restrict__ acol,
                        const int64_t* __restrict__ bptr, const int32_t* __restrict__ bcol, int32_t* table,
                        int32_t* sorted, int hcap, int kcap, int* count, int lane) {
    for (int h = lane; h < hcap; h += 32) table[h] = -1;
    if (lane == 0) *count = 0;
    __syncwarp();
    for (int64_t t = aptr[row]; t < aptr[row + 1]; ++t) {
        int64_t k = acol[t];
        for (int64_t u = bptr[k] + lane; u < bptr[k + 1]; u += 32) {
            if (*count < kcap) hash_insert(table, hcap, bcol[u], count);
        }
        __syncwarp();
        if (*count >= kcap) return -1;
    }
    __syncwarp();
    int m = *count;
    // compact
    __shared__ int cpos[32];
    if (lane == 0) cpos[threadIdx.x / 32] = 0;
    __syncwarp();
    for (int h = lane; h < hcap; h += 32) {
        int32_t key = table[h];
        if (key >= 0) sorted[atomicAdd(&cpos[threadIdx.x / 32], 1)] = key;
    }
    __syncwarp();
    int p2 = 1;
    while (p2 < m) p2 <<= 1;
    for (int i = m + lane; i < p2; i += 32) sorted[i] = 0x7fffffff;
    __syncwarp();
    warp_bitonic_sort(sorted, p2, lane);
    return m;
}

__global__ void k_spgemm_count(int64_t n, const int64_t* __restrict__ aptr, const int32_t* __restrict__ acol,
                               const int64_t* __restrict__ bptr, const int32_t* __restrict__ bcol, int hcap,
                               int kcap, int64_t* __restrict__ cnt, int64_t* __restrict__ long_rows,
                               unsigned long long* __restrict__ n_long) {
    extern __shared__ int32_t smem[];
    const int wib = threadIdx.x / 32, lane = threadIdx.x % 32, wpb = blockDim.x / 32;
    int32_t* table = smem + (int64_t)wib * (2 * hcap + 1);
    int32_t* sorted = table + hcap;
    int* count = sorted + hcap;
    int64_t row = (int64_t)blockIdx.x * wpb + wib;
    if (row >= n) return;
    int m = row_keys(row, aptr, acol, bptr, bcol, table, sorted, hcap, kcap, count, lane);
    if (lane == 0) {
        if (m < 0) long_rows[atomicAdd(n_long, 1ULL)] = row;   // finished by k_spgemm_long
        cnt[row] = m < 0 ? 0 : m;
    }
}

__global__ void k_spgemm_fill(int64_t n, const int64_t* __restrict__ aptr, const int32_t* __restrict__ acol,
                              const double* __restrict__ aval, const int64_t* __restrict__ bptr,
                              const int32_t* __restrict__ bcol, const double* __restrict__ bval, int hcap,
                              int kcap, const int64_t* __restrict__ cptr, int32_t* __restrict__ ccol,
                              double* __restrict__ cval) {
    extern __shared__ int32_t smem[];
    const int wib = threadIdx.x / 32, lane = threadIdx.x % 32, wpb = blockDim.x / 32;
    int32_t* table = smem + (int64_t)wib * (2 * hcap + 1);
    int32_t* sorted = table + hcap;
    int* count = sorted + hcap;
    int64_t row = (int64_t)blockIdx.x * wpb + wib;
    if (row >= n) return;
    int m = row_keys(row, aptr, acol, bptr, bcol, table, sorted, hcap, kcap, count, lane);
    if (m < 0) return;
    const int64_t base = cptr[row];
    double* out = cval + 4 * base;
    for (int q = lane; q < m; q += 32) {
        ccol[base + q] = sorted[q];
        for (int f = 0; f < 4; ++f) out[4 * q + f] = 0.0;
    }
    __syncwarp();
    for (int64_t t = aptr[row]; t < aptr[row + 1]; ++t) {
        int64_t k = acol[t];
        double a[4] = {aval[4 * t], aval[4 * t + 1], aval[4 * t + 2], aval[4 * t + 3]};
        for (int64_t u = bptr[k] + lane; u < bptr[k + 1]; u += 32) {
            int32_t key = bcol[u];
            int lo = 0, hi = m - 1;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (sorted[mid] < key)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            for (int f = 0; f < 4; ++f) out[4 * lo + f] += a[f] * bval[4 * u + f];
        }
        __syncwarp();
    }
}

__global__ void k_row_bound(int64_t n, const int64_t* __restrict__ aptr, const int32_t* __restrict__ acol,
                            const int64_t* __restrict__ bptr, unsigned long long* __restrict__ maxb) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long b = 0;
    for (int64_t t = aptr[i]; t < aptr[i + 1]; ++t) b += bptr[acol[t] + 1] - bptr[acol[t]];
    atomicMax(maxb, b);
}

// B = 1 per field except the pinned row's potential field (the near-null vectors of P_0)
__global__ void k_near_null(int64_t n4, int64_t pin4, double* __restrict__ b) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n4) b[i] = i == pin4 ? 0.0 : 1.0;
}

// the potential field of every entry (the strength scalar of the coarser levels)
__global__ void k_field3(int64_t nnz, const double* __restrict__ val, double* __restrict__ out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < nnz) out[t] = val[4 * t + 3];
}

// ------------------------------------------------------------------ P_0 from A_0 (Eq. 4.4)
// Row r of the region pattern: the sliced-ELL row up to its padding, which repeats the row id
// after the sorted columns.
__device__ __forceinline__ int64_t sell_row_len(int64_t r, const int64_t* __restrict__ slice_ptr,
                                                const int32_t* __restrict__ scol) {
    const int64_t s = r / SELL_C, base = slice_ptr[s] + r % SELL_C;
    const int64_t w = (slice_ptr[s + 1] - slice_ptr[s]) / SELL_C;
    int32_t prev = -1;
    int64_t k = 0;
    for (; k < w; ++k) {
        const int32_t c = scol[base + k * SELL_C];
        if (c <= prev) break;
        prev = c;
    }
    return k;
}

__global__ void k_p0_count(int64_t n, const int64_t* __restrict__ slice_ptr, const int32_t* __restrict__ scol,
                           int64_t* __restrict__ cnt) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n) cnt[r] = sell_row_len(r, slice_ptr, scol);
}

// Field values of P_0 per entry: c^k rows M + tau_r^k A; the potential row sum_k z_k e^k (which is
// sum_k z_k tau~_r^k A_r^{k,0} + C_m/F M_Gamma on the pattern); the pinned row and column of phi_e
// become the identity. Also the strength scalar (a) and the diagonal of every field.
__global__ void k_p0_fill(int64_t n, int64_t N_i, const int64_t* __restrict__ slice_ptr,
                          const int32_t* __restrict__ scol, const double* __restrict__ m, const double* __restrict__ a,
                          const double* __restrict__ e, int64_t ne, RegionCoef ri, RegionCoef re, double z0,
                          double z1, double z2, int64_t pin, const int64_t* __restrict__ ptr, int32_t* __restrict__ col,
                          double* __restrict__ val, double* __restrict__ strength, double* __restrict__ diag) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const RegionCoef& rc = r < N_i ? ri : re;
    const double z[3] = {z0, z1, z2};
    const int64_t s = r / SELL_C, base = slice_ptr[s] + r % SELL_C;
    const int64_t len = ptr[r + 1] - ptr[r];
    for (int f = 0; f < 4; ++f) diag[4 * r + f] = 0.0;
    for (int64_t k = 0; k < len; ++k) {
        const int64_t pos = base + k * SELL_C, t = ptr[r] + k;
        const int32_t c = scol[pos];
        double v[4];
        v[3] = 0;
        for (int i = 0; i < KI; ++i) {
            v[i] = m[pos] + rc.tau[i] * a[pos];
            v[3] += z[i] * e[i * ne + pos];
        }
        if (r == pin) v[3] = (c == r) ? 1.0 : 0.0;
        if (c == pin && r != pin) v[3] = 0.0;
        col[t] = c;
        for (int f = 0; f < 4; ++f) {
            val[4 * t + f] = v[f];
            if (c == r) diag[4 * r + f] = v[f];
        }
        strength[t] = a[pos];
    }
}

// S = sqrt(diag P_0), S^-1, and S with the pinned row left out of the stopping test's norms
__global__ void k_p0_scaling(int64_t n4, int64_t pin4, const double* __restrict__ diag, double* __restrict__ sv,
                             double* __restrict__ si, double* __restrict__ sw, int* __restrict__ bad) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n4) return;
    const double d = diag[i];
    if (!(d > 0.0) || !isfinite(d)) atomicExch(bad, 1);
    const double r = sqrt(d);
    sv[i] = r;
    si[i] = 1.0 / r;
    sw[i] = i == pin4 ? 0.0 : r;
}

// C = A B on the device. Rows whose keys overflow the shared-memory hash (more than hcap/2 of
// them) are finished by k_spgemm_long; the number of such rows is added to *long_rows_out.
void spgemm_gpu(const DevCsr4d& A, const DevCsr4d& B, DevCsr4d& C, cudaStream_t st, int64_t* long_rows_out,
                int short_row_max) {
    const int64_t n = A.n_rows;
    DArray<unsigned long long> maxb;
    maxb.alloc(1);
    maxb.zero(st);
    k_row_bound<<<nb(n, 256), 256, 0, st>>>(n, A.ptr.p, A.col.p, B.ptr.p, maxb.p);
    unsigned long long bound = 0;
    KNP_CUDA(cudaMemcpyAsync(&bound, maxb.p, sizeof(bound), cudaMemcpyDeviceToHost, st));
    KNP_CUDA(cudaStreamSynchronize(st));
    int64_t want = (int64_t)std::min<unsigned long long>(bound, (unsigned long long)B.n_cols);
    int hcap = 64;
    while (hcap < 2 * want + 2 && hcap < 8192) hcap <<= 1;
    const int kcap = short_row_max > 0 ? std::min(hcap / 2, short_row_max) : hcap / 2;
    const int wpb = hcap <= 1024 ? 4 : 1;
    const size_t smem = (size_t)wpb * (2 * hcap + 1) * sizeof(int32_t);
    if (smem > 48 * 1024) {
        KNP_CUDA(cudaFuncSetAttribute(k_spgemm_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        KNP_CUDA(cudaFuncSetAttribute(k_spgemm_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    DArray<int64_t> cnt, long_rows;
    DArray<unsigned long long> n_long;
    cnt.alloc(n);
    long_rows.alloc(std::max<int64_t>(n, 1));
    n_long.alloc(1);
    n_long.zero(st);
    const unsigned grid = (unsigned)((n + wpb - 1) / wpb);
    k_spgemm_count<<<grid, 32 * wpb, smem, st>>>(n, A.ptr.p, A.col.p, B.ptr.p, B.col.p, hcap, kcap, cnt.p, long_rows.p,
                                                 n_long.p);
    unsigned long long nl = 0;
    KNP_CUDA(cudaMemcpyAsync(&nl, n_long.p, sizeof(nl), cudaMemcpyDeviceToHost, st));
    KNP_CUDA(cudaStreamSynchronize(st));
    LongRowWork ws;
    if (nl) {
        ws.setup((int64_t)nl, B.n_cols, st);
        k_spgemm_long<<<ws.blocks, 256, 0, st>>>((int64_t)nl, long_rows.p, B.n_cols, A.ptr.p, A.col.p, A.val.p,
                                                 B.ptr.p, B.col.p, B.val.p, 0, cnt.p, nullptr, nullptr, nullptr,
                                                 ws.acc.p, ws.mark.p);
    }
    C.n_rows = n;
    C.n_cols = B.n_cols;
    C.ptr.alloc(n + 1);
    C.nnz = exclusive_scan(cnt.p, C.ptr.p, n, st);
    C.col.alloc(std::max<int64_t>(1, C.nnz));
    C.val.alloc(std::max<int64_t>(1, 4 * C.nnz));
    k_spgemm_fill<<<grid, 32 * wpb, smem, st>>>(n, A.ptr.p, A.col.p, A.val.p, B.ptr.p, B.col.p, B.val.p, hcap,
                                                kcap, C.ptr.p, C.col.p, C.val.p);
    if (nl)
        k_spgemm_long<<<ws.blocks, 256, 0, st>>>((int64_t)nl, long_rows.p, B.n_cols, A.ptr.p, A.col.p, A.val.p,
                                                 B.ptr.p, B.col.p, B.val.p, 1, nullptr, C.ptr.p, C.col.p, C.val.p,
                                                 ws.acc.p, ws.mark.p);
    KNP_CUDA(cudaGetLastError());
    if (long_rows_out) *long_rows_out += (int64_t)nl;
}

}  // namespace

int64_t device_exclusive_scan(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st) {
    return exclusive_scan(in, out, n, st);
}

void download(const DevCsr4d& d, HostCsr4& h, cudaStream_t st) {
    h.n_rows = d.n_rows;
    h.n_cols = d.n_cols;
    d.ptr.download(h.ptr, st);
    d.col.download(h.col, st);
    d.val.download(h.val, st);
    h.col.resize(d.nnz);
    h.val.resize(4 * d.nnz);
    KNP_CUDA(cudaStreamSynchronize(st));
}

void p0_extract(knp_problem* p, DevCsr4d& A0, DArray<double>& strength) {
    cudaStream_t st = p->stream;
    const int64_t n = p->n_nodes;
    const SellPattern& S = p->sell;
    A0.n_rows = A0.n_cols = n;
    DArray<int64_t> cnt;
    cnt.alloc(n);
    k_p0_count<<<nb(n, 256), 256, 0, st>>>(n, S.slice_ptr.p, S.col.p, cnt.p);
    A0.ptr.alloc(n + 1);
    A0.nnz = exclusive_scan(cnt.p, A0.ptr.p, n, st);
    A0.col.alloc(std::max<int64_t>(1, A0.nnz));
    A0.val.alloc(std::max<int64_t>(1, 4 * A0.nnz));
    strength.alloc(std::max<int64_t>(1, A0.nnz));
    DArray<double> diag;
    diag.alloc(4 * n);
    k_p0_fill<<<nb(n, 128), 128, 0, st>>>(n, p->N_i, S.slice_ptr.p, S.col.p, p->sell_m.p, p->sell_a.p, p->sell_e.p,
                                          S.n_entries, p->sp.reg[0], p->sp.reg[1], p->sp.z[0], p->sp.z[1], p->sp.z[2],
                                          p->pin, A0.ptr.p, A0.col.p, A0.val.p, strength.p, diag.p);
    DArray<int> bad;
    bad.alloc(1);
    bad.zero(st);
    k_p0_scaling<<<nb(4 * n, 256), 256, 0, st>>>(4 * n, 4 * (int64_t)p->pin + 3, diag.p, p->svec.p, p->sinv.p,
                                                 p->swt.p, bad.p);
    int hb = 0;
    KNP_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    KNP_CUDA(cudaStreamSynchronize(st));
    KNP_REQUIRE(hb == 0, KNP_ERR_NUMERIC, "P_0 diagonal is not positive");
}

// Device version of amg_build (same algorithm and output as the host one, see amg_setup.cpp).
void amg_build_gpu(DevCsr4d& A0, DArray<double>& s, int64_t pin_row, const AmgSetupOpts& o, GpuHierarchy& H,
                   cudaStream_t st, int short_row_max) {
    H.levels.clear();
    H.long_rows_p = H.long_rows_rap = 0;
    const int pmax = short_row_max > 0 ? std::min(short_row_max, PMAX) : PMAX;
    DArray<double> B;
    B.alloc(4 * A0.n_rows);
    k_near_null<<<nb(4 * A0.n_rows, 256), 256, 0, st>>>(4 * A0.n_rows, pin_row >= 0 ? 4 * pin_row + 3 : -1, B.p);
    DArray<int> flag;
    flag.alloc(1);
    auto cur = std::make_unique<GpuLevel>();
    cur->A = std::move(A0);
    for (int lev = 0;; ++lev) {
        GpuLevel& L = *cur;
        DevCsr4d& A = L.A;
        const int64_t n = A.n_rows;
        H.levels.push_back(std::move(cur));
        // diagonal, D^-1, Chebyshev bounds
        DArray<double> sdiag;
        L.dinv.alloc(4 * n);
        sdiag.alloc(n);
        flag.zero(st);
        k_diag<<<nb(n, 256), 256, 0, st>>>(n, A.ptr.p, A.col.p, A.val.p, lev == 0 ? s.p : nullptr, L.dinv.p,
                                            sdiag.p, flag.p);
        int bad = 0;
        KNP_CUDA(cudaMemcpyAsync(&bad, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        KNP_CUDA(cudaStreamSynchronize(st));
        KNP_REQUIRE(bad == 0, KNP_ERR_NUMERIC, "P_0 hierarchy: %s on level %d",
                    bad == 1 ? "missing diagonal" : "non-positive diagonal", lev);
        {
            DArray<double> x, y, partial, lam;
            x.alloc(4 * n);
            y.alloc(4 * n);
            const int pb = (int)std::min<int64_t>(1024, nb(n, 256));
            partial.alloc(8 * pb);
            lam.alloc(4);
            k_power_init<<<nb(4 * n, 256), 256, 0, st>>>(4 * n, x.p);
            for (int it = 0; it < 20; ++it) {
                k_power_step<<<pb, 256, 0, st>>>(n, A.ptr.p, A.col.p, A.val.p, L.dinv.p, x.p, y.p, partial.p);
                k_power_scale<<<pb, 256, 0, st>>>(4 * n, pb, partial.p, y.p, x.p, lam.p);
            }
            double rho[4];
            KNP_CUDA(cudaMemcpyAsync(rho, lam.p, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
            KNP_CUDA(cudaStreamSynchronize(st));
            for (int f = 0; f < 4; ++f) {
                L.lmax[f] = 1.1 * rho[f];
                L.lmin[f] = L.lmax[f] / o.cheb_ratio;
            }
        }
        if (n <= o.coarse_max || lev + 1 >= o.max_levels) break;
        // strength graph (level 0: the given scalar; coarser: the potential field)
        const double theta = (lev == 0 || o.theta_coarse < 0) ? o.theta : o.theta_coarse;
        DArray<double> sc;
        const double* sv = s.p;
        if (lev > 0) {
            sc.alloc(std::max<int64_t>(1, A.nnz));
            k_field3<<<nb(A.nnz, 256), 256, 0, st>>>(A.nnz, A.val.p, sc.p);
            sv = sc.p;
        }
        DArray<int64_t> cnt, gptr;
        DArray<int32_t> gadj;
        cnt.alloc(n);
        gptr.alloc(n + 1);
        k_strength_count<<<nb(n, 256), 256, 0, st>>>(n, A.ptr.p, A.col.p, sv, sdiag.p, theta, cnt.p);
        int64_t ne = exclusive_scan(cnt.p, gptr.p, n, st);
        gadj.alloc(std::max<int64_t>(1, ne));
        k_strength_fill<<<nb(n, 256), 256, 0, st>>>(n, A.ptr.p, A.col.p, sv, sdiag.p, theta, gptr.p, gadj.p);
        if (lev == 0) s.release();
        // MIS-2 rounds
        DArray<uint8_t> state;
        DArray<uint64_t> prio, m1, m2;
        DArray<unsigned long long> und;
        state.alloc(n);
        prio.alloc(n);
        m1.alloc(n);
        m2.alloc(n);
        und.alloc(1);
        k_mis2_init<<<nb(n, 256), 256, 0, st>>>(n, lev, gptr.p, state.p, prio.p);
        for (int round = 0; round < 1000; ++round) {
            und.zero(st);
            k_mis2_max1<<<nb(n, 256), 256, 0, st>>>(n, gptr.p, gadj.p, state.p, prio.p, m1.p);
            k_mis2_max2<<<nb(n, 256), 256, 0, st>>>(n, gptr.p, gadj.p, m1.p, m2.p);
            k_mis2_update<<<nb(n, 256), 256, 0, st>>>(n, m2.p, prio.p, state.p, und.p);
            unsigned long long u = 0;
            KNP_CUDA(cudaMemcpyAsync(&u, und.p, sizeof(u), cudaMemcpyDeviceToHost, st));
            KNP_CUDA(cudaStreamSynchronize(st));
            if (u == 0) break;
        }
        m1.release();
        m2.release();
        prio.release();
        // aggregates
        DArray<int64_t> fl, rank;
        fl.alloc(n);
        rank.alloc(n + 1);
        k_flag<<<nb(n, 256), 256, 0, st>>>(n, state.p, 1, fl.p);
        int64_t na = exclusive_scan(fl.p, rank.p, n, st);
        DArray<int32_t> agg, agg2;
        agg.alloc(n);
        agg2.alloc(n);
        k_root_ids<<<nb(n, 256), 256, 0, st>>>(n, state.p, rank.p, agg.p);
        k_root_neighbours<<<nb(n, 256), 256, 0, st>>>(n, gptr.p, gadj.p, state.p, agg.p);
        for (int pass = 0; pass < 8; ++pass) {
            flag.zero(st);
            k_leftover<<<nb(n, 256), 256, 0, st>>>(n, gptr.p, gadj.p, agg.p, agg2.p, flag.p);
            std::swap(agg.p, agg2.p);
            int ch = 0;
            KNP_CUDA(cudaMemcpyAsync(&ch, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
            KNP_CUDA(cudaStreamSynchronize(st));
            if (!ch) break;
        }
        k_unassigned<<<nb(n, 256), 256, 0, st>>>(n, agg.p, fl.p);
        int64_t extra = exclusive_scan(fl.p, rank.p, n, st);
        k_singletons<<<nb(n, 256), 256, 0, st>>>(n, na, rank.p, agg.p);
        na += extra;
        gadj.release();
        agg2.release();
        if (na >= n || na == 0 || (double)na > 0.85 * (double)n) break;
        // smoothed prolongator; rows with more than pmax aggregates go to k_prolong_long
        double om[4];
        for (int f = 0; f < 4; ++f) om[f] = (4.0 / 3.0) / (L.lmax[f] / 1.1);
        DevCsr4d& P = L.P;
        P.n_rows = n;
        P.n_cols = na;
        P.ptr.alloc(n + 1);
        DArray<int64_t> long_rows;
        DArray<unsigned long long> n_long;
        long_rows.alloc(n);
        n_long.alloc(1);
        n_long.zero(st);
        k_prolong<<<nb(n, 64), 64, 0, st>>>(n, A.ptr.p, A.col.p, A.val.p, L.dinv.p, B.p, agg.p, om[0], om[1], om[2],
                                            om[3], o.p_drop, 0, cnt.p, nullptr, nullptr, nullptr, long_rows.p, n_long.p,
                                            pmax);
        unsigned long long nl = 0;
        KNP_CUDA(cudaMemcpyAsync(&nl, n_long.p, sizeof(nl), cudaMemcpyDeviceToHost, st));
        KNP_CUDA(cudaStreamSynchronize(st));
        LongRowWork ws;
        if (nl) {
            ws.setup((int64_t)nl, na, st);
            k_prolong_long<<<ws.blocks, 256, 0, st>>>((int64_t)nl, long_rows.p, na, A.ptr.p, A.col.p, A.val.p,
                                                      L.dinv.p, B.p, agg.p, om[0], om[1], om[2], om[3], o.p_drop, 0,
                                                      cnt.p, nullptr, nullptr, nullptr, ws.acc.p, ws.mark.p);
            H.long_rows_p += (int64_t)nl;
        }
        P.nnz = exclusive_scan(cnt.p, P.ptr.p, n, st);
        P.col.alloc(std::max<int64_t>(1, P.nnz));
        P.val.alloc(std::max<int64_t>(1, 4 * P.nnz));
        k_prolong<<<nb(n, 64), 64, 0, st>>>(n, A.ptr.p, A.col.p, A.val.p, L.dinv.p, B.p, agg.p, om[0], om[1], om[2],
                                            om[3], o.p_drop, 1, nullptr, P.ptr.p, P.col.p, P.val.p, long_rows.p,
                                            n_long.p, pmax);
        if (nl)
            k_prolong_long<<<ws.blocks, 256, 0, st>>>((int64_t)nl, long_rows.p, na, A.ptr.p, A.col.p, A.val.p,
                                                      L.dinv.p, B.p, agg.p, om[0], om[1], om[2], om[3], o.p_drop, 1,
                                                      nullptr, P.ptr.p, P.col.p, P.val.p, ws.acc.p, ws.mark.p);
        long_rows.release();
        // R = P^T
        DevCsr4d& R = L.R;
        R.n_rows = na;
        R.n_cols = n;
        R.nnz = P.nnz;
        {
            DArray<unsigned long long> cc, fill;
            cc.alloc(na);
            cc.zero(st);
            fill.alloc(na);
            fill.zero(st);
            k_col_count<<<nb(P.nnz, 256), 256, 0, st>>>(P.nnz, P.col.p, cc.p);
            DArray<int64_t> cc64;
            cc64.alloc(na);
            KNP_CUDA(cudaMemcpyAsync(cc64.p, cc.p, na * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
            R.ptr.alloc(na + 1);
            exclusive_scan(cc64.p, R.ptr.p, na, st);
            R.col.alloc(std::max<int64_t>(1, R.nnz));
            R.val.alloc(std::max<int64_t>(1, 4 * R.nnz));
            k_transpose_fill<<<nb(n, 256), 256, 0, st>>>(n, P.ptr.p, P.col.p, P.val.p, R.ptr.p, fill.p, R.col.p,
                                                         R.val.p);
            k_sort_rows_block<<<(unsigned)na, SORT_THREADS, 0, st>>>(na, R.ptr.p, R.col.p, R.val.p);
        }
        // coarse near-null vectors
        DArray<unsigned long long> Bc;
        Bc.alloc(4 * na);
        Bc.zero(st);
        k_coarse_B<<<nb(n, 256), 256, 0, st>>>(n, agg.p, B.p, Bc.p);
        // Galerkin product
        auto next = std::make_unique<GpuLevel>();
        {
            DevCsr4d AP;
            spgemm_gpu(A, P, AP, st, &H.long_rows_rap, short_row_max);
            spgemm_gpu(R, AP, next->A, st, &H.long_rows_rap, short_row_max);
        }
        B.alloc(4 * na);
        KNP_CUDA(cudaMemcpyAsync(B.p, Bc.p, 4 * na * sizeof(double), cudaMemcpyDeviceToDevice, st));
        KNP_CUDA(cudaGetLastError());
        cur = std::move(next);
    }
    // dense inverse of the coarsest operator on the host (a few hundred unknowns)
    HostHierarchy Hc;
    Hc.levels.emplace_back();
    download(H.levels.back()->A, Hc.levels.back().A, st);
    amg_coarse_inverse(Hc);
    H.coarse_inv = std::move(Hc.coarse_inv);
    H.nc = Hc.nc;
}

}  // namespace knp
