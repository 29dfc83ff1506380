// One V-cycle of the smoothed-aggregation hierarchy on P_0, the inexact P_0^{-1} of
// Section 4.2 (the paper uses one BoomerAMG V-cycle; here smoothed aggregation with
// Chebyshev smoothing, all four fields of a node in one pass). Templated on the
// storage/arithmetic type of the hierarchy: double (plain FP64 form) or float (the
// mixed-precision form; the coarsest dense solve is FP64 in both).
//
// Layouts: a level operator with short rows (the finest, about 15 entries per row in 3D) or
// with enough rows to fill the GPU one thread per row is sliced-ELL with one thread per row;
// the other operators and the transfer operators are CSR processed by groups of 4 x S threads
// per row, one thread per (field, entry slot): each thread does one multiply-add per entry and
// the group reduces one value per field over its S slots (S a power of two chosen from the mean
// row length), so that the short, wide coarse levels still fill the GPU without spending the
// slow FP64 pipe on four-value reductions.
//
// Smoothing: Chebyshev steps on [lambda_max / ratio, 1.1 lambda_max] per field, `pre` of them
// before the coarse-grid correction (the first from x = 0 costs no operator product) and
// `degree` after; one before and two after by default, which makes the V-cycle non-symmetric
// (FGMRES takes any preconditioner; CG(P_0) is given as many steps before as after).
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <type_traits>

#include "amg.h"
#include "amg_gpu.h"
#include "problem.h"
#include "vcycle.h"

namespace knp {

namespace {

template <class T>
struct V4;
template <>
struct V4<double> {
    double v[4];
    __device__ __forceinline__ static V4 load(const double* p) {
        const double2* q = reinterpret_cast<const double2*>(p);
        double2 a = q[0], b = q[1];
        return V4{{a.x, a.y, b.x, b.y}};
    }
    __device__ __forceinline__ void store(double* p) const {
        double2* q = reinterpret_cast<double2*>(p);
        q[0] = make_double2(v[0], v[1]);
        q[1] = make_double2(v[2], v[3]);
    }
};
template <>
struct V4<float> {
    float v[4];
    __device__ __forceinline__ static V4 load(const float* p) {
        float4 a = *reinterpret_cast<const float4*>(p);
        return V4{{a.x, a.y, a.z, a.w}};
    }
    __device__ __forceinline__ void store(float* p) const {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};

struct Coef4 {
    double c1[4], c2[4];
};

// Row product of a sliced-ELL operator (one thread per row)
template <class T>
__device__ __forceinline__ void sell_row(int64_t r, const int64_t* __restrict__ sp, const int32_t* __restrict__ col,
                                         const T* __restrict__ val, const T* __restrict__ x, T acc[4]) {
    int64_t s = r / SELL_C;
    int64_t base = sp[s] + r % SELL_C;
    int64_t w = (sp[s + 1] - sp[s]) / SELL_C;
    acc[0] = acc[1] = acc[2] = acc[3] = T(0);
    for (int64_t k = 0; k < w; ++k) {
        int64_t pos = base + k * SELL_C;
        V4<T> a = V4<T>::load(val + 4 * pos);
        V4<T> xv = V4<T>::load(x + 4 * (int64_t)col[pos]);
        for (int f = 0; f < 4; ++f) acc[f] += a.v[f] * xv.v[f];
    }
}

// Field f of a CSR row product, by a group of 4 x S lanes (lane = 4 x slot + f): slot k takes
// entries k, k + S, ... of the row, and the S partial sums of each field are combined by
// shuffles (and, for S > 8, across the row's warps through shared memory); every lane of the
// group gets its field's sum. Blocks are 128 threads. Every thread of the block must call this
// (full-mask shuffles, and a block barrier for S > 8); rows r >= n pass active = false and
// contribute nothing.
template <class T, int S>
__device__ __forceinline__ T csr_row_field(bool active, int64_t r, int slot, int f, const int64_t* __restrict__ ptr,
                                           const int32_t* __restrict__ col, const T* __restrict__ val,
                                           const T* __restrict__ x) {
    static_assert(S >= 1 && S <= 32 && (S & (S - 1)) == 0, "slots: a power of two up to 32");
    T acc = T(0);
    if (active) {
        const int64_t t1 = ptr[r + 1];
        for (int64_t t = ptr[r] + slot; t < t1; t += S) acc += val[4 * t + f] * x[4 * (int64_t)col[t] + f];
    }
    constexpr int SW = S < 8 ? S : 8;   // slots of the row inside one warp
    for (int o = 2 * SW; o >= 4; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, 4 * SW);
    if constexpr (S > 8) {
        constexpr int NW = S / 8;   // warps per row
        __shared__ T part[4][4];    // [warp of the block][field]
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) < 4) part[w][threadIdx.x & 31] = acc;
        __syncthreads();
        const int w0 = w - w % NW;
        acc = T(0);
        for (int k = 0; k < NW; ++k) acc += part[w0 + k][f];
    }
    return acc;
}

__device__ __forceinline__ double pick4(const double c[4], int f) {
    return f == 0 ? c[0] : f == 1 ? c[1] : f == 2 ? c[2] : c[3];
}

// The coarse correction's input at node i: t = s .* v - (A Z y)_i. Row i of A Z y: its same-region
// phi columns hold its own group's constant (the row sums RS), its cross-region entries their
// groups' constants; the potential row is sum_k z_k of the concentration rows' terms, and the
// pinned potential row (the identity) gives 0.
__device__ __forceinline__ void defl_input(int64_t i, const double* __restrict__ v, const double* __restrict__ s,
                                           const DeflFuse& df, double t[4]) {
    const double yr = df.y[i < df.N_i ? df.rgrp[i] : df.ext_group];
    double ae[3];
    for (int q = 0; q < 3; ++q) ae[q] = df.RS[3 * i + q] * yr;
    for (int u = df.xptr[i]; u < df.xptr[i + 1]; ++u) {
        const int gq = df.xg[u];
        if (gq < 0) continue;
        const double yc = df.y[gq];
        for (int q = 0; q < 3; ++q) ae[q] += df.xe[q * df.n_cross + u] * yc;
    }
    double out3 = df.z[0] * ae[0] + df.z[1] * ae[1] + df.z[2] * ae[2];
    if (i == df.pin) out3 = 0.0;
    for (int q = 0; q < 3; ++q) t[q] = s[4 * i + q] * v[4 * i + q] - ae[q];
    t[3] = s[4 * i + 3] * v[4 * i + 3] - out3;
}

// first Chebyshev step from x = 0: d = c2 D^-1 b, x = d. On the finest level b = s .* v (double
// input), or s .* v - A Z y inside the coarse correction (df.y set).
template <class T>
__global__ void k_cheb_first(int64_t n, const double* __restrict__ v, const double* __restrict__ s, T* __restrict__ b,
                             const T* __restrict__ dinv, Coef4 c, T* __restrict__ x, T* __restrict__ d, DeflFuse df) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    V4<T> bb;
    if (v && df.y) {
        double t[4];
        defl_input(i, v, s, df, t);
        for (int f = 0; f < 4; ++f) bb.v[f] = (T)t[f];
        bb.store(b + 4 * i);
    } else if (v) {
        for (int f = 0; f < 4; ++f) bb.v[f] = (T)(s[4 * i + f] * v[4 * i + f]);
        bb.store(b + 4 * i);
    } else {
        bb = V4<T>::load(b + 4 * i);
    }
    V4<T> di = V4<T>::load(dinv + 4 * i), dd;
    for (int f = 0; f < 4; ++f) dd.v[f] = (T)c.c2[f] * di.v[f] * bb.v[f];
    dd.store(d + 4 * i);
    dd.store(x + 4 * i);
}

// Chebyshev update of one row given acc = (A x_in)_row
template <class T>
__device__ __forceinline__ void cheb_update(int64_t i, const T acc[4], const T* __restrict__ x_in,
                                            const T* __restrict__ b, const T* __restrict__ dinv, const Coef4& c,
                                            T* __restrict__ d, T* __restrict__ x_out) {
    V4<T> bb = V4<T>::load(b + 4 * i), di = V4<T>::load(dinv + 4 * i), dd = V4<T>::load(d + 4 * i),
          xx = V4<T>::load(x_in + 4 * i);
    for (int f = 0; f < 4; ++f) {
        dd.v[f] = (T)c.c1[f] * dd.v[f] + (T)c.c2[f] * di.v[f] * (bb.v[f] - acc[f]);
        xx.v[f] += dd.v[f];
    }
    dd.store(d + 4 * i);
    xx.store(x_out + 4 * i);
}

// Chebyshev step: r = b - A x_in; d = c1 d + c2 D^-1 r; x_out = x_in + d
template <class T>
__global__ void __launch_bounds__(128) k_cheb_sell(int64_t n, const int64_t* __restrict__ sp,
                                                   const int32_t* __restrict__ col, const T* __restrict__ val,
                                                   const T* __restrict__ x_in, const T* __restrict__ b,
                                                   const T* __restrict__ dinv, Coef4 c, T* __restrict__ d,
                                                   T* __restrict__ x_out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    T acc[4];
    sell_row<T>(i, sp, col, val, x_in, acc);
    cheb_update<T>(i, acc, x_in, b, dinv, c, d, x_out);
}

template <class T, int S>
__global__ void __launch_bounds__(128) k_cheb_csr(int64_t n, const int64_t* __restrict__ ptr,
                                                  const int32_t* __restrict__ col, const T* __restrict__ val,
                                                  const T* __restrict__ x_in, const T* __restrict__ b,
                                                  const T* __restrict__ dinv, Coef4 c, T* __restrict__ d,
                                                  T* __restrict__ x_out) {
    int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
    int64_t i = g / (4 * S);
    int lane = (int)(g % (4 * S)), f = lane & 3;
    T acc = csr_row_field<T, S>(i < n, i, lane >> 2, f, ptr, col, val, x_in);
    if (lane < 4 && i < n) {
        const int64_t k = 4 * i + f;
        T dd = (T)pick4(c.c1, f) * d[k] + (T)pick4(c.c2, f) * dinv[k] * (b[k] - acc);
        d[k] = dd;
        x_out[k] = x_in[k] + dd;
    }
}

template <class T>
__global__ void __launch_bounds__(128) k_resid_sell(int64_t n, const int64_t* __restrict__ sp,
                                                    const int32_t* __restrict__ col, const T* __restrict__ val,
                                                    const T* __restrict__ x, const T* __restrict__ b,
                                                    T* __restrict__ r) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    T acc[4];
    sell_row<T>(i, sp, col, val, x, acc);
    V4<T> bb = V4<T>::load(b + 4 * i);
    for (int f = 0; f < 4; ++f) bb.v[f] -= acc[f];
    bb.store(r + 4 * i);
}

// y = A x on a sliced-ELL level
template <class T>
__global__ void __launch_bounds__(128) k_sell_apply(int64_t n, const int64_t* __restrict__ sp,
                                                    const int32_t* __restrict__ col, const T* __restrict__ val,
                                                    const T* __restrict__ x, T* __restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    T acc[4];
    sell_row<T>(i, sp, col, val, x, acc);
    V4<T>{{acc[0], acc[1], acc[2], acc[3]}}.store(y + 4 * i);
}

template <class T, int S>
__global__ void __launch_bounds__(128) k_resid_csr(int64_t n, const int64_t* __restrict__ ptr,
                                                   const int32_t* __restrict__ col, const T* __restrict__ val,
                                                   const T* __restrict__ x, const T* __restrict__ b,
                                                   T* __restrict__ r) {
    int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
    int64_t i = g / (4 * S);
    int lane = (int)(g % (4 * S)), f = lane & 3;
    T acc = csr_row_field<T, S>(i < n, i, lane >> 2, f, ptr, col, val, x);
    if (lane < 4 && i < n) r[4 * i + f] = b[4 * i + f] - acc;
}

// y[i] (+)= (M x)[i] for a CSR with four values per entry (restriction and prolongation)
template <class T, int S>
__global__ void __launch_bounds__(128) k_csr4(int64_t n, const int64_t* __restrict__ ptr,
                                              const int32_t* __restrict__ col, const T* __restrict__ val,
                                              const T* __restrict__ x, T* __restrict__ y, int accumulate) {
    int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
    int64_t i = g / (4 * S);
    int lane = (int)(g % (4 * S)), f = lane & 3;
    T acc = csr_row_field<T, S>(i < n, i, lane >> 2, f, ptr, col, val, x);
    if (lane < 4 && i < n) {
        const int64_t k = 4 * i + f;
        y[k] = accumulate ? y[k] + acc : acc;
    }
}

// x_f = Ainv_f b_f on the coarsest level, FP64; one warp per (field, row)
template <class T>
__global__ void k_coarse(int64_t nc, const double* __restrict__ inv, const T* __restrict__ b, T* __restrict__ x) {
    int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    int lane = threadIdx.x % 32;
    if (wid >= 4 * nc) return;
    int f = (int)(wid / nc);
    int64_t row = wid % nc;
    const double* a = inv + ((int64_t)f * nc + row) * nc;
    double s = 0.0;
    for (int64_t j = lane; j < nc; j += 32) s += a[j] * (double)b[4 * j + f];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) x[4 * row + f] = (T)s;
}

template <class T>
__global__ void k_to_double(int64_t n4, const T* __restrict__ x, double* __restrict__ z) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n4) z[i] = (double)x[i];
}

// z = x + Z y: the V-cycle's output in FP64, every potential but the pinned one raised by its
// group's constant of the coarse correction
template <class T>
__global__ void k_out_defl(int64_t n, const T* __restrict__ x, double* __restrict__ z, DeflFuse df) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const V4<T> xx = V4<T>::load(x + 4 * r);
    double o3 = (double)xx.v[3];
    if (r != df.pin) o3 += df.y[r < df.N_i ? df.rgrp[r] : df.ext_group];
    double2* zp = reinterpret_cast<double2*>(z + 4 * r);
    zp[0] = make_double2((double)xx.v[0], (double)xx.v[1]);
    zp[1] = make_double2((double)xx.v[2], o3);
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <class T>
std::vector<T> cast_vec(const std::vector<double>& v) {
    return std::vector<T>(v.begin(), v.end());
}

// entry slots per row, a power of two up to 32 (4 x S threads per row): doubled while the grid
// stays within about two waves of 152 SMs x 2048 threads and each slot keeps at least two entries
int pick_slots(int64_t rows, double mean_len) {
    int sl = 1;
    while (sl < 32 && (double)rows * 4 * (2 * sl) <= 622592.0 && 4 * sl <= mean_len) sl *= 2;
    return sl;
}

}  // namespace

template <class T>
__global__ void k_cast(int64_t n, const double* __restrict__ in, T* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (T)in[i];
}

// device array of T from one of doubles: taken over as it is (T = double) or cast (T = float)
template <class T>
void take_values(DArray<T>& out, DArray<double>& in, int64_t count, cudaStream_t st) {
    if constexpr (std::is_same<T, double>::value) {
        out = std::move(in);
    } else {
        out.alloc(std::max<int64_t>(count, 1));
        if (count) k_cast<T><<<(unsigned)((count + 255) / 256), 256, 0, st>>>(count, in.p, out.p);
        KNP_CUDA(cudaStreamSynchronize(st));
        in.release();
    }
}

template <class T>
struct DevCsr4 {
    int64_t n = 0;
    int slots = 1;
    DArray<int64_t> ptr;
    DArray<int32_t> col;
    DArray<T> val;
    void upload(const HostCsr4& h, cudaStream_t st) {
        n = h.n_rows;
        slots = pick_slots(n, n ? (double)h.nnz() / (double)n : 1.0);
        ptr.upload(h.ptr, st);
        col.upload(h.col, st);
        val.upload(cast_vec<T>(h.val), st);
    }
    // takes over a device CSR built by the GPU setup (no copy through the host)
    void take(DevCsr4d& d, cudaStream_t st) {
        n = d.n_rows;
        slots = pick_slots(n, n ? (double)d.nnz / (double)n : 1.0);
        ptr = std::move(d.ptr);
        col = std::move(d.col);
        take_values(val, d.val, 4 * d.nnz, st);
    }
};

template <class T>
struct DevLevel {
    int64_t n = 0, nnz = 0;
    bool sell = false;
    // sliced ELL (every level whose padding is small)
    DArray<int64_t> sp;
    DArray<int32_t> scol;
    DArray<T> sval;
    // CSR (levels too irregular for sliced ELL)
    DevCsr4<T> A;
    DArray<T> dinv;
    double lmax[4], lmin[4];
    DevCsr4<T> P, R;
    DArray<T> x, x2, b, r, d;
};

template <class T>
struct AmgDev {
    std::vector<std::unique_ptr<DevLevel<T>>> L;
    DArray<double> cinv;
    int64_t nc = 0;
    int degree = 2;                          // Chebyshev steps after the coarse-grid correction
    int pre = 1;                             // and before it (the first from x = 0: no operator product)
    std::vector<std::vector<Coef4>> coef;   // per level: coefficients of each Chebyshev step
};

AmgHierarchy::~AmgHierarchy() {
    for (auto& kv : graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (gstream) cudaStreamDestroy(gstream);
    delete static_cast<AmgDev<double>*>(h64);
    delete static_cast<AmgDev<float>*>(h32);
}

// A level's operator is stored sliced-ELL (one thread per row, the value loads of a warp
// contiguous) if its rows are short (at most SELL_SHORT_ROW entries on average), or if they are
// long but there are enough of them to keep the GPU busy with one thread each (at least
// SELL_MIN_LONG_ROWS); and in either case only if padding every slice to its longest row stores
// at most SELL_MAX_STORED entries per nonzero. Otherwise CSR with 4 S lanes per row. Measured:
// the 512-cell 256^3 workload's first coarse level (1.7M rows of 58 entries) is 2.4% faster per
// FGMRES iteration as sliced ELL; P2's first coarse level at 32^3 (19.5k rows of 143 entries, four
// warps per SM with one thread per row) made the step 1.8 times slower.
constexpr double SELL_MAX_STORED = 2.0;
constexpr double SELL_SHORT_ROW = 24.0;
constexpr int64_t SELL_MIN_LONG_ROWS = 152 * 1024;

static bool sell_suits(int64_t rows, int64_t nnz) {
    return (double)nnz <= SELL_SHORT_ROW * (double)std::max<int64_t>(rows, 1) || rows >= SELL_MIN_LONG_ROWS;
}

// sliced ELL of a host CSR level; false (nothing done) if the level does not suit it (sell_suits,
// SELL_MAX_STORED)
template <class T>
static bool upload_sell(DevLevel<T>& L, const HostCsr4& A, cudaStream_t st) {
    const int64_t n = A.n_rows;
    int64_t ns = (n + SELL_C - 1) / SELL_C;
    std::vector<int64_t> sp(ns + 1, 0);
    for (int64_t s = 0; s < ns; ++s) {
        int64_t w = 0;
        for (int64_t r = s * SELL_C; r < std::min(n, (s + 1) * SELL_C); ++r) w = std::max(w, A.ptr[r + 1] - A.ptr[r]);
        sp[s + 1] = sp[s] + w * SELL_C;
    }
    if (!sell_suits(n, A.nnz()) || (double)sp[ns] > SELL_MAX_STORED * (double)std::max<int64_t>(A.nnz(), 1))
        return false;
    std::vector<int32_t> col(sp[ns]);
    std::vector<T> val(4 * sp[ns], T(0));
    for (int64_t s = 0; s < ns; ++s) {
        int64_t w = (sp[s + 1] - sp[s]) / SELL_C;
        for (int64_t lane = 0; lane < SELL_C; ++lane) {
            int64_t r = s * SELL_C + lane;
            int64_t len = r < n ? A.ptr[r + 1] - A.ptr[r] : 0;
            for (int64_t k = 0; k < w; ++k) {
                int64_t pos = sp[s] + k * SELL_C + lane;
                if (k < len) {
                    int64_t t = A.ptr[r] + k;
                    col[pos] = A.col[t];
                    for (int f = 0; f < 4; ++f) val[4 * pos + f] = (T)A.val[4 * t + f];
                } else {
                    col[pos] = (int32_t)std::min<int64_t>(r, n - 1);
                }
            }
        }
    }
    L.sp.upload(sp, st);
    L.scol.upload(col, st);
    L.sval.upload(val, st);
    return true;
}

// work vectors of a level and the coefficients of its Chebyshev steps (Saad's three-term
// recurrence on [lmin, lmax])
template <class T>
static void level_vectors_and_coefs(AmgDev<T>& D, DevLevel<T>& L, int degree, cudaStream_t st) {
    for (DArray<T>* v : {&L.x, &L.x2, &L.b, &L.r, &L.d}) {
        v->alloc(4 * L.n);
        v->zero(st);
    }
    std::vector<Coef4> cs(std::max(degree, 1));
    for (int f = 0; f < 4; ++f) {
        double th = 0.5 * (L.lmax[f] + L.lmin[f]), de = 0.5 * (L.lmax[f] - L.lmin[f]);
        double sigma = th / de;
        double rho0 = 1.0 / sigma;
        cs[0].c1[f] = 0.0;
        cs[0].c2[f] = 1.0 / th;
        for (int k = 1; k < degree; ++k) {
            double rho1 = 1.0 / (2.0 * sigma - rho0);
            cs[k].c1[f] = rho1 * rho0;
            cs[k].c2[f] = 2.0 * rho1 / de;
            rho0 = rho1;
        }
    }
    D.coef.push_back(cs);
}

template <class T>
static void upload_hierarchy(AmgDev<T>& D, const HostHierarchy& H, int degree, int pre, cudaStream_t st) {
    D.degree = degree;
    D.pre = pre;
    for (size_t l = 0; l < H.levels.size(); ++l) {
        const HostLevel& HL = H.levels[l];
        auto L = std::make_unique<DevLevel<T>>();
        const int64_t n = HL.A.n_rows;
        L->n = n;
        L->nnz = HL.A.nnz();
        L->sell = upload_sell(*L, HL.A, st);
        if (!L->sell) L->A.upload(HL.A, st);
        L->dinv.upload(cast_vec<T>(HL.dinv), st);
        for (int f = 0; f < 4; ++f) {
            L->lmax[f] = HL.lmax[f];
            L->lmin[f] = HL.lmin[f];
        }
        if (HL.P.n_rows) {
            L->P.upload(HL.P, st);
            L->R.upload(HL.R, st);
        }
        level_vectors_and_coefs(D, *L, std::max(degree, pre), st);
        D.L.push_back(std::move(L));
    }
    D.nc = H.nc;
    D.cinv.upload(H.coarse_inv, st);
}

// sliced-ELL slice widths (entries per slice) from CSR row lengths
__global__ void k_sell_widths(int64_t n, int64_t ns, const int64_t* __restrict__ ptr, int64_t* __restrict__ w) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= ns) return;
    int64_t m = 0;
    for (int64_t r = s * SELL_C; r < min(n, (s + 1) * SELL_C); ++r) m = max(m, ptr[r + 1] - ptr[r]);
    w[s] = m * SELL_C;
}

// CSR -> sliced ELL; padding repeats the (clamped) row id with zero values, as upload_sell does
template <class T>
__global__ void k_sell_fill(int64_t n, int64_t ns, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                            const double* __restrict__ val, const int64_t* __restrict__ sp, int32_t* __restrict__ scol,
                            T* __restrict__ sval) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= ns * SELL_C) return;
    const int64_t s = r / SELL_C, lane = r % SELL_C;
    const int64_t w = (sp[s + 1] - sp[s]) / SELL_C;
    const int64_t len = r < n ? ptr[r + 1] - ptr[r] : 0;
    for (int64_t k = 0; k < w; ++k) {
        const int64_t pos = sp[s] + k * SELL_C + lane;
        if (k < len) {
            const int64_t t = ptr[r] + k;
            scol[pos] = col[t];
            for (int f = 0; f < 4; ++f) sval[4 * pos + f] = (T)val[4 * t + f];
        } else {
            scol[pos] = (int32_t)min(r, n - 1);
            for (int f = 0; f < 4; ++f) sval[4 * pos + f] = T(0);
        }
    }
}

// sliced ELL of a device CSR level (its CSR arrays released); false (nothing done) if the level
// does not suit it (sell_suits, SELL_MAX_STORED)
template <class T>
static bool take_sell(DevLevel<T>& L, DevCsr4d& A, cudaStream_t st) {
    const int64_t n = A.n_rows, ns = (n + SELL_C - 1) / SELL_C;
    if (!sell_suits(n, A.nnz)) return false;
    DArray<int64_t> w;
    w.alloc(std::max<int64_t>(ns, 1));
    k_sell_widths<<<nblk(ns, 256), 256, 0, st>>>(n, ns, A.ptr.p, w.p);
    DArray<int64_t> sp;
    sp.alloc(ns + 1);
    const int64_t total = device_exclusive_scan(w.p, sp.p, ns, st);
    if ((double)total > SELL_MAX_STORED * (double)std::max<int64_t>(A.nnz, 1)) return false;
    L.sp = std::move(sp);
    L.scol.alloc(std::max<int64_t>(total, 1));
    L.sval.alloc(std::max<int64_t>(4 * total, 1));
    k_sell_fill<T><<<nblk(ns * SELL_C, 128), 128, 0, st>>>(n, ns, A.ptr.p, A.col.p, A.val.p, L.sp.p, L.scol.p, L.sval.p);
    KNP_CUDA(cudaStreamSynchronize(st));
    A.ptr.release();
    A.col.release();
    A.val.release();
    return true;
}

// The same device hierarchy as upload_hierarchy, taken over from the GPU setup level by level
// (each level's setup arrays are released as soon as its V-cycle copy exists)
template <class T>
static void take_hierarchy(AmgDev<T>& D, GpuHierarchy& H, int degree, int pre, cudaStream_t st) {
    D.degree = degree;
    D.pre = pre;
    for (auto& G : H.levels) {
        auto L = std::make_unique<DevLevel<T>>();
        const int64_t n = G->A.n_rows;
        L->n = n;
        L->nnz = G->A.nnz;
        L->sell = take_sell(*L, G->A, st);
        if (!L->sell) L->A.take(G->A, st);
        take_values(L->dinv, G->dinv, 4 * n, st);
        for (int f = 0; f < 4; ++f) {
            L->lmax[f] = G->lmax[f];
            L->lmin[f] = G->lmin[f];
        }
        if (G->P.n_rows) {
            L->P.take(G->P, st);
            L->R.take(G->R, st);
        }
        level_vectors_and_coefs(D, *L, std::max(degree, pre), st);
        D.L.push_back(std::move(L));
    }
    D.nc = H.nc;
    D.cinv.upload(H.coarse_inv, st);
}

void amg_upload(knp_problem* p, const HostHierarchy& H, int precision, int degree, int pre) {
    delete p->amg;
    p->amg = new AmgHierarchy();
    p->amg->precision = precision;
    p->amg->levels = (int)H.levels.size();
    p->amg->use_graphs = std::getenv("KNP_NO_GRAPHS") == nullptr;
    for (const HostLevel& L : H.levels) {
        p->amg->nodes.push_back(L.A.n_rows);
        p->amg->nnz.push_back(L.A.nnz());
    }
    if (precision == KNP_PREC_FP32) {
        auto* D = new AmgDev<float>();
        p->amg->h32 = D;
        upload_hierarchy(*D, H, degree, pre, p->stream);
    } else {
        auto* D = new AmgDev<double>();
        p->amg->h64 = D;
        upload_hierarchy(*D, H, degree, pre, p->stream);
    }
    KNP_CUDA(cudaStreamSynchronize(p->stream));
}

void amg_take_gpu(knp_problem* p, GpuHierarchy& H, int precision, int degree, int pre) {
    delete p->amg;
    p->amg = new AmgHierarchy();
    p->amg->precision = precision;
    p->amg->levels = (int)H.levels.size();
    p->amg->use_graphs = std::getenv("KNP_NO_GRAPHS") == nullptr;
    p->amg->setup_on_gpu = 1;
    p->amg->long_rows_p = H.long_rows_p;
    p->amg->long_rows_rap = H.long_rows_rap;
    for (auto& L : H.levels) {
        p->amg->nodes.push_back(L->A.n_rows);
        p->amg->nnz.push_back(L->A.nnz);
    }
    if (precision == KNP_PREC_FP32) {
        auto* D = new AmgDev<float>();
        p->amg->h32 = D;
        take_hierarchy(*D, H, degree, pre, p->stream);
    } else {
        auto* D = new AmgDev<double>();
        p->amg->h64 = D;
        take_hierarchy(*D, H, degree, pre, p->stream);
    }
    H.levels.clear();
    KNP_CUDA(cudaStreamSynchronize(p->stream));
}

#define KNP_SLOT_DISPATCH(slots, KERNEL, grid_rows, ...)                                                   \
    switch (slots) {                                                                                       \
        case 1: KERNEL<T, 1><<<nblk((grid_rows) * 4, 128), 128, 0, st>>>(__VA_ARGS__); break;             \
        case 2: KERNEL<T, 2><<<nblk((grid_rows) * 8, 128), 128, 0, st>>>(__VA_ARGS__); break;             \
        case 4: KERNEL<T, 4><<<nblk((grid_rows) * 16, 128), 128, 0, st>>>(__VA_ARGS__); break;            \
        case 8: KERNEL<T, 8><<<nblk((grid_rows) * 32, 128), 128, 0, st>>>(__VA_ARGS__); break;            \
        case 16: KERNEL<T, 16><<<nblk((grid_rows) * 64, 128), 128, 0, st>>>(__VA_ARGS__); break;          \
        default: KERNEL<T, 32><<<nblk((grid_rows) * 128, 128), 128, 0, st>>>(__VA_ARGS__); break;         \
    }

template <class T>
static void cheb_step(DevLevel<T>& L, const Coef4& c, Profiler* pr, bool fine, cudaStream_t st) {
    count_launch();
    if (L.sell) {
        ProfScope ps(fine ? pr : nullptr, KC_CHEB_FINE, st);
        k_cheb_sell<T><<<nblk(L.n, 128), 128, 0, st>>>(L.n, L.sp.p, L.scol.p, L.sval.p, L.x.p, L.b.p, L.dinv.p, c,
                                                       L.d.p, L.x2.p);
    } else {
        ProfScope ps(fine ? pr : nullptr, KC_CHEB_FINE, st);
        KNP_SLOT_DISPATCH(L.A.slots, k_cheb_csr, L.n, L.n, L.A.ptr.p, L.A.col.p, L.A.val.p, L.x.p, L.b.p, L.dinv.p, c,
                         L.d.p, L.x2.p);
    }
    std::swap(L.x.p, L.x2.p);
}

template <class T>
static void residual(DevLevel<T>& L, Profiler* pr, bool fine, cudaStream_t st) {
    count_launch();
    ProfScope ps(fine ? pr : nullptr, KC_RESID_FINE, st);
    if (L.sell) {
        k_resid_sell<T><<<nblk(L.n, 128), 128, 0, st>>>(L.n, L.sp.p, L.scol.p, L.sval.p, L.x.p, L.b.p, L.r.p);
    } else {
        KNP_SLOT_DISPATCH(L.A.slots, k_resid_csr, L.n, L.n, L.A.ptr.p, L.A.col.p, L.A.val.p, L.x.p, L.b.p, L.r.p);
    }
}

template <class T>
static void csr_apply(DevCsr4<T>& M, const T* x, T* y, int accumulate, cudaStream_t st) {
    count_launch();
    KNP_SLOT_DISPATCH(M.slots, k_csr4, M.n, M.n, M.ptr.p, M.col.p, M.val.p, x, y, accumulate);
}

template <class T>
static void smooth(DevLevel<T>& L, const std::vector<Coef4>& cs, int degree, bool zero_start, const double* v,
                   const double* s, const DeflFuse& df, Profiler* pr, bool fine, cudaStream_t st) {
    int k0 = 0;
    if (zero_start) {
        count_launch();
        k_cheb_first<T><<<nblk(L.n, 256), 256, 0, st>>>(L.n, v, s, L.b.p, L.dinv.p, cs[0], L.x.p, L.d.p, df);
        k0 = 1;
    }
    for (int k = k0; k < degree; ++k) cheb_step(L, cs[k], pr, fine, st);
}

template <class T>
static void vcycle_rec(AmgDev<T>& D, int l, const double* v, const double* s, const DeflFuse& df, Profiler* pr,
                       cudaStream_t st) {
    DevLevel<T>& L = *D.L[l];
    const int last = (int)D.L.size() - 1;
    if (l == last) {
        if (v) {
            // single-level hierarchy: build b from the scaled input first
            Coef4 c0{};
            count_launch();
            k_cheb_first<T><<<nblk(L.n, 256), 256, 0, st>>>(L.n, v, s, L.b.p, L.dinv.p, c0, L.x.p, L.d.p, df);
        }
        count_launch();
        k_coarse<T><<<nblk(4 * D.nc * 32, 256), 256, 0, st>>>(D.nc, D.cinv.p, L.b.p, L.x.p);
        return;
    }
    DevLevel<T>& C = *D.L[l + 1];
    smooth(L, D.coef[l], D.pre, true, v, s, df, pr, l == 0, st);
    residual(L, pr, l == 0, st);
    csr_apply(L.R, L.r.p, C.b.p, 0, st);
    vcycle_rec(D, l + 1, nullptr, nullptr, DeflFuse{}, pr, st);
    csr_apply(L.P, C.x.p, L.x.p, 1, st);
    smooth(L, D.coef[l], D.degree, false, nullptr, nullptr, DeflFuse{}, pr, l == 0, st);
}

static void vcycle_launch(knp_problem* p, const double* v, const double* s, double* z, const DeflFuse& df,
                          cudaStream_t st) {
    if (p->amg->h32) {
        auto& D = *static_cast<AmgDev<float>*>(p->amg->h32);
        vcycle_rec(D, 0, v, s, df, &p->prof, st);
        count_launch();
        if (df.y)
            k_out_defl<float><<<nblk(D.L[0]->n, 256), 256, 0, st>>>(D.L[0]->n, D.L[0]->x.p, z, df);
        else
            k_to_double<float><<<nblk(4 * D.L[0]->n, 256), 256, 0, st>>>(4 * D.L[0]->n, D.L[0]->x.p, z);
    } else {
        auto& D = *static_cast<AmgDev<double>*>(p->amg->h64);
        vcycle_rec(D, 0, v, s, df, &p->prof, st);
        if (df.y) {
            count_launch();
            k_out_defl<double><<<nblk(D.L[0]->n, 256), 256, 0, st>>>(D.L[0]->n, D.L[0]->x.p, z, df);
        } else {
            KNP_CUDA(cudaMemcpyAsync(z, D.L[0]->x.p, 4 * D.L[0]->n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        }
    }
}

// z = V-cycle(P_0)(s .* v); v, s, z are [n][4] doubles on the device. The V-cycle is a fixed
// sequence of about 15 launches, so it is captured once per (v, s, z) into a CUDA graph (on a
// private stream, since the problem's stream may be the legacy one) and replayed on the
// problem's stream. Each replay starts from
// scratch (the first kernel writes b, x and d of the finest level), so replays are independent.
// While a kernel class is being profiled the launches go out one by one.
void p0_apply(knp_problem* p, const double* x, double* y) {
    KNP_REQUIRE(p->amg && p->amg->h64, KNP_ERR_STATE, "P_0 products need the FP64 hierarchy");
    DevLevel<double>& L = *static_cast<AmgDev<double>*>(p->amg->h64)->L[0];
    KNP_REQUIRE(L.sell, KNP_ERR_STATE, "the finest level is not sliced ELL");
    count_launch();
    k_sell_apply<double><<<nblk(L.n, 128), 128, 0, p->stream>>>(L.n, L.sp.p, L.scol.p, L.sval.p, x, y);
    KNP_CUDA(cudaGetLastError());
}

void vcycle_apply(knp_problem* p, const double* v, const double* s, double* z, const DeflFuse* dfp) {
    KNP_REQUIRE(p->amg, KNP_ERR_STATE, "knp_amg_setup has not been called");
    AmgHierarchy& H = *p->amg;
    cudaStream_t st = p->stream;
    const DeflFuse df = dfp ? *dfp : DeflFuse{};
    if (!H.use_graphs || p->prof.active >= 0) {
        ProfScope ps(&p->prof, KC_VCYCLE, st);
        vcycle_launch(p, v, s, z, df, st);
        KNP_CUDA(cudaGetLastError());
        return;
    }
    if (!H.gstream) {
        KNP_CUDA(cudaStreamCreateWithFlags(&H.gstream, cudaStreamNonBlocking));
    }
    // the correction's arrays are fixed per problem, so its y pointer identifies them
    auto key = std::make_tuple(v, s, z, df.y);
    auto it = H.graphs.find(key);
    if (it == H.graphs.end()) {
        VcycleGraph g;
        int64_t before = g_launches.load();
        KNP_CUDA(cudaStreamBeginCapture(H.gstream, cudaStreamCaptureModeThreadLocal));
        try {
            vcycle_launch(p, v, s, z, df, H.gstream);
        } catch (...) {
            cudaGraph_t tmp;
            cudaStreamEndCapture(H.gstream, &tmp);
            if (tmp) cudaGraphDestroy(tmp);
            throw;
        }
        cudaGraph_t graph = nullptr;
        KNP_CUDA(cudaStreamEndCapture(H.gstream, &graph));
        g.launches = (int)(g_launches.load() - before);
        g_launches.fetch_sub(g.launches);
        KNP_CUDA(cudaGraphInstantiate(&g.exec, graph, 0));
        cudaGraphDestroy(graph);
        it = H.graphs.emplace(key, g).first;
    }
    KNP_CUDA(cudaGraphLaunch(it->second.exec, st));
    count_launch(it->second.launches);
}

}  // namespace knp

// ---------------------------------------------------------------------------------------------
// Allocation-free variant of knp_apply_preconditioner (include/knp.h). Some callers cannot call
// cudaMalloc when they need the preconditioner: code running under a CUDA stream capture or a
// graph being built, callers whose memory is fixed up front by a host framework, and embedded or
// plugin hosts that forbid allocation after start-up. The variant runs the same kernels as the
// V-cycle above on the same hierarchy, but all of its work vectors (the per-level x, x', b, r, d,
// the unit scale vector and the two layout-conversion buffers) live in one file-scope static
// device array of KNP_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds until
// the process exits. Calls share that array, so two calls that overlap on the GPU (different
// streams, different problems, or different host threads) race on it and must be serialised.
// Nothing in the array needs to start at zero: every work vector is written before it is read.
// ---------------------------------------------------------------------------------------------

namespace knp {

namespace {

constexpr size_t KNP_NOALLOC_SCRATCH_BYTES = size_t(32) << 20;   // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[KNP_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch on the current device. Host code cannot use the symbol
// itself (on the host it names a stand-in, not device memory), so the address is looked up with
// cudaGetSymbolAddress once per device, with that device current, and cached.
std::mutex g_noalloc_mu;
std::map<int, void*> g_noalloc_addr;

unsigned char* noalloc_scratch() {
    int dev = -1;
    KNP_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    auto it = g_noalloc_addr.find(dev);
    if (it != g_noalloc_addr.end()) return static_cast<unsigned char*>(it->second);
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    KNP_REQUIRE(e == cudaSuccess && ptr, KNP_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                cudaGetErrorString(e));
    g_noalloc_addr[dev] = ptr;
    return static_cast<unsigned char*>(ptr);
}

__global__ void k_fill(int64_t n, double v, double* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = v;
}

// Eq. 4.3 order [c_i^1..c_i^3, phi_i, c_e^1..c_e^3, phi_e] <-> node-major [node][4]
__global__ void k_eq42_to_nodes(int64_t Ni, int64_t Ne, const double* __restrict__ a, double* __restrict__ out) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= Ni + Ne) return;
    for (int k = 0; k < 4; ++k)
        out[4 * g + k] = g < Ni ? a[(int64_t)k * Ni + g] : a[4 * Ni + (int64_t)k * Ne + (g - Ni)];
}

__global__ void k_nodes_to_eq42(int64_t Ni, int64_t Ne, const double* __restrict__ in, double* __restrict__ a) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= Ni + Ne) return;
    for (int k = 0; k < 4; ++k) {
        if (g < Ni)
            a[(int64_t)k * Ni + g] = in[4 * g + k];
        else
            a[4 * Ni + (int64_t)k * Ne + (g - Ni)] = in[4 * g + k];
    }
}

// per-level work vectors carved out of the static array
template <class T>
struct NaWork {
    T *x, *x2, *b, *r, *d;
};

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

template <class T>
static void na_cheb_step(DevLevel<T>& L, NaWork<T>& w, const Coef4& c, cudaStream_t st) {
    count_launch();
    if (L.sell) {
        k_cheb_sell<T><<<nblk(L.n, 128), 128, 0, st>>>(L.n, L.sp.p, L.scol.p, L.sval.p, w.x, w.b, L.dinv.p, c, w.d,
                                                       w.x2);
    } else {
        KNP_SLOT_DISPATCH(L.A.slots, k_cheb_csr, L.n, L.n, L.A.ptr.p, L.A.col.p, L.A.val.p, w.x, w.b, L.dinv.p, c, w.d,
                         w.x2);
    }
    std::swap(w.x, w.x2);
}

template <class T>
static void na_vcycle_rec(AmgDev<T>& D, std::vector<NaWork<T>>& W, int l, const double* v, const double* s,
                          cudaStream_t st) {
    DevLevel<T>& L = *D.L[l];
    NaWork<T>& w = W[l];
    const int last = (int)D.L.size() - 1;
    if (l == last) {
        if (v) {
            Coef4 c0{};
            count_launch();
            k_cheb_first<T><<<nblk(L.n, 256), 256, 0, st>>>(L.n, v, s, w.b, L.dinv.p, c0, w.x, w.d, DeflFuse{});
        }
        count_launch();
        k_coarse<T><<<nblk(4 * D.nc * 32, 256), 256, 0, st>>>(D.nc, D.cinv.p, w.b, w.x);
        return;
    }
    DevLevel<T>& C = *D.L[l + 1];
    NaWork<T>& wc = W[l + 1];
    const std::vector<Coef4>& cs = D.coef[l];
    count_launch();
    k_cheb_first<T><<<nblk(L.n, 256), 256, 0, st>>>(L.n, v, s, w.b, L.dinv.p, cs[0], w.x, w.d, DeflFuse{});
    for (int k = 1; k < D.pre; ++k) na_cheb_step(L, w, cs[k], st);
    count_launch();
    if (L.sell) {
        k_resid_sell<T><<<nblk(L.n, 128), 128, 0, st>>>(L.n, L.sp.p, L.scol.p, L.sval.p, w.x, w.b, w.r);
    } else {
        KNP_SLOT_DISPATCH(L.A.slots, k_resid_csr, L.n, L.n, L.A.ptr.p, L.A.col.p, L.A.val.p, w.x, w.b, w.r);
    }
    count_launch();
    KNP_SLOT_DISPATCH(L.R.slots, k_csr4, C.n, C.n, L.R.ptr.p, L.R.col.p, L.R.val.p, w.r, wc.b, 0);
    na_vcycle_rec(D, W, l + 1, nullptr, nullptr, st);
    count_launch();
    KNP_SLOT_DISPATCH(L.P.slots, k_csr4, L.n, L.n, L.P.ptr.p, L.P.col.p, L.P.val.p, wc.x, w.x, 1);
    for (int k = 0; k < D.degree; ++k) na_cheb_step(L, w, cs[k], st);
}

// Lays the work vectors out in the static array; returns the bytes needed (and fills W when
// `base` is not NULL).
template <class T>
static size_t na_layout(AmgDev<T>& D, int64_t n0, unsigned char* base, std::vector<NaWork<T>>& W, double** ones,
                        double** rin, double** zout, T** xfine) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> unsigned char* {
        unsigned char* p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    *ones = reinterpret_cast<double*>(take(4 * n0 * sizeof(double)));
    *rin = reinterpret_cast<double*>(take(4 * n0 * sizeof(double)));
    *zout = reinterpret_cast<double*>(take(4 * n0 * sizeof(double)));
    W.assign(D.L.size(), NaWork<T>{});
    for (size_t l = 0; l < D.L.size(); ++l) {
        size_t b = 4 * (size_t)D.L[l]->n * sizeof(T);
        W[l].x = reinterpret_cast<T*>(take(b));
        W[l].x2 = reinterpret_cast<T*>(take(b));
        W[l].b = reinterpret_cast<T*>(take(b));
        W[l].r = reinterpret_cast<T*>(take(b));
        W[l].d = reinterpret_cast<T*>(take(b));
    }
    *xfine = nullptr;
    return off;
}

template <class T>
static void na_apply(knp_problem* p, AmgDev<T>& D, const double* r_eq42, double* z_eq42) {
    cudaStream_t st = p->stream;
    const int64_t n0 = D.L[0]->n;
    std::vector<NaWork<T>> W;
    double *ones, *rin, *zout;
    T* xf;
    size_t need = na_layout(D, n0, nullptr, W, &ones, &rin, &zout, &xf);
    KNP_REQUIRE(need <= KNP_NOALLOC_SCRATCH_BYTES, KNP_ERR_INVALID_ARG,
                "knp_apply_preconditioner_noalloc needs %zu bytes of scratch for this hierarchy; the static "
                "array holds %zu (use knp_apply_preconditioner)",
                need, KNP_NOALLOC_SCRATCH_BYTES);
    unsigned char* base = noalloc_scratch();
    na_layout(D, n0, base, W, &ones, &rin, &zout, &xf);
    count_launch(3);
    k_fill<<<nblk(4 * n0, 256), 256, 0, st>>>(4 * n0, 1.0, ones);
    k_eq42_to_nodes<<<nblk(n0, 256), 256, 0, st>>>(p->N_i, p->N_e, r_eq42, rin);
    na_vcycle_rec(D, W, 0, rin, ones, st);
    count_launch();
    k_to_double<T><<<nblk(4 * n0, 256), 256, 0, st>>>(4 * n0, W[0].x, zout);
    count_launch();
    k_nodes_to_eq42<<<nblk(n0, 256), 256, 0, st>>>(p->N_i, p->N_e, zout, z_eq42);
    KNP_CUDA(cudaGetLastError());
}

}  // namespace

}  // namespace knp

extern "C" knp_status knp_apply_preconditioner_noalloc(knp_problem* p, const double* r, double* z) {
    using namespace knp;
    return guarded([&] {
        KNP_REQUIRE(p && r && z, KNP_ERR_INVALID_ARG, "NULL argument");
        KNP_REQUIRE(p->amg, KNP_ERR_STATE, "knp_amg_setup has not been called");
        // the static array is looked up on the current device: it must be the problem's
        cudaPointerAttributes at{};
        KNP_CUDA(cudaPointerGetAttributes(&at, p->u.p));
        int dev = -1;
        KNP_CUDA(cudaGetDevice(&dev));
        KNP_REQUIRE(at.device == dev, KNP_ERR_INVALID_ARG,
                    "the current device (%d) is not the problem's device (%d); make it current first", dev,
                    at.device);
        if (p->amg->h32)
            na_apply(p, *static_cast<AmgDev<float>*>(p->amg->h32), r, z);
        else
            na_apply(p, *static_cast<AmgDev<double>*>(p->amg->h64), r, z);
    });
}

