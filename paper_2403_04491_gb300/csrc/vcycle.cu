// One V-cycle of the smoothed-aggregation hierarchy on P_0, the inexact P_0^{-1} of
// Section 4.2 (the paper uses one BoomerAMG V-cycle; here smoothed aggregation with
// Chebyshev smoothing, all four fields of a node in one pass). Templated on the
// storage/arithmetic type of the hierarchy: double (plain FP64 form) or float (the
// mixed-precision form; the coarsest dense solve is FP64 in both).
#include <cmath>

#include "amg.h"
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
    float dummy;
    double c1[4], c2[4];
};

// acc = (A x)_row over the sliced-ELL row
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

// first Chebyshev step from x = 0: d = c2 D^-1 b, x = d. On the finest level b = s .* v (double input).
template <class T>
__global__ void k_cheb_first(int64_t n, const double* __restrict__ v, const double* __restrict__ s, T* __restrict__ b,
                             const T* __restrict__ dinv, Coef4 c, T* __restrict__ x, T* __restrict__ d) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    V4<T> bb;
    if (v) {
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

// Chebyshev step: r = b - A x_in; d = c1 d + c2 D^-1 r; x_out = x_in + d
template <class T>
__global__ void __launch_bounds__(128) k_cheb_step(int64_t n, const int64_t* __restrict__ sp,
                                                   const int32_t* __restrict__ col, const T* __restrict__ val,
                                                   const T* __restrict__ x_in, const T* __restrict__ b,
                                                   const T* __restrict__ dinv, Coef4 c, T* __restrict__ d,
                                                   T* __restrict__ x_out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    T acc[4];
    sell_row<T>(i, sp, col, val, x_in, acc);
    V4<T> bb = V4<T>::load(b + 4 * i), di = V4<T>::load(dinv + 4 * i), dd = V4<T>::load(d + 4 * i),
          xx = V4<T>::load(x_in + 4 * i);
    for (int f = 0; f < 4; ++f) {
        dd.v[f] = (T)c.c1[f] * dd.v[f] + (T)c.c2[f] * di.v[f] * (bb.v[f] - acc[f]);
        xx.v[f] += dd.v[f];
    }
    dd.store(d + 4 * i);
    xx.store(x_out + 4 * i);
}

template <class T>
__global__ void __launch_bounds__(128) k_residual(int64_t n, const int64_t* __restrict__ sp,
                                                  const int32_t* __restrict__ col, const T* __restrict__ val,
                                                  const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ r) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    T acc[4];
    sell_row<T>(i, sp, col, val, x, acc);
    V4<T> bb = V4<T>::load(b + 4 * i);
    for (int f = 0; f < 4; ++f) bb.v[f] -= acc[f];
    bb.store(r + 4 * i);
}

// y[i] (+)= sum_t M(i, col[t]) x[col[t]] for a CSR with four values per entry
template <class T>
__global__ void k_csr4(int64_t n, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                       const T* __restrict__ val, const T* __restrict__ x, T* __restrict__ y, int accumulate) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    T acc[4] = {0, 0, 0, 0};
    for (int64_t t = ptr[i]; t < ptr[i + 1]; ++t) {
        V4<T> a = V4<T>::load(val + 4 * t);
        V4<T> xv = V4<T>::load(x + 4 * (int64_t)col[t]);
        for (int f = 0; f < 4; ++f) acc[f] += a.v[f] * xv.v[f];
    }
    V4<T> yy;
    if (accumulate) {
        yy = V4<T>::load(y + 4 * i);
        for (int f = 0; f < 4; ++f) yy.v[f] += acc[f];
    } else {
        for (int f = 0; f < 4; ++f) yy.v[f] = acc[f];
    }
    yy.store(y + 4 * i);
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

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <class T>
std::vector<T> cast_vec(const std::vector<double>& v) {
    return std::vector<T>(v.begin(), v.end());
}

}  // namespace

template <class T>
struct DevLevel {
    int64_t n = 0, nnz_pad = 0;
    DArray<int64_t> sp;
    DArray<int32_t> col;
    DArray<T> val;
    DArray<T> dinv;
    double lmax[4], lmin[4];
    DArray<int64_t> Pptr, Rptr;
    DArray<int32_t> Pcol, Rcol;
    DArray<T> Pval, Rval;
    DArray<T> x, x2, b, r, d;
    int64_t nnz_csr = 0;
};

template <class T>
struct AmgDev {
    std::vector<std::unique_ptr<DevLevel<T>>> L;
    DArray<double> cinv;
    int64_t nc = 0;
    int degree = 2;
    std::vector<std::vector<Coef4>> coef;   // per level: coefficients of each Chebyshev step
};

AmgHierarchy::~AmgHierarchy() {
    delete static_cast<AmgDev<double>*>(h64);
    delete static_cast<AmgDev<float>*>(h32);
}

template <class T>
static void upload_hierarchy(AmgDev<T>& D, const HostHierarchy& H, int degree, cudaStream_t st) {
    D.degree = degree;
    for (const HostLevel& HL : H.levels) {
        auto L = std::make_unique<DevLevel<T>>();
        const int64_t n = HL.A.n_rows;
        L->n = n;
        // CSR -> sliced ELL
        int64_t ns = (n + SELL_C - 1) / SELL_C;
        std::vector<int64_t> sp(ns + 1, 0);
        for (int64_t s = 0; s < ns; ++s) {
            int64_t w = 0;
            for (int64_t r = s * SELL_C; r < std::min(n, (s + 1) * SELL_C); ++r) w = std::max(w, HL.A.ptr[r + 1] - HL.A.ptr[r]);
            sp[s + 1] = sp[s] + w * SELL_C;
        }
        std::vector<int32_t> col(sp[ns]);
        std::vector<T> val(4 * sp[ns], T(0));
        for (int64_t s = 0; s < ns; ++s) {
            int64_t w = (sp[s + 1] - sp[s]) / SELL_C;
            for (int64_t lane = 0; lane < SELL_C; ++lane) {
                int64_t r = s * SELL_C + lane;
                int64_t len = r < n ? HL.A.ptr[r + 1] - HL.A.ptr[r] : 0;
                for (int64_t k = 0; k < w; ++k) {
                    int64_t pos = sp[s] + k * SELL_C + lane;
                    if (k < len) {
                        int64_t t = HL.A.ptr[r] + k;
                        col[pos] = HL.A.col[t];
                        for (int f = 0; f < 4; ++f) val[4 * pos + f] = (T)HL.A.val[4 * t + f];
                    } else {
                        col[pos] = (int32_t)std::min<int64_t>(r, n - 1);
                    }
                }
            }
        }
        L->nnz_pad = sp[ns];
        L->nnz_csr = HL.A.nnz();
        L->sp.upload(sp, st);
        L->col.upload(col, st);
        L->val.upload(val, st);
        L->dinv.upload(cast_vec<T>(HL.dinv), st);
        for (int f = 0; f < 4; ++f) {
            L->lmax[f] = HL.lmax[f];
            L->lmin[f] = HL.lmin[f];
        }
        if (HL.P.n_rows) {
            L->Pptr.upload(HL.P.ptr, st);
            L->Pcol.upload(HL.P.col, st);
            L->Pval.upload(cast_vec<T>(HL.P.val), st);
            L->Rptr.upload(HL.R.ptr, st);
            L->Rcol.upload(HL.R.col, st);
            L->Rval.upload(cast_vec<T>(HL.R.val), st);
        }
        for (DArray<T>* v : {&L->x, &L->x2, &L->b, &L->r, &L->d}) {
            v->alloc(4 * n);
            v->zero(st);
        }
        // Chebyshev coefficients
        std::vector<Coef4> cs(std::max(degree, 1));
        double rho0[4];
        for (int f = 0; f < 4; ++f) {
            double th = 0.5 * (L->lmax[f] + L->lmin[f]), de = 0.5 * (L->lmax[f] - L->lmin[f]);
            double sigma = th / de;
            rho0[f] = 1.0 / sigma;
            cs[0].c1[f] = 0.0;
            cs[0].c2[f] = 1.0 / th;
            for (int k = 1; k < degree; ++k) {
                double rho1 = 1.0 / (2.0 * sigma - rho0[f]);
                cs[k].c1[f] = rho1 * rho0[f];
                cs[k].c2[f] = 2.0 * rho1 / de;
                rho0[f] = rho1;
            }
        }
        D.coef.push_back(cs);
        D.L.push_back(std::move(L));
    }
    D.nc = H.nc;
    D.cinv.upload(H.coarse_inv, st);
}

void amg_upload(knp_problem* p, const HostHierarchy& H, int precision, int degree) {
    delete p->amg;
    p->amg = new AmgHierarchy();
    p->amg->precision = precision;
    p->amg->levels = (int)H.levels.size();
    for (const HostLevel& L : H.levels) {
        p->amg->nodes.push_back(L.A.n_rows);
        p->amg->nnz.push_back(L.A.nnz());
    }
    if (precision == KNP_PREC_FP32) {
        auto* D = new AmgDev<float>();
        p->amg->h32 = D;
        upload_hierarchy(*D, H, degree, p->stream);
    } else {
        auto* D = new AmgDev<double>();
        p->amg->h64 = D;
        upload_hierarchy(*D, H, degree, p->stream);
    }
    KNP_CUDA(cudaStreamSynchronize(p->stream));
}

template <class T>
static void smooth(DevLevel<T>& L, const std::vector<Coef4>& cs, int degree, bool zero_start, const double* v,
                   const double* s, cudaStream_t st) {
    const unsigned nb = nblk(L.n, 128);
    int k0 = 0;
    if (zero_start) {
        k_cheb_first<T><<<nblk(L.n, 256), 256, 0, st>>>(L.n, v, s, L.b.p, L.dinv.p, cs[0], L.x.p, L.d.p);
        k0 = 1;
    }
    for (int k = k0; k < degree; ++k) {
        k_cheb_step<T><<<nb, 128, 0, st>>>(L.n, L.sp.p, L.col.p, L.val.p, L.x.p, L.b.p, L.dinv.p, cs[k], L.d.p,
                                           L.x2.p);
        std::swap(L.x.p, L.x2.p);
    }
}

template <class T>
static void vcycle_rec(AmgDev<T>& D, int l, const double* v, const double* s, cudaStream_t st) {
    DevLevel<T>& L = *D.L[l];
    const int last = (int)D.L.size() - 1;
    if (l == last) {
        if (v) {
            // single-level hierarchy: build b from the scaled input first
            Coef4 c0{};
            k_cheb_first<T><<<nblk(L.n, 256), 256, 0, st>>>(L.n, v, s, L.b.p, L.dinv.p, c0, L.x.p, L.d.p);
        }
        k_coarse<T><<<nblk(4 * D.nc * 32, 256), 256, 0, st>>>(D.nc, D.cinv.p, L.b.p, L.x.p);
        return;
    }
    DevLevel<T>& C = *D.L[l + 1];
    smooth(L, D.coef[l], D.degree, true, v, s, st);
    k_residual<T><<<nblk(L.n, 128), 128, 0, st>>>(L.n, L.sp.p, L.col.p, L.val.p, L.x.p, L.b.p, L.r.p);
    k_csr4<T><<<nblk(C.n, 128), 128, 0, st>>>(C.n, L.Rptr.p, L.Rcol.p, L.Rval.p, L.r.p, C.b.p, 0);
    vcycle_rec(D, l + 1, nullptr, nullptr, st);
    k_csr4<T><<<nblk(L.n, 128), 128, 0, st>>>(L.n, L.Pptr.p, L.Pcol.p, L.Pval.p, C.x.p, L.x.p, 1);
    smooth(L, D.coef[l], D.degree, false, nullptr, nullptr, st);
}

// z = V-cycle(P_0)(s .* v); v, s, z are [n][4] doubles on the device.
void vcycle_apply(knp_problem* p, const double* v, const double* s, double* z) {
    KNP_REQUIRE(p->amg, KNP_ERR_STATE, "knp_amg_setup has not been called");
    cudaStream_t st = p->stream;
    if (p->amg->h32) {
        auto& D = *static_cast<AmgDev<float>*>(p->amg->h32);
        vcycle_rec(D, 0, v, s, st);
        k_to_double<float><<<nblk(4 * D.L[0]->n, 256), 256, 0, st>>>(4 * D.L[0]->n, D.L[0]->x.p, z);
    } else {
        auto& D = *static_cast<AmgDev<double>*>(p->amg->h64);
        vcycle_rec(D, 0, v, s, st);
        KNP_CUDA(cudaMemcpyAsync(z, D.L[0]->x.p, 4 * D.L[0]->n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    KNP_CUDA(cudaGetLastError());
}

}  // namespace knp
