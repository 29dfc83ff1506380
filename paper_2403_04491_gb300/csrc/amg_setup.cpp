// Host construction of the smoothed-aggregation hierarchy (run once per simulation,
// on P_0, Section 4.2). Steps per level: strength graph, MIS-2 aggregation
// (Luby-style rounds with hashed priorities: roots are a distance-2 independent
// set, aggregates are roots plus their strong neighbours, leftovers join a
// neighbouring aggregate), tentative prolongator from the constant near-null
// vector of each field, one damped-Jacobi smoothing step per field, and the
// Galerkin product R A P per field on a shared pattern. The coarsest operator is
// inverted densely in FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "amg.h"
#include "common.h"

namespace knp {

namespace {

inline uint32_t hash32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

struct Graph {
    std::vector<int64_t> ptr;
    std::vector<int32_t> adj;
};

Graph strength_graph(const HostCsr4& A, const std::vector<double>& s, double theta) {
    const int64_t n = A.n_rows;
    std::vector<double> diag(n, 0.0);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t t = A.ptr[i]; t < A.ptr[i + 1]; ++t)
            if (A.col[t] == i) diag[i] = std::fabs(s[t]);
    Graph G;
    G.ptr.assign(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t t = A.ptr[i]; t < A.ptr[i + 1]; ++t) {
            int64_t j = A.col[t];
            if (j == i) continue;
            if (std::fabs(s[t]) >= theta * std::sqrt(diag[i] * diag[j]) && s[t] != 0.0) G.adj.push_back((int32_t)j);
        }
        G.ptr[i + 1] = (int64_t)G.adj.size();
    }
    return G;
}

// MIS-2 aggregation; returns the aggregate of every node and the aggregate count.
int64_t mis2_aggregate(const Graph& G, int64_t n, int level, std::vector<int32_t>& agg) {
    // state: 0 undecided, 1 root, 2 excluded
    std::vector<uint8_t> state(n, 0);
    std::vector<uint64_t> prio(n);
    for (int64_t i = 0; i < n; ++i)
        prio[i] = ((uint64_t)hash32((uint32_t)i * 2654435761u + (uint32_t)level * 97u) << 32) | (uint64_t)i;
    // isolated nodes become singleton roots right away
    for (int64_t i = 0; i < n; ++i)
        if (G.ptr[i] == G.ptr[i + 1]) state[i] = 1;
    std::vector<uint64_t> m1(n), m2(n);
    for (int round = 0; round < 1000; ++round) {
        bool any = false;
        // max undecided priority over the closed 1-neighbourhood, then over the 2-neighbourhood;
        // decided roots dominate (UINT64_MAX) so their distance-2 neighbours get excluded
        auto key = [&](int64_t i) -> uint64_t { return state[i] == 0 ? prio[i] : (state[i] == 1 ? UINT64_MAX : 0); };
        for (int64_t i = 0; i < n; ++i) {
            uint64_t v = key(i);
            for (int64_t t = G.ptr[i]; t < G.ptr[i + 1]; ++t) v = std::max(v, key(G.adj[t]));
            m1[i] = v;
        }
        for (int64_t i = 0; i < n; ++i) {
            uint64_t v = m1[i];
            for (int64_t t = G.ptr[i]; t < G.ptr[i + 1]; ++t) v = std::max(v, m1[G.adj[t]]);
            m2[i] = v;
        }
        for (int64_t i = 0; i < n; ++i) {
            if (state[i] != 0) continue;
            if (m2[i] == prio[i]) {
                state[i] = 1;
            } else if (m2[i] == UINT64_MAX) {
                state[i] = 2;
            } else {
                any = true;
            }
        }
        if (!any) break;
    }
    // aggregates: roots and their strong neighbours (disjoint because roots are >= 3 apart)
    agg.assign(n, -1);
    int64_t na = 0;
    for (int64_t i = 0; i < n; ++i)
        if (state[i] == 1) agg[i] = (int32_t)na++;
    for (int64_t i = 0; i < n; ++i) {
        if (state[i] != 1) continue;
        for (int64_t t = G.ptr[i]; t < G.ptr[i + 1]; ++t)
            if (agg[G.adj[t]] < 0) agg[G.adj[t]] = agg[i];
    }
    // leftovers join the aggregate of an aggregated strong neighbour (first by id); repeat until stable
    for (int pass = 0; pass < 8; ++pass) {
        bool changed = false;
        std::vector<int32_t> next = agg;
        for (int64_t i = 0; i < n; ++i) {
            if (agg[i] >= 0) continue;
            for (int64_t t = G.ptr[i]; t < G.ptr[i + 1]; ++t)
                if (agg[G.adj[t]] >= 0) {
                    next[i] = agg[G.adj[t]];
                    changed = true;
                    break;
                }
        }
        agg.swap(next);
        if (!changed) break;
    }
    for (int64_t i = 0; i < n; ++i)
        if (agg[i] < 0) agg[i] = (int32_t)na++;
    return na;
}

// Largest eigenvalue of D^-1 A for each field by power iteration.
void spectral_radius(const HostCsr4& A, const std::vector<double>& dinv, double rho[4]) {
    const int64_t n = A.n_rows;
    std::vector<double> x(4 * n), y(4 * n);
    for (int64_t i = 0; i < n; ++i)
        for (int f = 0; f < 4; ++f) x[4 * i + f] = 1.0 + 0.5 * ((hash32((uint32_t)(4 * i + f)) & 1023) / 1023.0);
    double lam[4] = {0, 0, 0, 0};
    for (int it = 0; it < 20; ++it) {
        double nrm[4] = {0, 0, 0, 0};
        for (int64_t i = 0; i < n; ++i) {
            double s[4] = {0, 0, 0, 0};
            for (int64_t t = A.ptr[i]; t < A.ptr[i + 1]; ++t)
                for (int f = 0; f < 4; ++f) s[f] += A.val[4 * t + f] * x[4 * (int64_t)A.col[t] + f];
            for (int f = 0; f < 4; ++f) {
                y[4 * i + f] = dinv[4 * i + f] * s[f];
                nrm[f] += y[4 * i + f] * y[4 * i + f];
            }
        }
        double xn[4] = {0, 0, 0, 0};
        for (int64_t i = 0; i < n; ++i)
            for (int f = 0; f < 4; ++f) xn[f] += x[4 * i + f] * x[4 * i + f];
        for (int f = 0; f < 4; ++f) {
            lam[f] = std::sqrt(nrm[f] / std::max(xn[f], 1e-300));
            double sc = 1.0 / std::sqrt(std::max(nrm[f], 1e-300));
            for (int64_t i = 0; i < n; ++i) x[4 * i + f] = y[4 * i + f] * sc;
        }
    }
    for (int f = 0; f < 4; ++f) rho[f] = lam[f];
}

void transpose(const HostCsr4& P, HostCsr4& R) {
    R.n_rows = P.n_cols;
    R.n_cols = P.n_rows;
    R.ptr.assign(R.n_rows + 1, 0);
    for (int32_t c : P.col) R.ptr[c + 1]++;
    for (int64_t i = 0; i < R.n_rows; ++i) R.ptr[i + 1] += R.ptr[i];
    R.col.resize(P.nnz());
    R.val.resize(4 * P.nnz());
    std::vector<int64_t> fill(R.ptr.begin(), R.ptr.end() - 1);
    for (int64_t i = 0; i < P.n_rows; ++i)
        for (int64_t t = P.ptr[i]; t < P.ptr[i + 1]; ++t) {
            int64_t q = fill[P.col[t]]++;
            R.col[q] = (int32_t)i;
            for (int f = 0; f < 4; ++f) R.val[4 * q + f] = P.val[4 * t + f];
        }
}

// C = A * B (four independent fields), Gustavson with a dense marker.
void spgemm4(const HostCsr4& A, const HostCsr4& B, HostCsr4& C) {
    C.n_rows = A.n_rows;
    C.n_cols = B.n_cols;
    C.ptr.assign(C.n_rows + 1, 0);
    C.col.clear();
    C.val.clear();
    std::vector<int64_t> mark(B.n_cols, -1);
    std::vector<int32_t> cols;
    std::vector<double> acc;
    for (int64_t i = 0; i < A.n_rows; ++i) {
        cols.clear();
        for (int64_t t = A.ptr[i]; t < A.ptr[i + 1]; ++t) {
            int64_t k = A.col[t];
            for (int64_t u = B.ptr[k]; u < B.ptr[k + 1]; ++u) {
                int32_t j = B.col[u];
                if (mark[j] < 0) {
                    mark[j] = (int64_t)cols.size();
                    cols.push_back(j);
                }
            }
        }
        acc.assign(4 * cols.size(), 0.0);
        for (int64_t t = A.ptr[i]; t < A.ptr[i + 1]; ++t) {
            int64_t k = A.col[t];
            for (int64_t u = B.ptr[k]; u < B.ptr[k + 1]; ++u) {
                int64_t q = mark[B.col[u]];
                for (int f = 0; f < 4; ++f) acc[4 * q + f] += A.val[4 * t + f] * B.val[4 * u + f];
            }
        }
        std::vector<int32_t> order(cols.size());
        std::iota(order.begin(), order.end(), 0);
        std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cols[a] < cols[b]; });
        for (int32_t o : order) {
            C.col.push_back(cols[o]);
            for (int f = 0; f < 4; ++f) C.val.push_back(acc[4 * o + f]);
        }
        for (int32_t c : cols) mark[c] = -1;
        C.ptr[i + 1] = (int64_t)C.col.size();
    }
}

void dense_inverse(std::vector<double>& a, int64_t n) {
    // Gauss-Jordan with partial pivoting, in place
    std::vector<double> inv(n * n, 0.0);
    for (int64_t i = 0; i < n; ++i) inv[i * n + i] = 1.0;
    double amax = 0;
    for (double v : a) amax = std::max(amax, std::fabs(v));
    for (int64_t c = 0; c < n; ++c) {
        int64_t p = c;
        for (int64_t r = c + 1; r < n; ++r)
            if (std::fabs(a[r * n + c]) > std::fabs(a[p * n + c])) p = r;
        KNP_REQUIRE(std::fabs(a[p * n + c]) > 1e-300 && std::fabs(a[p * n + c]) > 1e-17 * amax, KNP_ERR_NUMERIC,
                    "coarsest AMG matrix is singular (column %lld)", (long long)c);
        if (p != c) {
            for (int64_t k = 0; k < n; ++k) {
                std::swap(a[p * n + k], a[c * n + k]);
                std::swap(inv[p * n + k], inv[c * n + k]);
            }
        }
        double d = 1.0 / a[c * n + c];
        for (int64_t k = 0; k < n; ++k) {
            a[c * n + k] *= d;
            inv[c * n + k] *= d;
        }
        for (int64_t r = 0; r < n; ++r) {
            if (r == c) continue;
            double fct = a[r * n + c];
            if (fct == 0.0) continue;
            for (int64_t k = 0; k < n; ++k) {
                a[r * n + k] -= fct * a[c * n + k];
                inv[r * n + k] -= fct * inv[c * n + k];
            }
        }
    }
    a.swap(inv);
}

void finish_level(HostLevel& L, double cheb_ratio) {
    const int64_t n = L.A.n_rows;
    L.dinv.assign(4 * n, 0.0);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t t = L.A.ptr[i]; t < L.A.ptr[i + 1]; ++t)
            if (L.A.col[t] == i)
                for (int f = 0; f < 4; ++f) {
                    double d = L.A.val[4 * t + f];
                    if (d == 0.0) {
                        // a field with an empty row (e.g. the pinned potential alone in an aggregate)
                        // is decoupled; give it a unit diagonal
                        bool empty = true;
                        for (int64_t u = L.A.ptr[i]; u < L.A.ptr[i + 1]; ++u) empty &= L.A.val[4 * u + f] == 0.0;
                        if (empty) L.A.val[4 * t + f] = d = 1.0;
                    }
                    KNP_REQUIRE(d > 0.0 && std::isfinite(d), KNP_ERR_NUMERIC,
                                "non-positive diagonal %g in P_0 hierarchy (row %lld, field %d)", d, (long long)i, f);
                    L.dinv[4 * i + f] = 1.0 / d;
                }
    double rho[4];
    spectral_radius(L.A, L.dinv, rho);
    for (int f = 0; f < 4; ++f) {
        L.lmax[f] = 1.1 * rho[f];
        L.lmin[f] = L.lmax[f] / cheb_ratio;
    }
}

}  // namespace

void amg_build(const HostCsr4& A0, const std::vector<double>& strength0, int64_t pin_row, const AmgSetupOpts& o,
               HostHierarchy& H) {
    H.levels.clear();
    H.levels.emplace_back();
    H.levels[0].A = A0;
    std::vector<double> strength = strength0;
    std::vector<double> B(4 * A0.n_rows, 1.0);   // near-null vectors per field
    if (pin_row >= 0) B[4 * pin_row + 3] = 0.0;
    for (int lev = 0;; ++lev) {
        HostLevel& L = H.levels[lev];
        finish_level(L, o.cheb_ratio);
        const int64_t n = L.A.n_rows;
        if (n <= o.coarse_max || lev + 1 >= o.max_levels) break;
        Graph G = strength_graph(L.A, strength, lev == 0 || o.theta_coarse < 0 ? o.theta : o.theta_coarse);
        std::vector<int32_t> agg;
        int64_t na = mis2_aggregate(G, n, lev, agg);
        if (na >= n || na == 0 || (double)na > 0.85 * (double)n) break;
        // smoothed prolongator P_f = (I - omega_f D_f^-1 A_f) P_tent,f; pattern shared by the fields
        double omega[4];
        for (int f = 0; f < 4; ++f) omega[f] = (4.0 / 3.0) / (L.lmax[f] / 1.1);
        HostCsr4& P = L.P;
        P.n_rows = n;
        P.n_cols = na;
        P.ptr.assign(n + 1, 0);
        std::vector<int64_t> mark(na, -1);
        std::vector<int32_t> cols;
        std::vector<double> acc;
        for (int64_t i = 0; i < n; ++i) {
            cols.clear();
            acc.clear();
            auto slot = [&](int32_t c) -> int64_t {
                if (mark[c] < 0) {
                    mark[c] = (int64_t)cols.size();
                    cols.push_back(c);
                    acc.insert(acc.end(), 4, 0.0);
                }
                return mark[c];
            };
            int64_t q0 = slot(agg[i]);
            for (int f = 0; f < 4; ++f) acc[4 * q0 + f] += B[4 * i + f];
            for (int64_t t = L.A.ptr[i]; t < L.A.ptr[i + 1]; ++t) {
                int64_t j = L.A.col[t];
                int64_t q = slot(agg[j]);
                for (int f = 0; f < 4; ++f)
                    acc[4 * q + f] -= omega[f] * L.dinv[4 * i + f] * L.A.val[4 * t + f] * B[4 * j + f];
            }
            std::vector<int32_t> order(cols.size());
            std::iota(order.begin(), order.end(), 0);
            std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cols[a] < cols[b]; });
            double rmax[4] = {0, 0, 0, 0};
            for (size_t q = 0; q < cols.size(); ++q)
                for (int f = 0; f < 4; ++f) rmax[f] = std::max(rmax[f], std::fabs(acc[4 * q + f]));
            for (int32_t oo : order) {
                // keep an entry if it is significant in any field (the pattern is shared)
                bool keep = cols[oo] == agg[i] || o.p_drop <= 0;
                for (int f = 0; f < 4 && !keep; ++f) keep = std::fabs(acc[4 * oo + f]) >= o.p_drop * rmax[f];
                if (!keep) continue;
                P.col.push_back(cols[oo]);
                for (int f = 0; f < 4; ++f) P.val.push_back(acc[4 * oo + f]);
            }
            for (int32_t c : cols) mark[c] = -1;
            P.ptr[i + 1] = (int64_t)P.col.size();
        }
        transpose(P, L.R);
        HostCsr4 AP, Ac;
        spgemm4(L.A, P, AP);
        spgemm4(L.R, AP, Ac);
        // coarse near-null vectors: aggregate restriction of B is 1 wherever the aggregate has a
        // member with B = 1 (the tentative prolongator reproduces the constant)
        std::vector<double> Bc(4 * na, 0.0);
        for (int64_t i = 0; i < n; ++i)
            for (int f = 0; f < 4; ++f) Bc[4 * agg[i] + f] = std::max(Bc[4 * agg[i] + f], B[4 * i + f]);
        B.swap(Bc);
        // strength on coarse levels: the potential field
        strength.assign(Ac.nnz(), 0.0);
        for (int64_t t = 0; t < Ac.nnz(); ++t) strength[t] = Ac.val[4 * t + 3];
        H.levels.emplace_back();
        H.levels[lev + 1].A = std::move(Ac);
    }
    amg_coarse_inverse(H);
}

void amg_host_spgemm(const HostCsr4& A, const HostCsr4& B, HostCsr4& C) { spgemm4(A, B, C); }

void amg_coarse_inverse(HostHierarchy& H) {
    // dense inverse of the coarsest operator, per field
    HostLevel& Lc = H.levels.back();
    const int64_t nc = Lc.A.n_rows;
    KNP_REQUIRE(nc <= 8192, KNP_ERR_INVALID_ARG, "coarsest level has %lld nodes; raise max_levels", (long long)nc);
    H.nc = nc;
    H.coarse_inv.assign(4 * nc * nc, 0.0);
    for (int f = 0; f < 4; ++f) {
        std::vector<double> a(nc * nc, 0.0);
        for (int64_t i = 0; i < nc; ++i)
            for (int64_t t = Lc.A.ptr[i]; t < Lc.A.ptr[i + 1]; ++t) a[i * nc + Lc.A.col[t]] = Lc.A.val[4 * t + f];
        dense_inverse(a, nc);
        std::copy(a.begin(), a.end(), H.coarse_inv.begin() + f * nc * nc);
    }
}

}  // namespace knp
