// Mesh intake: membrane facets, duplicated membrane nodes, region numbering, pin
// (Section 3.3 spatial discretisation; Remark 4.1 point pin).
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <numeric>
#include <thread>
#include <vector>

#include "common.h"

namespace knp {

thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

namespace {

struct FacetKey {
    int32_t v[3];
    int32_t elem;
    int32_t opp;
};

double simplex_det(const double* x, int dim, const int32_t* el) {
    if (dim == 2) {
        const double* a = x + 2 * (int64_t)el[0];
        const double* b = x + 2 * (int64_t)el[1];
        const double* c = x + 2 * (int64_t)el[2];
        return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]);
    }
    const double* a = x + 3 * (int64_t)el[0];
    double e[3][3];
    for (int j = 0; j < 3; ++j)
        for (int d = 0; d < 3; ++d) e[j][d] = x[3 * (int64_t)el[j + 1] + d] - a[d];
    return e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) - e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
           e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
}

// Runs f(t, begin, end) on n_threads contiguous slices of [0, n).
template <class F>
void parallel_slices(int n_threads, int64_t n, F f) {
    if (n_threads <= 1) {
        f(0, (int64_t)0, n);
        return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < n_threads; ++t)
        th.emplace_back([&, t] { f(t, n * t / n_threads, n * (t + 1) / n_threads); });
    for (auto& x : th) x.join();
}

int topology_threads(int64_t work) {
    if (work < (int64_t)1 << 20) return 1;
    const unsigned hw = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(hw ? hw : 1u, 64u));
}

}  // namespace

void build_topology(knp_mesh& m) {
    const int dim = m.dim;
    const int nvpe = dim + 1;
    const int64_t ne = m.ne, nv = m.nv;
    // element checks
    double max_abs = 0.0;
    for (int64_t i = 0; i < nv * dim; ++i) max_abs = std::max(max_abs, std::fabs(m.coords[i]));
    const int nthr = topology_threads(ne * nvpe);
    auto check_element = [&](int64_t e) {
        const int32_t* el = &m.elems[e * nvpe];
        for (int j = 0; j < nvpe; ++j)
            KNP_REQUIRE(el[j] >= 0 && el[j] < nv, KNP_ERR_INVALID_ARG, "element %lld has vertex id %d out of range",
                        (long long)e, el[j]);
        KNP_REQUIRE(m.tag[e] >= 0, KNP_ERR_INVALID_ARG, "negative tag on element %lld", (long long)e);
        double det = simplex_det(m.coords.data(), dim, el);
        KNP_REQUIRE(std::fabs(det) > 1e-14 * std::pow(max_abs, dim) && std::isfinite(det), KNP_ERR_INVALID_MESH,
                    "element %lld is degenerate", (long long)e);
    };
    {
        // the first failing element of each slice, found in parallel without throwing; the
        // lowest one is then checked again serially, which raises its error
        std::vector<int64_t> bad(nthr, ne);
        parallel_slices(nthr, ne, [&](int t, int64_t a, int64_t b) {
            for (int64_t e = a; e < b; ++e) {
                const int32_t* el = &m.elems[e * nvpe];
                bool ok = m.tag[e] >= 0;
                for (int j = 0; j < nvpe; ++j) ok &= el[j] >= 0 && el[j] < nv;
                if (ok) {
                    const double det = simplex_det(m.coords.data(), dim, el);
                    ok = std::fabs(det) > 1e-14 * std::pow(max_abs, dim) && std::isfinite(det);
                }
                if (!ok) {
                    bad[t] = e;
                    break;
                }
            }
        });
        const int64_t first = *std::min_element(bad.begin(), bad.end());
        if (first < ne) check_element(first);
    }
    // facets: slot s of element e is the facet opposite local vertex s. The keys are bucketed by
    // their smallest vertex id (equal facets share it), each bucket is sorted and scanned on its
    // own, and the buckets are taken in vertex order, which is the order of one global sort.
    auto make_key = [&](int64_t e, int s) {
        const int32_t* el = &m.elems[e * nvpe];
        FacetKey k{{-1, -1, -1}, (int32_t)e, s};
        int c = 0;
        for (int j = 0; j < nvpe; ++j)
            if (j != s) k.v[c++] = el[j];
        std::sort(k.v, k.v + dim);
        return k;
    };
    const int nb = nthr > 1 ? 64 * nthr : 1;
    auto bucket_of = [&](int32_t v0) { return (int)((int64_t)v0 * nb / nv); };
    std::vector<int64_t> cnt((size_t)nthr * nb, 0);
    parallel_slices(nthr, ne, [&](int t, int64_t a, int64_t b) {
        int64_t* c = &cnt[(size_t)t * nb];
        for (int64_t e = a; e < b; ++e)
            for (int s = 0; s < nvpe; ++s) c[bucket_of(make_key(e, s).v[0])]++;
    });
    std::vector<int64_t> bstart(nb + 1, 0), pos((size_t)nthr * nb);
    for (int b = 0; b < nb; ++b) {
        int64_t acc = bstart[b];
        for (int t = 0; t < nthr; ++t) {
            pos[(size_t)t * nb + b] = acc;
            acc += cnt[(size_t)t * nb + b];
        }
        bstart[b + 1] = acc;
    }
    std::vector<FacetKey> keys((size_t)ne * nvpe);
    parallel_slices(nthr, ne, [&](int t, int64_t a, int64_t b) {
        int64_t* p = &pos[(size_t)t * nb];
        for (int64_t e = a; e < b; ++e)
            for (int s = 0; s < nvpe; ++s) {
                FacetKey k = make_key(e, s);
                keys[p[bucket_of(k.v[0])]++] = k;
            }
    });
    auto less = [dim](const FacetKey& a, const FacetKey& b) {
        for (int d = 0; d < dim; ++d)
            if (a.v[d] != b.v[d]) return a.v[d] < b.v[d];
        return a.elem < b.elem;
    };
    auto same = [dim](const FacetKey& a, const FacetKey& b) {
        for (int d = 0; d < dim; ++d)
            if (a.v[d] != b.v[d]) return false;
        return true;
    };
    // per bucket: sort, then pair the equal keys; an error is recorded (not thrown) as the
    // position of the first offending key, and raised below in bucket order
    std::vector<std::vector<FacetKey>> mem_b(nb);
    std::vector<int64_t> err_at(nb, -1);
    std::vector<int> err_kind(nb, 0);
    std::atomic<int> next{0};
    parallel_slices(nthr, nthr, [&](int, int64_t, int64_t) {
        for (int b = next++; b < nb; b = next++) {
            const int64_t lo = bstart[b], hi = bstart[b + 1];
            std::sort(keys.begin() + lo, keys.begin() + hi, less);
            for (int64_t i = lo; i + 1 < hi; ++i) {
                if (!same(keys[i], keys[i + 1])) continue;
                if (i + 2 < hi && same(keys[i], keys[i + 2])) {
                    err_at[b] = i;
                    err_kind[b] = 1;
                    break;
                }
                const int32_t ta = m.tag[keys[i].elem], tb = m.tag[keys[i + 1].elem];
                if (ta != tb) {
                    if (ta != 0 && tb != 0) {
                        err_at[b] = i;
                        err_kind[b] = 2;
                        break;
                    }
                    mem_b[b].push_back(ta > 0 ? keys[i] : keys[i + 1]);
                }
                ++i;
            }
        }
    });
    for (int b = 0; b < nb; ++b) {
        if (err_at[b] < 0) continue;
        const FacetKey& k = keys[err_at[b]];
        KNP_REQUIRE(err_kind[b] != 1, KNP_ERR_INVALID_MESH, "a facet is shared by more than two elements");
        KNP_FAIL(KNP_ERR_INVALID_MESH, "cells %d and %d share a facet", m.tag[k.elem], m.tag[keys[err_at[b] + 1].elem]);
    }
    std::vector<FacetKey> mem;  // intracellular side of each membrane facet
    for (int b = 0; b < nb; ++b) mem.insert(mem.end(), mem_b[b].begin(), mem_b[b].end());
    // keys are sorted lexicographically, so mem is in facet order already
    const int64_t nf = (int64_t)mem.size();
    m.facets.resize(nf * dim);
    m.facet_elem_i.resize(nf);
    m.facet_opp_i.resize(nf);
    m.facet_cell.resize(nf);
    for (int64_t f = 0; f < nf; ++f) {
        for (int d = 0; d < dim; ++d) m.facets[f * dim + d] = mem[f].v[d];
        m.facet_elem_i[f] = mem[f].elem;
        m.facet_opp_i[f] = mem[f].opp;
        m.facet_cell[f] = m.tag[mem[f].elem];
    }
    std::vector<char> in_i(nv, 0), in_e(nv, 0), on_g(nv, 0);
    std::vector<int32_t> vcell(nv, 0);
    m.n_cells = 0;
    for (int64_t e = 0; e < ne; ++e) {
        const int32_t* el = &m.elems[e * nvpe];
        int32_t t = m.tag[e];
        m.n_cells = std::max(m.n_cells, t);
        if (t > 0) {
            m.elems_i.push_back((int32_t)e);
            for (int j = 0; j < nvpe; ++j) {
                int32_t v = el[j];
                KNP_REQUIRE(vcell[v] == 0 || vcell[v] == t, KNP_ERR_INVALID_MESH,
                            "vertex %d belongs to cells %d and %d", v, vcell[v], t);
                vcell[v] = t;
                in_i[v] = 1;
            }
        } else {
            m.elems_e.push_back((int32_t)e);
            for (int j = 0; j < nvpe; ++j) in_e[el[j]] = 1;
        }
    }
    for (int64_t i = 0; i < nf * dim; ++i) on_g[m.facets[i]] = 1;
    for (int64_t v = 0; v < nv; ++v)
        KNP_REQUIRE((in_i[v] && in_e[v]) == (bool)on_g[v], KNP_ERR_INVALID_MESH,
                    "vertex %lld touches both regions outside the membrane facets", (long long)v);
    std::vector<char> cell_has_facet(m.n_cells + 1, 0);
    for (int64_t f = 0; f < nf; ++f) cell_has_facet[m.facet_cell[f]] = 1;
    std::vector<char> cell_present(m.n_cells + 1, 0);
    for (int32_t e : m.elems_i) cell_present[m.tag[e]] = 1;
    for (int c = 1; c <= m.n_cells; ++c)
        KNP_REQUIRE(!cell_present[c] || cell_has_facet[c], KNP_ERR_INVALID_MESH, "cell %d has no membrane facet", c);
    KNP_REQUIRE(!m.elems_e.empty(), KNP_ERR_INVALID_MESH, "no extracellular elements");
    m.loc_i.assign(nv, -1);
    m.loc_e.assign(nv, -1);
    for (int64_t v = 0; v < nv; ++v) {
        if (in_i[v]) {
            m.loc_i[v] = (int32_t)m.nodes_i.size();
            m.nodes_i.push_back((int32_t)v);
            m.node_cell_i.push_back(vcell[v]);
        }
        if (in_e[v]) {
            m.loc_e[v] = (int32_t)m.nodes_e.size();
            m.nodes_e.push_back((int32_t)v);
        }
        if (on_g[v]) m.mverts.push_back((int32_t)v);
    }
    // pin: extracellular vertex nearest to the pin point (the origin by default), ties by lowest id
    double best = INFINITY;
    for (int32_t v : m.nodes_e) {
        double d2 = 0;
        for (int d = 0; d < dim; ++d) {
            const double x = m.coords[(int64_t)v * dim + d] - m.pin_point[d];
            d2 += x * x;
        }
        if (d2 < best) {
            best = d2;
            m.pin_vertex = v;
        }
    }
}

namespace {

// Local edges (a, b), a < b, of an m-simplex in lexicographic order.
int local_pairs(int m, int out[6][2]) {
    int k = 0;
    for (int a = 0; a <= m; ++a)
        for (int b = a + 1; b <= m; ++b) {
            out[k][0] = a;
            out[k][1] = b;
            ++k;
        }
    return k;
}

void build_p2(const knp_mesh& m, knp_p2_nodes& t) {
    const int dim = m.dim, nvpe = dim + 1;
    const int64_t nv = m.nv, ne = m.ne, nf = m.nf();
    int pe[6][2], pf[6][2];
    const int npe_edges = local_pairs(dim, pe);
    const int nf_edges = local_pairs(dim - 1, pf);
    auto key = [nv](int32_t a, int32_t b) {
        return a < b ? (int64_t)a * nv + b : (int64_t)b * nv + a;
    };
    // edges: the sorted distinct vertex pairs of all element edges
    std::vector<int64_t> keys((size_t)ne * npe_edges);
    parallel_slices(topology_threads(ne * npe_edges), ne, [&](int, int64_t b, int64_t e) {
        for (int64_t el = b; el < e; ++el) {
            const int32_t* v = &m.elems[el * nvpe];
            for (int k = 0; k < npe_edges; ++k) keys[el * npe_edges + k] = key(v[pe[k][0]], v[pe[k][1]]);
        }
    });
    std::vector<int64_t> ek(keys);
    std::sort(ek.begin(), ek.end());
    ek.erase(std::unique(ek.begin(), ek.end()), ek.end());
    t.n_edges = (int64_t)ek.size();
    const int64_t nn = nv + t.n_edges;
    KNP_REQUIRE(nn < INT32_MAX, KNP_ERR_INVALID_ARG, "too many P2 nodes for 32-bit ids (%lld)", (long long)nn);
    t.edges.resize(2 * t.n_edges);
    for (int64_t i = 0; i < t.n_edges; ++i) {
        t.edges[2 * i] = (int32_t)(ek[i] / nv);
        t.edges[2 * i + 1] = (int32_t)(ek[i] % nv);
    }
    // node id of the edge with key k, -1 if no element has it (never throws: runs on worker threads)
    auto edge_id = [&](int64_t k) -> int32_t {
        auto it = std::lower_bound(ek.begin(), ek.end(), k);
        return (it != ek.end() && *it == k) ? (int32_t)(nv + (it - ek.begin())) : -1;
    };
    const int npe = nvpe + npe_edges;
    t.elem_nodes.resize((size_t)ne * npe);
    parallel_slices(topology_threads(ne * npe_edges), ne, [&](int, int64_t b, int64_t e) {
        for (int64_t el = b; el < e; ++el) {
            for (int j = 0; j < nvpe; ++j) t.elem_nodes[el * npe + j] = m.elems[el * nvpe + j];
            for (int k = 0; k < npe_edges; ++k) t.elem_nodes[el * npe + nvpe + k] = edge_id(keys[el * npe_edges + k]);
        }
    });
    keys.clear();
    keys.shrink_to_fit();
    const int nfn = dim + nf_edges;
    t.facet_nodes.resize((size_t)nf * nfn);
    for (int64_t f = 0; f < nf; ++f) {
        const int32_t* v = &m.facets[f * dim];
        for (int j = 0; j < dim; ++j) t.facet_nodes[f * nfn + j] = v[j];
        for (int k = 0; k < nf_edges; ++k) {
            const int32_t x = edge_id(key(v[pf[k][0]], v[pf[k][1]]));
            KNP_REQUIRE(x >= 0, KNP_ERR_INVALID_MESH, "an edge of membrane facet %lld is not an element edge", (long long)f);
            t.facet_nodes[f * nfn + dim + k] = x;
        }
    }
    // region membership, membrane nodes and the cell of each intracellular node
    std::vector<char> in_i(nn, 0), in_e(nn, 0), on_g(nn, 0);
    std::vector<int32_t> cell(nn, 0);
    for (int32_t el : m.elems_i)
        for (int j = 0; j < npe; ++j) {
            const int32_t x = t.elem_nodes[(int64_t)el * npe + j];
            in_i[x] = 1;
            cell[x] = m.tag[el];
        }
    for (int32_t el : m.elems_e)
        for (int j = 0; j < npe; ++j) in_e[t.elem_nodes[(int64_t)el * npe + j]] = 1;
    for (int32_t x : t.facet_nodes) on_g[x] = 1;
    t.loc_i.assign(nn, -1);
    t.loc_e.assign(nn, -1);
    for (int64_t x = 0; x < nn; ++x) {
        KNP_REQUIRE((in_i[x] && in_e[x]) == (bool)on_g[x], KNP_ERR_INVALID_MESH,
                    "regions share an edge outside the membrane facets (P2 node %lld)", (long long)x);
        if (in_i[x]) {
            t.loc_i[x] = (int32_t)t.nodes_i.size();
            t.nodes_i.push_back((int32_t)x);
            t.node_cell_i.push_back(cell[x]);
        }
        if (in_e[x]) {
            t.loc_e[x] = (int32_t)t.nodes_e.size();
            t.nodes_e.push_back((int32_t)x);
        }
        if (on_g[x]) t.mnodes.push_back((int32_t)x);
    }
    // pin: extracellular node (vertex or edge midpoint) nearest to the pin point, ties by lowest id
    double best = INFINITY;
    for (int32_t x : t.nodes_e) {
        double d2 = 0;
        for (int d = 0; d < dim; ++d) {
            double c;
            if (x < nv) {
                c = m.coords[(int64_t)x * dim + d];
            } else {
                const int64_t i = x - nv;
                c = 0.5 * (m.coords[(int64_t)t.edges[2 * i] * dim + d] + m.coords[(int64_t)t.edges[2 * i + 1] * dim + d]);
            }
            const double y = c - m.pin_point[d];
            d2 += y * y;
        }
        if (d2 < best) {
            best = d2;
            t.pin_node = x;
        }
    }
}

}  // namespace

const knp_p2_nodes& p2_nodes(const knp_mesh& m) {
    std::call_once(m.p2_once, [&] {
        auto t = std::make_unique<knp_p2_nodes>();
        build_p2(m, *t);
        m.p2 = std::move(t);
    });
    return *m.p2;
}

}  // namespace knp

using namespace knp;

extern "C" {

const char* knp_last_error(void) { return g_last_error.c_str(); }

knp_status knp_mesh_create(const knp_mesh_desc* d, knp_mesh** out) {
    return guarded([&] {
        KNP_REQUIRE(d && out, KNP_ERR_INVALID_ARG, "NULL argument");
        *out = nullptr;
        KNP_REQUIRE(d->dim == 2 || d->dim == 3, KNP_ERR_INVALID_ARG, "dim must be 2 or 3 (got %d)", d->dim);
        KNP_REQUIRE(d->n_vertices > 0 && d->n_elems > 0 && d->coords && d->elems && d->elem_tag, KNP_ERR_INVALID_ARG,
                    "empty mesh or NULL array");
        KNP_REQUIRE(d->n_vertices < INT32_MAX && d->n_elems * (d->dim + 1) < INT32_MAX, KNP_ERR_INVALID_ARG,
                    "mesh too large for 32-bit ids");
        auto m = new knp_mesh();
        try {
            m->dim = d->dim;
            m->nv = d->n_vertices;
            m->ne = d->n_elems;
            m->coords.assign(d->coords, d->coords + d->n_vertices * d->dim);
            m->elems.assign(d->elems, d->elems + d->n_elems * (d->dim + 1));
            m->tag.assign(d->elem_tag, d->elem_tag + d->n_elems);
            if (d->pin_point)
                for (int k = 0; k < d->dim; ++k) {
                    KNP_REQUIRE(std::isfinite(d->pin_point[k]), KNP_ERR_INVALID_ARG, "pin point is not finite");
                    m->pin_point[k] = d->pin_point[k];
                }
            build_topology(*m);
        } catch (...) {
            delete m;
            throw;
        }
        *out = m;
    });
}

knp_status knp_mesh_get_info(const knp_mesh* m, knp_mesh_info* info) {
    return guarded([&] {
        KNP_REQUIRE(m && info, KNP_ERR_INVALID_ARG, "NULL argument");
        info->dim = m->dim;
        info->n_vertices = m->nv;
        info->n_elems = m->ne;
        info->N_i = (int64_t)m->nodes_i.size();
        info->N_e = (int64_t)m->nodes_e.size();
        info->n_facets = m->nf();
        info->n_membrane_vertices = (int64_t)m->mverts.size();
        info->n_cells = m->n_cells;
        info->pin_vertex = m->pin_vertex;
        info->n_dof = (info->N_i + info->N_e) * 4;
    });
}

knp_status knp_mesh_nodes(const knp_mesh* m, int32_t* nodes_i, int32_t* nodes_e) {
    return guarded([&] {
        KNP_REQUIRE(m, KNP_ERR_INVALID_ARG, "NULL mesh");
        if (nodes_i) std::copy(m->nodes_i.begin(), m->nodes_i.end(), nodes_i);
        if (nodes_e) std::copy(m->nodes_e.begin(), m->nodes_e.end(), nodes_e);
    });
}

knp_status knp_mesh_facets(const knp_mesh* m, int32_t* vertices, int32_t* elem_i, int32_t* opp_i, int32_t* cell) {
    return guarded([&] {
        KNP_REQUIRE(m, KNP_ERR_INVALID_ARG, "NULL mesh");
        if (vertices) std::copy(m->facets.begin(), m->facets.end(), vertices);
        if (elem_i) std::copy(m->facet_elem_i.begin(), m->facet_elem_i.end(), elem_i);
        if (opp_i) std::copy(m->facet_opp_i.begin(), m->facet_opp_i.end(), opp_i);
        if (cell) std::copy(m->facet_cell.begin(), m->facet_cell.end(), cell);
    });
}

knp_status knp_mesh_p2_get_info(const knp_mesh* m, knp_p2_info* info) {
    return guarded([&] {
        KNP_REQUIRE(m && info, KNP_ERR_INVALID_ARG, "NULL argument");
        const knp_p2_nodes& t = p2_nodes(*m);
        info->n_edges = t.n_edges;
        info->n_nodes = m->nv + t.n_edges;
        info->N_i = (int64_t)t.nodes_i.size();
        info->N_e = (int64_t)t.nodes_e.size();
        info->n_membrane_nodes = (int64_t)t.mnodes.size();
        info->pin_node = t.pin_node;
        info->n_dof = (info->N_i + info->N_e) * 4;
    });
}

knp_status knp_mesh_p2_tables(const knp_mesh* m, int32_t* edges, int32_t* elem_nodes, int32_t* facet_nodes,
                              int32_t* nodes_i, int32_t* nodes_e, int32_t* membrane_nodes, int32_t* node_cell_i) {
    return guarded([&] {
        KNP_REQUIRE(m, KNP_ERR_INVALID_ARG, "NULL mesh");
        const knp_p2_nodes& t = p2_nodes(*m);
        if (edges) std::copy(t.edges.begin(), t.edges.end(), edges);
        if (elem_nodes) std::copy(t.elem_nodes.begin(), t.elem_nodes.end(), elem_nodes);
        if (facet_nodes) std::copy(t.facet_nodes.begin(), t.facet_nodes.end(), facet_nodes);
        if (nodes_i) std::copy(t.nodes_i.begin(), t.nodes_i.end(), nodes_i);
        if (nodes_e) std::copy(t.nodes_e.begin(), t.nodes_e.end(), nodes_e);
        if (membrane_nodes) std::copy(t.mnodes.begin(), t.mnodes.end(), membrane_nodes);
        if (node_cell_i) std::copy(t.node_cell_i.begin(), t.node_cell_i.end(), node_cell_i);
    });
}

void knp_mesh_destroy(knp_mesh* m) { delete m; }

}  // extern "C"
