// Internal declarations shared by the translation units of libknp.so.
#pragma once

#include <cstdint>
#include <cstdio>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/knp.h"

namespace knp {

// Thread-local error message behind knp_last_error().
void set_error(const std::string& msg);

struct Error {
    knp_status code;
    std::string msg;
};

#define KNP_FAIL(code, ...)                                   \
    do {                                                      \
        char _buf[512];                                       \
        std::snprintf(_buf, sizeof(_buf), __VA_ARGS__);       \
        throw ::knp::Error{(code), std::string(_buf)};        \
    } while (0)

#define KNP_REQUIRE(cond, code, ...) \
    do {                             \
        if (!(cond)) KNP_FAIL(code, __VA_ARGS__); \
    } while (0)

// Runs f, converting exceptions into a status and a message.
template <class F>
knp_status guarded(F&& f) {
    try {
        f();
        return KNP_OK;
    } catch (const Error& e) {
        set_error(e.msg);
        return e.code;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return KNP_ERR_OOM;
    } catch (const std::exception& e) {
        set_error(e.what());
        return KNP_ERR_INVALID_ARG;
    }
}

}  // namespace knp

// P2 nodes of a mesh (Section 3.3 with p = 2): the vertices, then the edges in lexicographic
// order of their sorted vertex pair; a node belongs to a region when it is a node of one of the
// region's elements, so the vertices and edges of membrane facets are repeated.
struct knp_p2_nodes {
    int64_t n_edges = 0;
    std::vector<int32_t> edges;              // [n_edges*2] sorted vertex pairs, lexicographic
    std::vector<int32_t> elem_nodes;         // [ne*npe]: the element's vertices, then its edges (a<b)
    std::vector<int32_t> facet_nodes;        // [nf*nfn]: the facet's sorted vertices, then its edges
    std::vector<int32_t> nodes_i, nodes_e;   // region node -> global node id (increasing)
    std::vector<int32_t> loc_i, loc_e;       // global node id -> region node, -1 if absent
    std::vector<int32_t> mnodes;             // membrane nodes, increasing
    std::vector<int32_t> node_cell_i;        // cell tag of each intracellular node
    int64_t pin_node = -1;
};

// Topology of a conforming mesh with duplicated membrane nodes (Section 3.3).
struct knp_mesh {
    int32_t dim = 0;
    int64_t nv = 0, ne = 0;
    std::vector<double> coords;       // [nv*dim]
    std::vector<int32_t> elems;       // [ne*(dim+1)]
    std::vector<int32_t> tag;         // [ne]
    std::vector<int32_t> nodes_i, nodes_e;   // region node -> vertex (increasing)
    std::vector<int32_t> loc_i, loc_e;       // vertex -> region node, -1 if absent
    std::vector<int32_t> elems_i, elems_e;   // element ids per region
    std::vector<int32_t> facets;             // [nf*dim] sorted vertex ids, lexicographic
    std::vector<int32_t> facet_elem_i, facet_opp_i, facet_cell;
    std::vector<int32_t> mverts;             // membrane vertices, increasing
    std::vector<int32_t> node_cell_i;        // cell tag of each intracellular node
    int64_t pin_vertex = -1;
    double pin_point[3] = {0.0, 0.0, 0.0};   // the pin goes on the e-vertex nearest to this point
    int32_t n_cells = 0;
    int64_t nf() const { return (int64_t)facet_cell.size(); }
    // P2 nodes, built on first use (knp_mesh_p2_*)
    mutable std::once_flag p2_once;
    mutable std::unique_ptr<knp_p2_nodes> p2;
};

namespace knp {
// The P2 nodes of m, built on first call (thread-safe); throws Error on an invalid mesh.
const knp_p2_nodes& p2_nodes(const knp_mesh& m);
}  // namespace knp
