/* Plain C99 caller of the library's mesh intake (include/knp.h): reads a mesh from a binary
 * file (int32 dim; int64 n_vertices, n_elems; double coords[nv*dim]; int32 elems[ne*(dim+1)];
 * int32 tags[ne]; double pin[dim]), creates it through the C ABI, and prints the mesh info and
 * the membrane facets, the P2 node counts and the total of the intracellular P2 mass matrix. Then
 * it passes an out-of-range vertex id and prints the error code and message. Used by
 * tests/test_c_abi.py. */
#include <stdio.h>
#include <stdlib.h>

#include "knp.h"

static int read_all(FILE* f, void* p, size_t size, size_t n) { return fread(p, size, n, f) == n; }

int main(int argc, char** argv) {
    if (argc != 2) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    int32_t dim;
    int64_t nv, ne;
    if (!read_all(f, &dim, sizeof dim, 1) || !read_all(f, &nv, sizeof nv, 1) || !read_all(f, &ne, sizeof ne, 1)) return 2;
    double* coords = malloc(sizeof(double) * (size_t)(nv * dim));
    int32_t* elems = malloc(sizeof(int32_t) * (size_t)(ne * (dim + 1)));
    int32_t* tags = malloc(sizeof(int32_t) * (size_t)ne);
    double pin[3];
    if (!read_all(f, coords, sizeof(double), (size_t)(nv * dim)) ||
        !read_all(f, elems, sizeof(int32_t), (size_t)(ne * (dim + 1))) ||
        !read_all(f, tags, sizeof(int32_t), (size_t)ne) || !read_all(f, pin, sizeof(double), (size_t)dim))
        return 2;
    fclose(f);

    knp_mesh_desc d = {dim, nv, coords, ne, elems, tags, pin};
    knp_mesh* mesh = NULL;
    knp_status st = knp_mesh_create(&d, &mesh);
    if (st != KNP_OK) {
        printf("create failed %d %s\n", st, knp_last_error());
        return 1;
    }
    knp_mesh_info info;
    if (knp_mesh_get_info(mesh, &info) != KNP_OK) return 1;
    printf("info %d %lld %lld %lld %lld %lld %lld %d %lld %lld\n", info.dim, (long long)info.n_vertices,
           (long long)info.n_elems, (long long)info.N_i, (long long)info.N_e, (long long)info.n_facets,
           (long long)info.n_membrane_vertices, info.n_cells, (long long)info.pin_vertex, (long long)info.n_dof);
    int32_t* fv = malloc(sizeof(int32_t) * (size_t)(info.n_facets * dim));
    int32_t* fe = malloc(sizeof(int32_t) * (size_t)info.n_facets);
    int32_t* fo = malloc(sizeof(int32_t) * (size_t)info.n_facets);
    int32_t* fc = malloc(sizeof(int32_t) * (size_t)info.n_facets);
    if (knp_mesh_facets(mesh, fv, fe, fo, fc) != KNP_OK) return 1;
    for (int64_t k = 0; k < info.n_facets; ++k) {
        printf("facet");
        for (int j = 0; j < dim; ++j) printf(" %d", fv[k * dim + j]);
        printf(" %d %d %d\n", fe[k], fo[k], fc[k]);
    }
    /* P2 nodes (Section 3.3, p = 2) and the summed mass of the intracellular P2 elements */
    knp_p2_info p2;
    if (knp_mesh_p2_get_info(mesh, &p2) != KNP_OK) return 1;
    printf("p2 %lld %lld %lld %lld %lld %lld %lld\n", (long long)p2.n_edges, (long long)p2.n_nodes,
           (long long)p2.N_i, (long long)p2.N_e, (long long)p2.n_membrane_nodes, (long long)p2.pin_node,
           (long long)p2.n_dof);
    int64_t cnt = 0;
    if (knp_mesh_p2_region_matrices(mesh, 0, NULL, &cnt, NULL, NULL, NULL, NULL, NULL) != KNP_OK) return 1;
    double* mv = malloc(sizeof(double) * (size_t)cnt);
    if (knp_mesh_p2_region_matrices(mesh, 0, NULL, &cnt, NULL, NULL, mv, NULL, NULL) != KNP_OK) return 1;
    double vol = 0.0;
    for (int64_t k = 0; k < cnt; ++k) vol += mv[k];
    printf("p2mass %lld %.17g\n", (long long)cnt, vol);
    free(mv);
    knp_mesh_destroy(mesh);

    elems[0] = (int32_t)nv;   /* out of range */
    knp_mesh* bad = NULL;
    st = knp_mesh_create(&d, &bad);
    printf("error %d %s\n", st, knp_last_error());
    free(coords);
    free(elems);
    free(tags);
    free(fv);
    free(fe);
    free(fo);
    free(fc);
    return bad == NULL ? 0 : 1;
}
