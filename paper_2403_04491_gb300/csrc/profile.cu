// Launch counter and per-class event timing behind knp_profile_begin / knp_profile_end.
#include "problem.h"
#include "profile.h"

namespace knp {

std::atomic<int64_t> g_launches{0};

Profiler::~Profiler() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

void Profiler::begin(int, cudaStream_t s) {
    if (used + 2 > pool.size()) {
        for (int k = 0; k < 256; ++k) {
            cudaEvent_t e;
            KNP_CUDA(cudaEventCreate(&e));
            pool.push_back(e);
        }
    }
    KNP_CUDA(cudaEventRecord(pool[used], s));
}

void Profiler::end(int, cudaStream_t s) {
    KNP_CUDA(cudaEventRecord(pool[used + 1], s));
    used += 2;
}

}  // namespace knp

using namespace knp;

extern "C" {

knp_status knp_profile_begin(knp_problem* p, int32_t cls) {
    return guarded([&] {
        KNP_REQUIRE(p, KNP_ERR_INVALID_ARG, "NULL problem");
        KNP_REQUIRE(cls >= 0 && cls <= 5, KNP_ERR_INVALID_ARG, "unknown kernel class %d", cls);
        p->prof.active = cls;
        p->prof.used = 0;
    });
}

knp_status knp_profile_end(knp_problem* p, int64_t* launches, double* total_ms) {
    return guarded([&] {
        KNP_REQUIRE(p, KNP_ERR_INVALID_ARG, "NULL problem");
        KNP_CUDA(cudaStreamSynchronize(p->stream));
        double tot = 0;
        for (size_t i = 0; i + 1 < p->prof.used; i += 2) {
            float ms = 0;
            KNP_CUDA(cudaEventElapsedTime(&ms, p->prof.pool[i], p->prof.pool[i + 1]));
            tot += ms;
        }
        if (launches) *launches = (int64_t)(p->prof.used / 2);
        if (total_ms) *total_ms = tot;
        p->prof.active = -1;
        p->prof.used = 0;
    });
}

knp_status knp_launch_count(int64_t* count) {
    return guarded([&] {
        KNP_REQUIRE(count, KNP_ERR_INVALID_ARG, "NULL argument");
        *count = g_launches.load();
    });
}

knp_status knp_problem_get_info(const knp_problem* p, knp_problem_info* info) {
    return guarded([&] {
        KNP_REQUIRE(p && info, KNP_ERR_INVALID_ARG, "NULL argument");
        info->n_nodes = p->n_nodes;
        int64_t real = 0;
        const SellPattern& S = p->sell;
        for (int64_t r = 0; r < p->n_nodes; ++r) {
            int64_t s = r / SELL_C, base = S.h_slice_ptr[s] + r % SELL_C;
            int64_t w = (S.h_slice_ptr[s + 1] - S.h_slice_ptr[s]) / SELL_C;
            int32_t prev = -1;
            for (int64_t k = 0; k < w; ++k) {
                int32_t c = S.h_col[base + k * SELL_C];
                if (c <= prev) break;
                prev = c;
                ++real;
            }
        }
        info->nnz_region = real;
        info->nnz_padded = S.n_entries;
        info->nnz_cross = (int64_t)p->h_xcol.size();
        info->n_membrane_pairs = p->n_pairs;
        info->n_edges = p->n_edges;
        info->edge_incidences = p->n_edge_inc;
        info->step_index = p->step_index;
    });
}

}  // extern "C"
