// Launch counting and optional per-class CUDA-event timing (knp_profile_begin/end).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <vector>

struct knp_problem;

namespace knp {

enum KernelClass { KC_SPMV = 0, KC_CHEB_FINE = 1, KC_RESID_FINE = 2, KC_ASSEMBLY = 3, KC_VCYCLE = 4, KC_ORTHO = 5 };

extern std::atomic<int64_t> g_launches;
inline void count_launch(int n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

struct Profiler {
    int active = -1;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    ~Profiler();
    void begin(int cls, cudaStream_t s);
    void end(int cls, cudaStream_t s);
};

// RAII interval: records an event pair around a launch group when its class is active.
struct ProfScope {
    Profiler* pr;
    int cls;
    cudaStream_t s;
    ProfScope(Profiler* p, int c, cudaStream_t st) : pr(p), cls(c), s(st) {
        if (pr && pr->active == cls) pr->begin(cls, s);
    }
    ~ProfScope() {
        if (pr && pr->active == cls) pr->end(cls, s);
    }
};

}  // namespace knp
