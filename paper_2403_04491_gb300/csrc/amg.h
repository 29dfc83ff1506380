// Smoothed-aggregation hierarchy for the block-diagonal preconditioner P_0 (Eq. 4.4).
//
// P_0 has 2(|K|+1) diagonal blocks: per region, M_r + tau_r^k A_r for each ion and
// C_m/F M_{r,Gamma} + sum_k z_k tau~_r^k A_r^{k,0} for the potential. All blocks of a
// region share the region's node graph, so the hierarchy aggregates nodes once and
// carries four independent fields per node ("field-diagonal node blocks"): one
// aggregation, one sparsity pattern per level, four value sets. The intracellular and
// extracellular graphs are disconnected, so aggregates never cross the membrane or
// join two cells (the per-cell split of Section 4.2 falls out of the graph).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace knp {

// CSR with four values per entry ([nnz][4], field-major inside an entry).
struct HostCsr4 {
    int64_t n_rows = 0, n_cols = 0;
    std::vector<int64_t> ptr;
    std::vector<int32_t> col;
    std::vector<double> val;
    int64_t nnz() const { return (int64_t)col.size(); }
};

struct HostLevel {
    HostCsr4 A;                   // operator of this level
    std::vector<double> dinv;     // [n][4] inverse diagonal
    double lmax[4], lmin[4];      // Chebyshev interval of D^-1 A per field
    HostCsr4 P;                   // prolongation to this level from the next (n_l x n_{l+1}); empty on the last
    HostCsr4 R;                   // P^T
};

struct HostHierarchy {
    std::vector<HostLevel> levels;
    std::vector<double> coarse_inv;   // [4][nc][nc] dense inverses of the coarsest operator, row-major
    int64_t nc = 0;
};

struct AmgSetupOpts {
    double theta;
    int coarse_max;
    int max_levels;
    double cheb_ratio;
    double theta_coarse;
    double p_drop;
};

// Builds the hierarchy from the fine operator (field values) and the fine
// strength operator (one scalar per entry). pin_row: row whose field 3 is pinned
// (excluded from the field-3 near-null vector), or -1.
void amg_build(const HostCsr4& A0, const std::vector<double>& strength0, int64_t pin_row,
               const AmgSetupOpts& o, HostHierarchy& H);
// the same on the GPU (amg_gpu.cu); the coarsest dense inverse stays on the host. Returns false
// when a row of P exceeds the kernel's fixed capacity (the caller then builds on the host).
bool amg_build_gpu(const HostCsr4& A0, const std::vector<double>& strength0, int64_t pin_row,
                   const AmgSetupOpts& o, HostHierarchy& H, cudaStream_t st,
                   void (*host_spgemm)(const HostCsr4&, const HostCsr4&, HostCsr4&));
void amg_host_spgemm(const HostCsr4& A, const HostCsr4& B, HostCsr4& C);
void amg_coarse_inverse(HostHierarchy& H);

}  // namespace knp
