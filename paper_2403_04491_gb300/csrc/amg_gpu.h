// The GPU construction of the smoothed-aggregation hierarchy on P_0 (Eq. 4.4, Section 4.2) and
// its device-resident result, which the V-cycle takes over without a copy through the host.
#pragma once

#include <memory>
#include <vector>

#include "amg.h"
#include "problem.h"

namespace knp {

// CSR with four values per entry ([nnz][4], field-major inside an entry), on the device.
struct DevCsr4d {
    int64_t n_rows = 0, n_cols = 0, nnz = 0;
    DArray<int64_t> ptr;
    DArray<int32_t> col;
    DArray<double> val;
};

struct GpuLevel {
    DevCsr4d A;                   // operator of this level
    DArray<double> dinv;          // [n][4] inverse diagonal
    double lmax[4], lmin[4];      // Chebyshev interval of D^-1 A per field
    DevCsr4d P, R;                // prolongation from the next level and P^T; empty on the last
};

struct GpuHierarchy {
    std::vector<std::unique_ptr<GpuLevel>> levels;
    std::vector<double> coarse_inv;   // [4][nc][nc] dense inverses of the coarsest operator
    int64_t nc = 0;
    int64_t long_rows_p = 0;          // rows of P finished by the long-row kernel
    int64_t long_rows_rap = 0;        // rows of A P and R (A P) finished by the long-row kernel
};

// P_0 from the assembled A_0 (Eq. 4.4): the field-diagonal node blocks on the region pattern with
// the point pin of Remark 4.1, the strength scalar per entry (the stiffness value a) and the
// diagonal scaling vectors of the solver (S = sqrt(diag P_0), S^-1, and S with the pinned row
// zeroed). All on the device; KNP_ERR_NUMERIC if a diagonal entry is not positive.
void p0_extract(knp_problem* p, DevCsr4d& A0, DArray<double>& strength);
// The hierarchy on the GPU from P_0 (consumes A0 and strength). Rows of P or of the Galerkin
// products that exceed the short-row kernels' capacity are finished on the GPU by the long-row
// kernels. `short_row_max` > 0 lowers that capacity (a testing aid that sends more rows down the
// long-row path); 0 keeps the default.
void amg_build_gpu(DevCsr4d& A0, DArray<double>& strength, int64_t pin_row, const AmgSetupOpts& o, GpuHierarchy& H,
                   cudaStream_t st, int short_row_max = 0);
void download(const DevCsr4d& d, HostCsr4& h, cudaStream_t st);
// out[0..n] = exclusive scan of in[0..n-1], out[n] = total; returns the total (synchronises)
int64_t device_exclusive_scan(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st);

}  // namespace knp
