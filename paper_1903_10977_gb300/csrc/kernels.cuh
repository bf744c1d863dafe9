// Device-side data of one multigrid level and the launch wrappers of the hot-path
// kernels (operator apply, Schwarz smoother, restriction, prolongation, coarse solve,
// CG vector updates).  All arithmetic is FP64.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace imgm {

// One level as the kernels see it (all pointers are device pointers).
struct DevLevel {
    int dim = 2, p = 2, m = 0, ncoef = 0;
    int64_t N = 0;
    const int32_t* rowinfo = nullptr;   // [N]: -2 inactive, -1 tensor-stencil row, >= 0 stored row id
    const double* band_coef = nullptr;  // [ncoef][nb]
    int32_t nb = 0;
    const double* K1 = nullptr;         // [m][2p+1]
    const double* M1 = nullptr;         // [m][2p+1]
    const double* dinv = nullptr;       // [N]
    int32_t nblk = 0;
    int32_t max_block = 1;
    const int64_t* blk_ptr = nullptr;
    const int32_t* blk_idx = nullptr;
    const int64_t* blk_vptr = nullptr;
    const double* blk_val = nullptr;
    // restriction to the next coarser level (levels >= 2)
    const int32_t* r_first = nullptr;   // [m_c]
    const double* r_w = nullptr;        // [m_c][p+2]
    const int32_t* t_first = nullptr;   // [m]
    const double* t_w = nullptr;        // [m][TW]
    int TW = 0;
};

// Scalars of the CG iteration, kept on the device.
struct PcgState {
    double rz;          // r^T z of the current iterate
    double pq;          // p^T A p
    double rr;          // ||r||^2
    double bb;          // ||b||^2
    double alpha, beta;
    double tol2;        // rtol^2
    double true_rr;     // ||b - A x||^2 at exit
    int iter, maxit, done, status;
    unsigned int ticket[4];   // last-block reduction counters
};

enum ApplyMode { APPLY = 0, RESID = 1, RESID_SMOOTH = 2 };

// y = A x (APPLY), out = rin - A x (RESID), or out = rin - A x followed by
// xs += gamma * dinv .* out (RESID_SMOOTH).  `out` may alias `rin`.
cudaError_t launch_apply(const DevLevel& L, int mode, const double* x, const double* rin, double* out, double* xs,
                         double gamma, const int* done, cudaStream_t s);
// q = A p and the partial sums of p^T q; the last block sets alpha = rz / (p^T q) in st.
cudaError_t launch_apply_pq(const DevLevel& L, const double* p, double* q, double* partial, PcgState* st,
                            cudaStream_t s);
// x = gamma * dinv .* r
cudaError_t launch_scale_diag(const DevLevel& L, const double* r, double* x, double gamma, const int* done,
                              cudaStream_t s);
// x[idx_j] += gamma * A_j^{-1} r[idx_j] for every stored Schwarz block (atomic adds)
cudaError_t launch_blocks(const DevLevel& L, const double* r, double* x, double gamma, const int* done,
                          cudaStream_t s);
// rc = R rf on the coarse rows; if xc != nullptr also xc = gamma * dinv_c .* rc
cudaError_t launch_restrict(const DevLevel& F, const DevLevel& C, const double* rf, double* rc, double* xc,
                            double gamma, const int* done, cudaStream_t s);
// e = R^T xc on the fine rows (0 on inactive rows); if x != nullptr also x += e
cudaError_t launch_prolong(const DevLevel& F, const DevLevel& C, const double* xc, double* e, double* x,
                           const int* done, cudaStream_t s);
// x[rows] = Cinv r[rows] (dense coarsest-level inverse, row-major nc x nc)
cudaError_t launch_coarse(const int32_t* rows, const double* Cinv, int nc, const double* r, double* x,
                          const int* done, cudaStream_t s);
// CG: x += alpha p, r -= alpha q, rr = ||r||^2 (last block: iteration count, history,
// convergence); then xv = gamma * dinv .* r for the V-cycle's first smoothing step
cudaError_t launch_pcg_update(const DevLevel& L, double* x, double* r, const double* p, const double* q, double* xv,
                              double gamma, double* partial, PcgState* st, double* hist, cudaStream_t s);
// rz_new = r^T z; beta = rz_new / rz; rz = rz_new (last block)
cudaError_t launch_pcg_rz(int64_t N, const double* r, const double* z, double* partial, PcgState* st, cudaStream_t s);
// p = z + beta p
cudaError_t launch_pcg_xpay(int64_t N, const double* z, double* p, PcgState* st, cudaStream_t s);
// CG start: rr = ||r||^2, bb = ||b||^2, convergence test of the initial guess (last block)
cudaError_t launch_pcg_init_norms(int64_t N, const double* r, const double* b, double* partial, PcgState* st,
                                  double* hist, cudaStream_t s);
// CG start after the first V-cycle: rz = r^T z, p = z
cudaError_t launch_pcg_init_dir(int64_t N, const double* r, const double* z, double* p, double* partial,
                                PcgState* st, cudaStream_t s);
// true_rr = ||v||^2 (last block)
cudaError_t launch_true_residual_norm(int64_t N, const double* v, double* partial, PcgState* st, cudaStream_t s);
// sets the conditional of the solve loop to !done
cudaError_t launch_set_continue(PcgState* st, unsigned long long handle, cudaStream_t s);

int reduction_blocks();   // fixed number of blocks of every reducing kernel

}  // namespace imgm
