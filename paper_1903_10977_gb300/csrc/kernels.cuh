// Device-side data of one multigrid level and the launch wrappers of the hot-path
// kernels (operator apply, Schwarz smoother, restriction, prolongation, coarse solve,
// CG vector updates).  The V-cycle kernels are templated on the storage and arithmetic
// type T (double for the FP64 path, float for the mixed-precision path); the CG kernels
// are FP64 and read the preconditioned residual z in either type.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace imgm {

// One level as the kernels see it (all pointers are device pointers).
template <typename T>
struct DevLevelT {
    int dim = 2, p = 2, m = 0, ncoef = 0;
    int64_t N = 0;
    const int32_t* rowinfo = nullptr;   // [N]: -2 inactive, -1 tensor-stencil row, >= 0 stored row id
    const T* band_coef = nullptr;       // [ncoef][nb]
    int32_t nb = 0;
    const int32_t* band_row = nullptr;  // [nb]: row of each stored row id
    const T* K1 = nullptr;              // [m][2p+1]
    const T* M1 = nullptr;              // [m][2p+1]
    const T* dinv = nullptr;            // [N]
    int32_t nblk = 0;
    int32_t max_block = 1;
    const int64_t* blk_ptr = nullptr;
    const int32_t* blk_idx = nullptr;
    const int64_t* blk_vptr = nullptr;
    const T* blk_val = nullptr;
    const int32_t* blk_of = nullptr;    // [npair]: block of each (block, function) pair
    int64_t npair = 0;                  // blk_ptr[nblk]
    // restriction to the next coarser level (levels >= 2)
    const int32_t* r_first = nullptr;   // [m_c]
    const T* r_w = nullptr;             // [m_c][p+2]
    const int32_t* t_first = nullptr;   // [m]
    const T* t_w = nullptr;             // [m][TW]
    int TW = 0;
    // Jacobi scaling of the mixed-precision V-cycle (nullptr on the FP64 path):
    // s = 1/sqrt(A_ii), d = sqrt(A_ii) on active rows, 0 elsewhere
    const T* s = nullptr;
    const T* d = nullptr;
    // work counter of the FP64 tile kernels ([0] next tile, [1] blocks done); zero between launches
    unsigned int* tile_ctr = nullptr;
    // scratch of the sum-factorised 3-D transfers from this level to the next coarser one
    // (m^2 m_c and m m_c^2 doubles; nullptr where the direct kernels run)
    double* xs1 = nullptr;
    double* xs2 = nullptr;
    // task shape of the 3-D z-marching apply (rows per lane, planes per chunk), picked by the
    // setup-time autotuner; 0 = the built-in rule
    int zm_yt = 0, zm_zc = 0;
    int zm_stage = 1;                   // FP32 input planes: 0 registers, 1 per-warp cp.async ring, 2 CTA ring
};
using DevLevel = DevLevelT<double>;

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
    double rz_prev;     // r_{k+1}^T z_k (flexible CG)
    int flexible;       // 1: Polak-Ribiere beta (mixed-precision V-cycle)
    int pad;
    // truncated flexible CG, FCG(m): p_j^T A p_j of the stored directions (ring slot j) and
    // the projection coefficients (z^T A p_j) / (p_j^T A p_j) of the current step
    double fcg_pq[8];
    double fcg_c[8];
};
constexpr int FCG_MAX = 8;

enum ApplyMode { APPLY = 0, RESID = 1, RESID_SMOOTH = 2 };

// whether a 3-D level of m functions per direction takes the z-marching apply (whose task
// shape, DevLevelT::zm_yt / zm_zc, the setup autotuner picks)
bool zm_applies(int m);
// whether a 2-D level takes the y-marching apply (rows per chunk: DevLevelT::zm_zc)
bool ym_applies(int m);

// y = A x (APPLY), out = rin - A x (RESID), or out = rin - A x followed by
// xs += gamma * dinv .* out (RESID_SMOOTH).  `out` may alias `rin`.
template <typename T>
cudaError_t launch_apply(const DevLevelT<T>& L, int mode, const T* x, const T* rin, T* out, T* xs, double gamma,
                         const int* done, cudaStream_t s);
// x = gamma * dinv .* r
template <typename T>
cudaError_t launch_scale_diag(const DevLevelT<T>& L, const T* r, T* x, double gamma, const int* done, cudaStream_t s);
// x[idx_j] += gamma * A_j^{-1} r[idx_j] for every stored Schwarz block (atomic adds)
template <typename T>
cudaError_t launch_blocks(const DevLevelT<T>& L, const T* r, T* x, double gamma, const int* done, cudaStream_t s);
// one colour of the multiplicative Schwarz sweep: x += P_j A_j^{-1} P_j^T r for the stored
// blocks [b_first, b_end) and x_i += sg_inv[k] r_i for the one-function blocks
// (i = sg_row[k], k < ns) of that colour
template <typename T>
cudaError_t launch_colour_smooth(const DevLevelT<T>& L, int64_t b_first, int64_t b_end, const int32_t* sg_row,
                                 const T* sg_inv, int64_t ns, const T* r, T* x, const int* done, cudaStream_t s);
// rc = R rf on the coarse rows; if xc != nullptr also xc = gamma * dinv_c .* rc
template <typename T>
cudaError_t launch_restrict(const DevLevelT<T>& F, const DevLevelT<T>& C, const T* rf, T* rc, T* xc, double gamma,
                            const int* done, cudaStream_t s);
// e = R^T xc on the fine rows (0 on inactive rows); if x != nullptr also x += e
template <typename T>
cudaError_t launch_prolong(const DevLevelT<T>& F, const DevLevelT<T>& C, const T* xc, T* e, T* x, const int* done,
                           cudaStream_t s);
// the transfers between an FP64 finest level and the FP32 (Jacobi-scaled) level below it:
// rc = D_c^{-1} R rf (and xc = gamma dinv_c .* rc when xc != nullptr), e = R^T D_c^{-1} xc, x += e
cudaError_t launch_restrict_64to32(const DevLevel& F, const DevLevelT<float>& C, const double* rf, float* rc, float* xc,
                                   double gamma, cudaStream_t s);
cudaError_t launch_prolong_32to64(const DevLevel& F, const DevLevelT<float>& C, const float* xc, double* e, double* x,
                                  cudaStream_t s);
// x[rows] = Cinv r[rows] (dense coarsest-level inverse, row-major nc x nc)
template <typename T>
cudaError_t launch_coarse(const int32_t* rows, const T* Cinv, int nc, const T* r, T* x, const int* done,
                          cudaStream_t s);

// V-cycle input from an FP64 residual: r_lo = (TZ)(rs .* r) (rs == nullptr: (TZ) r) and
// xv = gamma * dinv .* r_lo (the diagonal part of the first smoothing step)
template <typename TZ>
cudaError_t launch_vcycle_in(int64_t N, const double* r, const TZ* rs, const TZ* dinv, double gamma, TZ* r_lo, TZ* xv,
                             const int* done, cudaStream_t s);
// V-cycle output in FP64: out = zs .* z (zs == nullptr: out = z)
template <typename TZ>
cudaError_t launch_vcycle_out(int64_t N, const TZ* z, const TZ* zs, double* out, cudaStream_t s);

// q = A p (FP64) and the partial sums of p^T q; the last block sets alpha = rz / (p^T q).
cudaError_t launch_apply_pq(const DevLevel& L, const double* p, double* q, double* partial, PcgState* st,
                            cudaStream_t s);
// CG: x += alpha p, r -= alpha q, rr = ||r||^2 (last block: iteration count, history,
// convergence); then xv = gamma * dinv .* r in the V-cycle's type (the first smoothing
// step), and r_lo = (TZ) r when r_lo != nullptr (the V-cycle's copy of r)
// (rs: the V-cycle's scale 1/sqrt(A_ii), nullptr on the FP64 path)
template <typename TZ>
cudaError_t launch_pcg_update(const DevLevel& L, const TZ* dinv_z, double* x, double* r, const double* p,
                              const double* q, TZ* xv, TZ* r_lo, const TZ* rs, double gamma, double* partial,
                              PcgState* st, double* hist, cudaStream_t s);
// rz_new = r^T z; beta = rz_new / rz, or (r^T (z - z_prev)) / rz when zprev != nullptr, or
// -alpha (z^T q_prev) / rz when qprev (= A p of the step just taken) != nullptr: the
// Polak-Ribiere beta z^T (r - r_prev) / rz of flexible CG; rz = rz_new.
// z = zs .* z^ when zs != nullptr (scaled V-cycle), z otherwise.
template <typename TZ>
cudaError_t launch_pcg_rz(int64_t N, const double* r, const TZ* z, const TZ* zs, const TZ* zprev, double* partial,
                          PcgState* st, cudaStream_t s, const double* qprev = nullptr);
// p = z + beta p (and zprev = z^ when zprev != nullptr)
// Truncated flexible CG, FCG(m) (Notay 2000), FP64 z (after the V-cycle of this
// iteration and any learned stage): push_dots stores the direction just used (p, A p and
// p^T A p, the step's st->pq) in ring slot (iter - 1) mod m and forms
// c_j = (z^T A p_j) / (p_j^T A p_j) over the min(iter, m) stored directions; dir sets
// p = z - sum_j c_j p_j and st->rz = r^T p, from which the next apply takes alpha.
// Pring, Qring: m x N doubles each.
cudaError_t launch_fcg_push_dots(int64_t N, int m, const double* z, const double* p, const double* q, double* Pring,
                                 double* Qring, double* partial, PcgState* st, cudaStream_t s);
cudaError_t launch_fcg_dir(int64_t N, int m, const double* z, const double* r, double* p, const double* Pring,
                           double* partial, PcgState* st, cudaStream_t s);

template <typename TZ>
cudaError_t launch_pcg_xpay(int64_t N, const TZ* z, const TZ* zs, double* p, TZ* zprev, PcgState* st,
                            cudaStream_t s);
// CG start: rr = ||r||^2, bb = ||b||^2, convergence test of the initial guess (last block)
cudaError_t launch_pcg_init_norms(int64_t N, const double* r, const double* b, double* partial, PcgState* st,
                                  double* hist, cudaStream_t s);
// CG start after the first V-cycle: rz = r^T z, p = z (and zprev = z when zprev != nullptr)
template <typename TZ>
cudaError_t launch_pcg_init_dir(int64_t N, const double* r, const TZ* z, const TZ* zs, double* p, TZ* zprev,
                                double* partial, PcgState* st, cudaStream_t s);
// true_rr = ||v||^2 (last block)
cudaError_t launch_true_residual_norm(int64_t N, const double* v, double* partial, PcgState* st, cudaStream_t s);
// sets the conditional of the solve loop to !done
cudaError_t launch_set_continue(PcgState* st, unsigned long long handle, cudaStream_t s);

// ---- the coarse levels of the FP32 V-cycle resident in distributed shared memory ----
// One thread-block cluster holds levels 1..top+1 (indices 0..top) entirely on chip: the
// rows of every level are split into `ch`-row chunks, block k of the cluster owning
// chunk k.  Per-row vectors (x, r, t, e and the scales s, d) sit at the same offsets in
// every block, so any row's value is reached through the owner's shared memory (DSMEM);
// the tables a block needs only for its own rows (row kinds, stored coefficients, dinv,
// the Schwarz blocks it applies) and the small 1-D tables are its private image, built at
// setup and copied in at the start of each launch.  Offsets are in bytes from the start of
// the dynamic shared memory.
constexpr int DS_MAX_LEVELS = 8;
constexpr int DS_TPB = 1024;
constexpr uint32_t DS_SMEM_MAX = 200 * 1024;   // dynamic shared memory per block, at most
struct DsLevel {
    int m, N, ch, TW;                        // functions per direction, rows, rows per block, prolongation taps
    int nst, nblk;                           // stored rows and Schwarz blocks of this block
    uint32_t off_x, off_r, off_t, off_e, off_s, off_d;          // common per-row vectors (ch floats each)
    uint32_t off_ri, off_coef, off_dinv;                        // own rows: kind / local stored id, coefficients, dinv
    uint32_t off_K1, off_M1;                                    // 1-D rows [m][2p+1]
    uint32_t off_bptr, off_bvptr, off_bidx, off_bval;           // own Schwarz blocks
    uint32_t off_rfirst, off_rw, off_tfirst, off_tw;            // transfer to the next coarser level (index >= 1)
};
struct DsImage {                             // header of every block's image
    DsLevel lv[DS_MAX_LEVELS];
    int top, dim, p, max_block;
    float gamma;
    uint32_t vec_bytes;                      // common vector region (image starts there)
    uint32_t image_bytes;                    // largest image (all blocks reserve it)
    uint32_t scratch_off;                    // per-warp block scratch (max_block floats per warp)
};
struct DsVcycle {                            // launch parameters (by value)
    const unsigned char* images;             // cluster-size images, image_bytes apart
    const float* s_glob[DS_MAX_LEVELS];      // global scales s, d of each level (copied in per launch)
    const float* d_glob[DS_MAX_LEVELS];
    float* x_top;                            // global x, r of level top (from the finest restriction; x is written back)
    float* r_top;
    const int32_t* c_rows;                   // coarsest solve: kept rows and FP32 inverse (global)
    const float* c_inv;
    int nc, top, cs;
    uint32_t vec_bytes, image_bytes;         // as in the images' header
    uint32_t smem_bytes;                     // vec_bytes + image_bytes + block scratch
};
// dynamic shared memory and the launch; 0 when the device has no clusters of that size
int ds_cluster_size();
cudaError_t launch_vcycle_dsmem(int dim, int p, const DsVcycle& V, cudaStream_t s);

int reduction_blocks();   // fixed number of blocks of every reducing kernel
// programmatic dependent launch of the kernels issued by this host thread (default on)
void set_programmatic_launch(bool on);
// kernels launched (or captured) so far by this host thread
int64_t launch_count();
// counts k kernels launched by this host thread outside this file's launch helper
void add_launches(int64_t k);

}  // namespace imgm
