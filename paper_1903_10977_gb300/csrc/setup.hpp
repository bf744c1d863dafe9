// Host-side construction of the immersed discretisation and of the multigrid
// hierarchy (everything the GPU kernels read).  Plain C++17, no CUDA types.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace imgm {

struct Ball {
    double c[3];
    double r;
};

struct Problem {
    int dim = 2;
    std::vector<Ball> holes;
    double lo = 0.0, hi = 1.0;
    int n = 32, basis = 0, p = 2, levels = 3, depth = 0, bc = 1;
    double gamma = 0.0;
    int precision = 0;   // 0: FP64 V-cycle, 1: FP32 V-cycle, 2: FP64 finest level + FP32 below (FP32 copies for 1, 2)
    int smoother = 0;    // 0: additive Schwarz, 1: coloured multiplicative Schwarz
};

// Everything the kernels of one level need.  Row index = ix + m*(iy + m*iz).
struct LevelData {
    int n = 0, m = 0;
    double h = 0.0;
    int64_t N = 0;
    int64_t n_active = 0;
    std::vector<uint8_t> active;       // [N]
    std::vector<int32_t> rowinfo;      // [N]: -2 inactive, -1 tensor-stencil row, >= 0 stored row id
    std::vector<int32_t> band_rows;    // stored row id -> row
    std::vector<double> band_coef;     // [ncoef][n_band] (structure of arrays)
    std::vector<double> K1, M1;        // [m][2p+1] 1-D stiffness / mass rows (offset -p..p)
    std::vector<double> dinv;          // [N] sum of 1/A_ii over one-function blocks holding i
    // Schwarz blocks with >= 2 functions after pruning
    std::vector<int64_t> blk_ptr;      // [nblk+1] into blk_idx
    std::vector<int32_t> blk_idx;      // rows of each block
    std::vector<int64_t> blk_vptr;     // [nblk+1] into blk_val
    std::vector<double> blk_val;       // A_j^{-1}, column-major n_j x n_j
    int64_t pruned = 0, max_block = 1;
    // coloured multiplicative Schwarz (smoother 1): the stored blocks above are sorted by
    // colour, blocks [blk_cptr[c], blk_cptr[c+1]) have colour c; the one-function blocks
    // are listed per colour as (row, 1/A_kk) in [sg_cptr[c], sg_cptr[c+1])
    int ncolour = 0;
    std::vector<int64_t> blk_cptr, sg_cptr;
    std::vector<int32_t> sg_row;
    std::vector<double> sg_inv;
    // restriction to the next coarser level (levels >= 2), 1-D tables
    std::vector<int32_t> r_first;      // [m_c] first fine index of coarse function i
    std::vector<double> r_w;           // [m_c][p+2]
    std::vector<int32_t> t_first;      // [m_f] first coarse index of fine function a
    std::vector<double> t_w;           // [m_f][TW] weights R[t_first+k][a]
    int TW = 0;
    // element status (finest-descendant based)
    std::vector<uint8_t> elem_active;  // [n^d]
    std::vector<uint8_t> elem_full;    // [n^d]
    // FP32 copies for the mixed-precision V-cycle, in Jacobi-scaled variables
    // (D = diag(A)^{1/2}): stored rows A_ij/(d_i d_j), block inverses d_a A_j^{-1}_ab d_b,
    // dinv d_i^2 / A_ii-sums, the scale s = 1/d and d itself; tables unscaled
    std::vector<float> f_band_coef, f_K1, f_M1, f_dinv, f_blk_val, f_r_w, f_t_w, f_s, f_d, f_sg_inv;
};

struct Hierarchy {
    int dim = 2, p = 2, L = 2, bc = 1, ncoef = 0, smoother = 0;
    double gamma = 0.0;
    std::vector<LevelData> lv;         // lv[0] = level 1 (coarsest) ... lv[L-1] = finest
    std::vector<double> b;             // finest right-hand side [N_L]
    std::vector<int32_t> c_rows;       // active rows of level 1 kept by the Remark 3.3 rule
    std::vector<double> c_inv;         // [nc x nc] row-major inverse on those rows
    std::vector<float> f_c_inv;        // FP32 d_a C_ab d_b (scaled variables of level 1)
    int64_t coarse_pruned = 0;
    int64_t n_cut = 0;
    double setup_seconds = 0.0;
};

// Builds the hierarchy; returns false and sets err on failure.
bool build_hierarchy(const Problem& pb, Hierarchy& H, std::string& err);

}  // namespace imgm
