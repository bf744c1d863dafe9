// Hot-path kernels of the immersed multigrid-preconditioned CG solve.
//
//   operator apply   A_l x            (Eq. systemMulti; Galerkin rows of Remark 3.1)
//   Schwarz smoother gamma M^{-1} r   (Sec. 3.4, additive Schwarz with stored block inverses)
//   restriction      R_l r            (Eq. coarsening)
//   prolongation     R_l^T x          (Sec. 3.3)
//   coarsest solve   A_1^{-1} r       (Algorithm 1, direct solve on level 1)
//   CG updates and dot products       (Sec. 3.2, the V-cycle as CG preconditioner)
//
// Rows of a level are either "tensor" rows, whose whole support lies in full elements,
// where A = K (x) M + M (x) K [+ ...] with the 1-D stiffness/mass rows K1/M1, or "stored"
// rows (support touching a cut, empty or partly active element) whose (2p+1)^d
// coefficients were assembled at setup.  Vectors hold 0 on inactive rows.
//
// The V-cycle kernels are templates on T.  T = double: the FP64 path, plain variables.
// T = float: the mixed-precision V-cycle, which works in Jacobi-scaled variables
// x^ = D x, r^ = D^{-1} r with D = diag(A_l)^{1/2} per level (L.s = 1/d, L.d = d): the
// stored coefficients, block inverses and coarse inverse arrive pre-scaled from setup,
// the tensor rows scale on the fly (y^ = s_i sum_j A_ij s_j x^_j), and the transfers use
// D_c^{-1} R D_f.  Cut functions make diagonal entries span 40+ orders of magnitude,
// which FP32 cannot hold unscaled.
// Reductions are FP64 and deterministic: fixed grid, per-block partials summed in a
// fixed order by the last block to finish.
#include "common.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace imgm {
namespace {

int g_red_blocks = 0;
// (A x)_i for one row (scaled variables when L.s != nullptr)
template <typename T, int DIM, int P>
__device__ __forceinline__ T row_apply(const DevLevelT<T>& L, int64_t i, const T* __restrict__ x) {
    constexpr int W = 2 * P + 1;
    const int ri = L.rowinfo[i];
    if (ri == -2) return T(0);
    const int m = L.m;
    const int ix = (int)(i % m);
    const int iy = (int)((i / m) % m);
    const int iz = (DIM == 3) ? (int)(i / ((int64_t)m * m)) : 0;
    const int64_t sy = m, sz = (int64_t)m * m;
    const T* __restrict__ sc = L.s;
    T y = T(0);
    if (ri >= 0) {
        const T* __restrict__ c = L.band_coef + ri;
        const int64_t nb = L.nb;
#pragma unroll
        for (int oz = (DIM == 3 ? -P : 0); oz <= (DIM == 3 ? P : 0); ++oz) {
            if (DIM == 3 && (unsigned)(iz + oz) >= (unsigned)m) continue;
#pragma unroll
            for (int oy = -P; oy <= P; ++oy) {
                if ((unsigned)(iy + oy) >= (unsigned)m) continue;
#pragma unroll
                for (int ox = -P; ox <= P; ++ox) {
                    if ((unsigned)(ix + ox) >= (unsigned)m) continue;
                    const int ci = (ox + P) + W * ((oy + P) + (DIM == 3 ? W * (oz + P) : 0));
                    y = fmaT(ro(c + (int64_t)ci * nb), x[i + ox + oy * sy + (DIM == 3 ? oz * sz : 0)], y);
                }
            }
        }
        return y;
    }
    const T* __restrict__ Kx = L.K1 + (int64_t)ix * W + P;
    const T* __restrict__ Mx = L.M1 + (int64_t)ix * W + P;
    const T* __restrict__ Ky = L.K1 + (int64_t)iy * W + P;
    const T* __restrict__ My = L.M1 + (int64_t)iy * W + P;
    T kx[W], mx[W];
#pragma unroll
    for (int ox = -P; ox <= P; ++ox) {
        kx[ox + P] = ro(Kx + ox);
        mx[ox + P] = ro(Mx + ox);
    }
    if (DIM == 2) {
#pragma unroll
        for (int oy = -P; oy <= P; ++oy) {
            if ((unsigned)(iy + oy) >= (unsigned)m) continue;
            T a = T(0), b = T(0);
            const int64_t rb = i + oy * sy;
#pragma unroll
            for (int ox = -P; ox <= P; ++ox) {
                if ((unsigned)(ix + ox) >= (unsigned)m) continue;
                const T xv = sc ? x[rb + ox] * ro(sc + rb + ox) : x[rb + ox];
                a = fmaT(kx[ox + P], xv, a);
                b = fmaT(mx[ox + P], xv, b);
            }
            y = fmaT(ro(My + oy), a, y);
            y = fmaT(ro(Ky + oy), b, y);
        }
        return sc ? y * ro(sc + i) : y;
    }
    const T* __restrict__ Kz = L.K1 + (int64_t)iz * W + P;
    const T* __restrict__ Mz = L.M1 + (int64_t)iz * W + P;
#pragma unroll
    for (int oz = -P; oz <= P; ++oz) {
        if ((unsigned)(iz + oz) >= (unsigned)m) continue;
        const T mz = ro(Mz + oz), kz = ro(Kz + oz);
#pragma unroll
        for (int oy = -P; oy <= P; ++oy) {
            if ((unsigned)(iy + oy) >= (unsigned)m) continue;
            const T my = ro(My + oy), ky = ro(Ky + oy);
            T a = T(0), b = T(0);
            const int64_t rb = i + oy * sy + oz * sz;
#pragma unroll
            for (int ox = -P; ox <= P; ++ox) {
                if ((unsigned)(ix + ox) >= (unsigned)m) continue;
                const T xv = sc ? x[rb + ox] * ro(sc + rb + ox) : x[rb + ox];
                a = fmaT(kx[ox + P], xv, a);
                b = fmaT(mx[ox + P], xv, b);
            }
            // sum_ox (kx my mz + mx ky mz + mx my kz) x = my mz a + (ky mz + my kz) b
            y = fmaT(my * mz, a, y);
            y = fmaT(fmaT(ky, mz, my * kz), b, y);
        }
    }
    return sc ? y * ro(sc + i) : y;
}

template <typename T, int DIM, int P>
__device__ __forceinline__ void apply_rows(const DevLevelT<T>& L, int mode, const T* __restrict__ x, const T* rin,
                                           T* out, T* __restrict__ xs, T gamma, int64_t start, int64_t stride) {
    for (int64_t i = start; i < L.N; i += stride) {
        const T ax = row_apply<T, DIM, P>(L, i, x);
        if (mode == APPLY) {
            out[i] = ax;
        } else {
            const T v = (L.rowinfo[i] == -2) ? T(0) : rin[i] - ax;
            out[i] = v;
            if (mode == RESID_SMOOTH) xs[i] = fmaT(gamma * ro(L.dinv + i), v, xs[i]);
        }
    }
}

template <typename T, int DIM, int P>
__global__ void __launch_bounds__(TPB) k_apply(DevLevelT<T> L, int mode, const T* __restrict__ x, const T* rin,
                                               T* out, T* __restrict__ xs, T gamma, const int* done) {
    pdl_begin();
    if (done && *done) return;
    apply_rows<T, DIM, P>(L, mode, x, rin, out, xs, gamma, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                          (int64_t)gridDim.x * blockDim.x);
}

// ---------------------------------------------------------------------------------
// 2-D operator apply on TX x TY tiles with sum factorisation.  The x values of the tile
// and a p-wide halo are staged in shared memory; the tensor rows then cost
//   u = M_y x, v = K_y x  on the (TX+2p) x TY strip   (2 (2p+1) FMA per point)
//   y = K_x u + M_x v     on the TX x TY outputs      (2 (2p+1) FMA per point)
// i.e. about 4(2p+1) FMA per row instead of 2(2p+1)^2 + 2(2p+1) for the direct sum.
// Stored rows read their (2p+1)^2 coefficients and take x from the same staged tile.
// MODE: APPLY, RESID, RESID_SMOOTH as in k_apply; DOT (FP64 only) also accumulates
// sum_i x_i (A x)_i and finishes with alpha = rz / (p^T A p) (the CG step length).
constexpr int TX = 32, TY = 16;

template <typename T, int P, int MODE, bool DOT>
__global__ void __launch_bounds__(TPB) k_apply_tile2d(DevLevelT<T> L, const T* __restrict__ x, const T* rin, T* out,
                                                      T* __restrict__ xs, T gamma, const int* done, double* partial,
                                                      PcgState* st) {
    pdl_begin();
    constexpr int W = 2 * P + 1;
    constexpr int SX = TX + 2 * P, SY = TY + 2 * P;
    constexpr int OUT_PER_THREAD = (TX * TY) / TPB;
    static_assert(OUT_PER_THREAD * TPB == TX * TY, "tile must be a multiple of the block");
    __shared__ T sx[SY][SX];     // x (scaled variables x^ in the FP32 path)
    __shared__ T ss[SY][SX];     // 1/d (FP32 path) or 1
    __shared__ T su[TY][SX];
    __shared__ T sv[TY][SX];
    __shared__ T tMy[TY][W], tKy[TY][W];   // 1-D rows of the tile's y indices
    __shared__ T tKx[TX][W], tMx[TX][W];   // 1-D rows of the tile's x indices
    __shared__ int s_tile;
    if (done && *done) return;
    const int m = L.m;
    const bool scaled = L.s != nullptr;
    const int tiles_x = (m + TX - 1) / TX, tiles_y = (m + TY - 1) / TY;
    const int ntiles = tiles_x * tiles_y;
    // FP64: a grid smaller than the tile count takes tiles from a counter, so that SMs that
    // finish early take more (tiles along a cut cost more, and FP64 issue is per SM);
    // FP32: one tile per block, no counter round trip
    const bool dyn = sizeof(T) == 8 && MODE == APPLY && (int)gridDim.x < ntiles;
    double acc = 0.0;
    for (int tb = blockIdx.x;; tb += gridDim.x) {
        __syncthreads();   // the previous tile's smem reads (and s_tile) are done
        if (dyn) {
            if (threadIdx.x == 0) s_tile = (int)atomicAdd(&L.tile_ctr[0], 1u);
            __syncthreads();
        }
        const int tile = dyn ? s_tile : tb;
        if (tile >= ntiles) break;
        const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
        // one round of independent global loads: the x tile with its halo, the 1-D table
        // rows, and everything the outputs of this thread need that does not depend on x
        for (int k = threadIdx.x; k < SX * SY; k += TPB) {
            const int ly = k / SX, lx = k % SX;
            const int gx = x0 + lx - P, gy = y0 + ly - P;
            const bool in = (unsigned)gx < (unsigned)m && (unsigned)gy < (unsigned)m;
            const int64_t g = (int64_t)gy * m + gx;
            sx[ly][lx] = in ? x[g] : T(0);
            ss[ly][lx] = in ? (scaled ? ro(L.s + g) : T(1)) : T(0);
        }
        for (int k = threadIdx.x; k < TY * W; k += TPB) {
            const int ly = k / W, o = k % W;
            const int gy = y0 + ly;
            tMy[ly][o] = gy < m ? ro(L.M1 + (int64_t)gy * W + o) : T(0);
            tKy[ly][o] = gy < m ? ro(L.K1 + (int64_t)gy * W + o) : T(0);
        }
        for (int k = threadIdx.x; k < TX * W; k += TPB) {
            const int lx = k / W, o = k % W;
            const int gx = x0 + lx;
            tKx[lx][o] = gx < m ? ro(L.K1 + (int64_t)gx * W + o) : T(0);
            tMx[lx][o] = gx < m ? ro(L.M1 + (int64_t)gx * W + o) : T(0);
        }
        int ri[OUT_PER_THREAD];
        T rv[OUT_PER_THREAD], dv[OUT_PER_THREAD], xv[OUT_PER_THREAD];
#pragma unroll
        for (int q = 0; q < OUT_PER_THREAD; ++q) {
            const int k = threadIdx.x + q * TPB;
            const int gx = x0 + k % TX, gy = y0 + k / TX;
            const bool in = gx < m && gy < m;
            const int64_t i = (int64_t)gy * m + gx;
            ri[q] = in ? ro(L.rowinfo + i) : -3;
            rv[q] = (MODE != APPLY && in) ? rin[i] : T(0);
            dv[q] = (MODE == RESID_SMOOTH && in) ? ro(L.dinv + i) : T(0);
            xv[q] = (MODE == RESID_SMOOTH && in) ? xs[i] : T(0);
        }
        __syncthreads();
        // stage 1: along y, for all columns of the strip
        for (int k = threadIdx.x; k < TY * SX; k += TPB) {
            const int ly = k / SX, lx = k % SX;
            T u = T(0), v = T(0);
#pragma unroll
            for (int o = 0; o < W; ++o) {
                const T xq = scaled ? sx[ly + o][lx] * ss[ly + o][lx] : sx[ly + o][lx];
                u = fmaT(tMy[ly][o], xq, u);
                v = fmaT(tKy[ly][o], xq, v);
            }
            su[ly][lx] = u;
            sv[ly][lx] = v;
        }
        __syncthreads();
        // stage 2: along x; stored rows take their coefficients from global memory
#pragma unroll
        for (int q = 0; q < OUT_PER_THREAD; ++q) {
            if (ri[q] == -3) continue;
            const int k = threadIdx.x + q * TPB;
            const int ly = k / TX, lx = k % TX;
            const int64_t i = (int64_t)(y0 + ly) * m + (x0 + lx);
            T y = T(0);
            if (ri[q] == -1) {
#pragma unroll
                for (int o = 0; o < W; ++o) {
                    y = fmaT(tKx[lx][o], su[ly][lx + o], y);
                    y = fmaT(tMx[lx][o], sv[ly][lx + o], y);
                }
                if (scaled) y *= ss[ly + P][lx + P];
            } else if (ri[q] >= 0) {
                const T* __restrict__ c = L.band_coef + ri[q];
                const int64_t nb = L.nb;
#pragma unroll
                for (int oy = 0; oy < W; ++oy)
#pragma unroll
                    for (int ox = 0; ox < W; ++ox) y = fmaT(ro(c + (int64_t)(ox + W * oy) * nb), sx[ly + oy][lx + ox], y);
            }
            if (MODE == APPLY) {
                out[i] = y;
            } else {
                const T r = (ri[q] == -2) ? T(0) : rv[q] - y;
                out[i] = r;
                if (MODE == RESID_SMOOTH) xs[i] = fmaT(gamma * dv[q], r, xv[q]);
            }
            if (DOT) acc = fma((double)sx[ly + P][lx + P], (double)y, acc);
        }
    }
    if (dyn && threadIdx.x == 0) {
        // every block has drawn past the end once; the last one re-arms the counter for the
        // next launch (which starts only after this grid has completed)
        if (atomicAdd(&L.tile_ctr[1], 1u) == gridDim.x - 1) {
            L.tile_ctr[0] = 0u;
            L.tile_ctr[1] = 0u;
        }
    }
    if (DOT) {
        double pq;
        if (finish_reduction(acc, partial, &st->ticket[0], &pq) && threadIdx.x == 0) {
            st->pq = pq;
            if (!(pq > 0.0) || !isfinite(pq)) {
                st->done = 1;
                st->status = -5;
                st->alpha = 0.0;
            } else {
                st->alpha = st->rz / pq;
            }
        }
    }
}


// ---------------------------------------------------------------------------------
// 2-D operator apply by y-marching warps, the 2-D form of k_apply_zm3d: a warp owns 32 - 2P
// x columns (lanes, P halo lanes each side) and a chunk of y rows, and walks the input rows
// with a ring of 2P + 1 register accumulators: per row a = M_x v and b = K_x v (neighbours
// by shuffles), and the outputs y = yp - P .. yp + P receive K_y a + M_y b; an output is
// written when its last input row has passed.  (2 + 2)(2P + 1) FMA per row in all (x 32/(32
// - 2P) for the halo lanes), one load per lane and row.  Stored rows are tasks of 32 rows.
template <typename T, int P, int MODE, bool DOT>
__global__ void __launch_bounds__(TPB) k_apply_ym2d(DevLevelT<T> L, const T* __restrict__ x, const T* rin, T* out,
                                                    T* __restrict__ xs, T gamma, const int* done, double* partial,
                                                    PcgState* st, ZmShape sh) {
    pdl_begin();
    if (done && *done) return;
    constexpr int W = 2 * P + 1, XS = 32 - 2 * P;
    constexpr bool SC = sizeof(T) == 4;              // FP32 path: Jacobi-scaled variables
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int m = L.m;
    double acc = 0.0;
    for (;;) {
        unsigned int t = 0;
        if (lane == 0) t = atomicAdd(&L.tile_ctr[0], 1u);
        t = __shfl_sync(FULL, t, 0);
        if (t >= sh.ntotal) break;
        if (t < sh.ntensor) {
            const int sxi = (int)(t % (unsigned)sh.sx);
            const int syi = (int)(t / (unsigned)sh.sx);
            const int gx = sxi * XS - P + lane;
            const int yc0 = syi * sh.zc;
            const int yend = min(yc0 + sh.zc, m);
            const bool xin = (unsigned)gx < (unsigned)m;
            const bool own = lane >= P && lane < 32 - P && xin;
            T kx[W], mx[W];
#pragma unroll
            for (int o = 0; o < W; ++o) {
                kx[o] = xin ? ro(L.K1 + (int64_t)gx * W + o) : T(0);
                mx[o] = xin ? ro(L.M1 + (int64_t)gx * W + o) : T(0);
            }
            bool symx = true;
#pragma unroll
            for (int o = 0; o < P; ++o) symx = symx && kx[o] == kx[2 * P - o] && mx[o] == mx[2 * P - o];
            symx = __all_sync(FULL, symx);
            T ring[W];
#pragma unroll
            for (int q = 0; q < W; ++q) ring[q] = T(0);
            const int nrows = (yend - yc0) + 2 * P;
            auto load_row = [&](int yp) -> T {
                const bool in = xin && (unsigned)yp < (unsigned)m;
                const int64_t g = (int64_t)yp * m + gx;
                return in ? (SC ? x[g] * ro(L.s + g) : x[g]) : T(0);
            };
            T v = load_row(yc0 - P);
            for (int base = 0; base < nrows; base += W) {
#pragma unroll
                for (int u = 0; u < W; ++u) {
                    const int k = base + u;
                    if (k >= nrows) break;
                    const int yp = yc0 - P + k;
                    const T vn = (k + 1 < nrows) ? load_row(yp + 1) : T(0);
                    T aa, bb;
                    if (symx) {
                        aa = mx[P] * v;
                        bb = kx[P] * v;
#pragma unroll
                        for (int o = 0; o < P; ++o) {
                            const T sv = __shfl_sync(FULL, v, (lane - P + o) & 31) +
                                         __shfl_sync(FULL, v, (lane + P - o) & 31);
                            aa = fmaT(mx[o], sv, aa);
                            bb = fmaT(kx[o], sv, bb);
                        }
                    } else {
                        aa = T(0);
                        bb = T(0);
#pragma unroll
                        for (int o = 0; o < W; ++o) {
                            const T vo = __shfl_sync(FULL, v, (lane - P + o) & 31);
                            aa = fmaT(mx[o], vo, aa);
                            bb = fmaT(kx[o], vo, bb);
                        }
                    }
                    // outputs y = yp - P + jy receive K_y[y][2P - jy] a + M_y[y][2P - jy] b; output y
                    // keeps ring slot (y - yc0 + 2P + 1) mod W, here (u + 1 + jy) mod W
#pragma unroll
                    for (int jy = 0; jy < W; ++jy) {
                        const int y = yp - P + jy;
                        if ((unsigned)y < (unsigned)m) {
                            T& r = ring[(u + 1 + jy) % W];
                            r = fmaT(ro(L.K1 + (int64_t)y * W + (2 * P - jy)), aa, r);
                            r = fmaT(ro(L.M1 + (int64_t)y * W + (2 * P - jy)), bb, r);
                        }
                    }
                    const int yo = yp - P;
                    T& r = ring[(u + 1) % W];
                    if (own && yo >= yc0 && yo < yend) {
                        const int64_t oi = (int64_t)yo * m + gx;
                        const int ri = L.rowinfo[oi];
                        if (ri < 0) {
                            T y = T(0);
                            if (ri == -1) y = SC ? r * ro(L.s + oi) : r;
                            if (MODE == APPLY) {
                                out[oi] = y;
                            } else {
                                const T rr = (ri == -2) ? T(0) : rin[oi] - y;
                                out[oi] = rr;
                                if (MODE == RESID_SMOOTH && ri == -1) xs[oi] = fmaT(gamma * ro(L.dinv + oi), rr, xs[oi]);
                            }
                            if (DOT && ri == -1) acc = fma((double)x[oi], (double)y, acc);
                        }
                    }
                    r = T(0);
                    v = vn;
                }
            }
        } else {
            // stored rows: 32 consecutive stored row ids, one per lane
            const int64_t k = (int64_t)(t - sh.ntensor) * 32 + lane;
            if (k < L.nb) {
                const int64_t oi = L.band_row[k];
                const int ix = (int)(oi % m), iy = (int)(oi / m);
                const T* __restrict__ c = L.band_coef + k;
                const int64_t nb = L.nb;
                T y = T(0);
#pragma unroll
                for (int oy = 0; oy < W; ++oy) {
                    const bool yin = (unsigned)(iy + oy - P) < (unsigned)m;
#pragma unroll
                    for (int ox = 0; ox < W; ++ox) {
                        const bool in = yin && (unsigned)(ix + ox - P) < (unsigned)m;
                        const int64_t g = oi + (ox - P) + (int64_t)(oy - P) * m;
                        y = fmaT(ro(c + (int64_t)(ox + W * oy) * nb), in ? x[g] : T(0), y);
                    }
                }
                if (MODE == APPLY) {
                    out[oi] = y;
                } else {
                    const T rr = rin[oi] - y;
                    out[oi] = rr;
                    if (MODE == RESID_SMOOTH) xs[oi] = fmaT(gamma * ro(L.dinv + oi), rr, xs[oi]);
                }
                if (DOT) acc = fma((double)x[oi], (double)y, acc);
            }
        }
    }
    if (lane == 0 && atomicAdd(&L.tile_ctr[1], 1u) == gridDim.x * (TPB / 32) - 1) {
        L.tile_ctr[0] = 0u;
        L.tile_ctr[1] = 0u;
    }
    if (DOT) {
        double pq;
        if (finish_reduction(acc, partial, &st->ticket[0], &pq) && threadIdx.x == 0) {
            st->pq = pq;
            if (!(pq > 0.0) || !isfinite(pq)) {
                st->done = 1;
                st->status = -5;
                st->alpha = 0.0;
            } else {
                st->alpha = st->rz / pq;
            }
        }
    }
}

template <int DIM, int P>
__global__ void __launch_bounds__(TPB) k_apply_pq(DevLevel L, const double* __restrict__ p, double* __restrict__ q,
                                                  double* partial, PcgState* st) {
    pdl_begin();
    if (st->done) return;
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * TPB;
    for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < L.N; i += stride) {
        const double ax = row_apply<double, DIM, P>(L, i, p);
        q[i] = ax;
        acc = fma(p[i], ax, acc);
    }
    double pq;
    if (finish_reduction(acc, partial, &st->ticket[0], &pq) && threadIdx.x == 0) {
        st->pq = pq;
        if (!(pq > 0.0) || !isfinite(pq)) {
            st->done = 1;
            st->status = -5;
            st->alpha = 0.0;
        } else {
            st->alpha = st->rz / pq;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_scale_diag(int64_t N, const T* __restrict__ dinv, const T* __restrict__ r,
                                                    T* __restrict__ x, T gamma, const int* done) {
    pdl_begin();
    if (done && *done) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) x[i] = gamma * dinv[i] * r[i];
}

// one warp per stored block of [b_first, b_end): gather r_j, z_j = A_j^{-1} r_j,
// x[idx_j] += gamma z_j
template <typename T>
__device__ __forceinline__ void blocks_warps(const DevLevelT<T>& L, const T* __restrict__ r, T* x, T gamma,
                                             int64_t b_first, int64_t b_end, int64_t warp0, int64_t nwarps, int lane,
                                             T* rs) {
    for (int64_t b = b_first + warp0; b < b_end; b += nwarps) {
        const int64_t s = ro(L.blk_ptr + b);
        const int nj = (int)(ro(L.blk_ptr + b + 1) - s);
        const T* __restrict__ A = L.blk_val + ro(L.blk_vptr + b);
        for (int a = lane; a < nj; a += 32) rs[a] = r[ro(L.blk_idx + s + a)];
        __syncwarp();
        for (int a = lane; a < nj; a += 32) {
            T acc = T(0);
            for (int c = 0; c < nj; ++c) acc = fmaT(ro(A + (int64_t)c * nj + a), rs[c], acc);
            atomicAdd(&x[ro(L.blk_idx + s + a)], gamma * acc);
        }
        __syncwarp();
    }
}

// Additive Schwarz, stored blocks (Eq. applyCS): x_i += gamma (A_j^{-1} r_j)_a for every
// (block j, function i = idx_j[a]) pair, one thread per pair: the pair's row of the
// inverse against the block's gathered residual, then one atomic add.  Blocks on the cut
// band hold a few functions each (about 3 on average at the 3-D workloads), so a thread
// per pair keeps every lane busy where a warp per block would leave most of them idle.
template <typename T>
__global__ void __launch_bounds__(TPB) k_blocks_pairs(DevLevelT<T> L, int64_t npairs, const T* __restrict__ r, T* x,
                                                      T gamma, const int* done) {
    pdl_begin();
    if (done && *done) return;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < npairs; q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = ro(L.blk_of + q);
        const int64_t s = ro(L.blk_ptr + b);
        const int nj = (int)(ro(L.blk_ptr + b + 1) - s);
        const int a = (int)(q - s);
        const T* __restrict__ A = L.blk_val + ro(L.blk_vptr + b) + a;
        T acc = T(0);
        for (int c = 0; c < nj; ++c) acc = fmaT(ro(A + (int64_t)c * nj), r[ro(L.blk_idx + s + c)], acc);
        atomicAdd(&x[ro(L.blk_idx + q)], gamma * acc);
    }
}

// One colour of the multiplicative Schwarz sweep (Sec. 3.4): x += sum_{j of colour c}
// P_j A_j^{-1} P_j^T r.  The first ceil(ns/32) warps take the one-function blocks
// (x_i += r_i / A_ii, one per thread), the others one stored block each.  Blocks of one
// colour share no function, so no two threads write the same entry of x.
template <typename T>
__global__ void __launch_bounds__(TPB) k_colour_smooth(DevLevelT<T> L, int64_t b_first, int64_t b_end,
                                                       const int32_t* __restrict__ sg_row,
                                                       const T* __restrict__ sg_inv, int64_t ns,
                                                       const T* __restrict__ r, T* x, const int* done) {
    pdl_begin();
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    if (done && *done) return;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t wsg = (ns + 31) >> 5;
    const int64_t w = gt >> 5;
    if (w < wsg) {                 // warp-uniform branch
        if (gt < ns) {
            const int32_t i = ro(sg_row + gt);
            x[i] += ro(sg_inv + gt) * r[i];
        }
        return;
    }
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    blocks_warps<T>(L, r, x, T(1), b_first, b_end, w - wsg, ((int64_t)gridDim.x * blockDim.x >> 5) - wsg, lane,
                    sm + (int64_t)wib * L.max_block);
}

// fine level in type TF, coarse level in type TC (equal, or FP64 fine and FP32 coarse in
// the V-cycle whose finest level is FP64); sums in TF
template <typename TF, typename TC, int DIM, int P>
__device__ __forceinline__ void restrict_rows(const DevLevelT<TF>& F, const DevLevelT<TC>& C, const TF* __restrict__ rf,
                                              TC* __restrict__ rc, TC* __restrict__ xc, TC gamma, int64_t start,
                                              int64_t stride) {
    using T = TF;
    constexpr int P2 = P + 2;
    const int mc = C.m, mf = F.m;
    const T* __restrict__ df = F.d;      // fine scale d (FP32 path) or nullptr
    for (int64_t i = start; i < C.N; i += stride) {
        // the row's activity is applied at the end, so that its load overlaps the others
        const bool inactive = C.rowinfo[i] == -2;
        const int cx = (int)(i % mc), cy = (int)((i / mc) % mc), cz = (DIM == 3) ? (int)(i / ((int64_t)mc * mc)) : 0;
        const int fx = ro(F.r_first + cx), fy = ro(F.r_first + cy), fz = (DIM == 3) ? ro(F.r_first + cz) : 0;
        const T* wx = F.r_w + (int64_t)cx * P2;
        const T* wy = F.r_w + (int64_t)cy * P2;
        const T* wz = F.r_w + (int64_t)cz * P2;
        T s = T(0);
#pragma unroll
        for (int kz = 0; kz < (DIM == 3 ? P2 : 1); ++kz) {
            const T wzk = (DIM == 3) ? ro(wz + kz) : T(1);
#pragma unroll
            for (int ky = 0; ky < P2; ++ky) {
                const T wyz = ro(wy + ky) * wzk;
                const int64_t rb = (int64_t)(fx) + (int64_t)mf * ((fy + ky) + (DIM == 3 ? (int64_t)mf * (fz + kz) : 0));
                T t = T(0);
#pragma unroll
                for (int kx = 0; kx < P2; ++kx) t = fmaT(ro(wx + kx), df ? rf[rb + kx] * ro(df + rb + kx) : rf[rb + kx], t);
                s = fmaT(wyz, t, s);
            }
        }
        if (C.s) s *= (T)ro(C.s + i);
        if (inactive) s = T(0);
        const TC sc = (TC)s;
        rc[i] = sc;
        if (xc) xc[i] = gamma * ro(C.dinv + i) * sc;
    }
}

template <typename TF, typename TC, int DIM, int P>
__global__ void __launch_bounds__(TPB) k_restrict(DevLevelT<TF> F, DevLevelT<TC> C, const TF* __restrict__ rf,
                                                  TC* __restrict__ rc, TC* __restrict__ xc, TC gamma, const int* done) {
    pdl_begin();
    if (done && *done) return;
    restrict_rows<TF, TC, DIM, P>(F, C, rf, rc, xc, gamma, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                                  (int64_t)gridDim.x * blockDim.x);
}

// fine level in type TF, coarse in TC (see restrict_rows); sums in TF
template <typename TF, typename TC, int DIM, int P>
__device__ __forceinline__ void prolong_rows(const DevLevelT<TF>& F, const DevLevelT<TC>& C, const TC* __restrict__ xc,
                                             TF* __restrict__ e, TF* __restrict__ x, int64_t start, int64_t stride) {
    using T = TF;
    const int mc = C.m, mf = F.m, TW = F.TW;
    const TC* __restrict__ sc = C.s;     // coarse scale 1/d (FP32 path) or nullptr
    for (int64_t a = start; a < F.N; a += stride) {
        const bool inactive = F.rowinfo[a] == -2;    // applied at the end (overlapping loads)
        const int ax = (int)(a % mf), ay = (int)((a / mf) % mf), az = (DIM == 3) ? (int)(a / ((int64_t)mf * mf)) : 0;
        const int cx = ro(F.t_first + ax), cy = ro(F.t_first + ay), cz = (DIM == 3) ? ro(F.t_first + az) : 0;
        const T* wx = F.t_w + (int64_t)ax * TW;
        const T* wy = F.t_w + (int64_t)ay * TW;
        const T* wz = F.t_w + (int64_t)az * TW;
        T s = T(0);
        for (int tz = 0; tz < (DIM == 3 ? TW : 1); ++tz) {
            const T wzk = (DIM == 3) ? ro(wz + tz) : T(1);
            for (int ty = 0; ty < TW; ++ty) {
                const T wyz = ro(wy + ty) * wzk;
                const int64_t rb = (int64_t)cx + (int64_t)mc * ((cy + ty) + (DIM == 3 ? (int64_t)mc * (cz + tz) : 0));
                T t = T(0);
                for (int tx = 0; tx < TW; ++tx)
                    t = fmaT(ro(wx + tx), (T)(sc ? xc[rb + tx] * ro(sc + rb + tx) : xc[rb + tx]), t);
                s = fmaT(wyz, t, s);
            }
        }
        if (F.d) s *= ro(F.d + a);
        if (inactive) s = T(0);
        e[a] = s;
        if (x && !inactive) x[a] += s;
    }
}

template <typename TF, typename TC, int DIM, int P>
__global__ void __launch_bounds__(TPB) k_prolong(DevLevelT<TF> F, DevLevelT<TC> C, const TC* __restrict__ xc,
                                                 TF* __restrict__ e, TF* __restrict__ x, const int* done) {
    pdl_begin();
    if (done && *done) return;
    prolong_rows<TF, TC, DIM, P>(F, C, xc, e, x, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                                 (int64_t)gridDim.x * blockDim.x);
}

// Sum-factorised 3-D transfers.  R = R_1 (x) R_1 (x) R_1 is applied one direction at a
// time: along the pass's axis every output index o takes sum_k w[o][k] in[first[o] + k]
// (the 1-D two-scale table of the restriction, p + 2 weights per coarse index, or of the
// prolongation, TW per fine index), the other two indices unchanged.  Per fine row that is
// about (p + 2)(1/2 + 1/4 + 1/8) FMA for the restriction and TW (1/4 + 1/2 + 1) for the
// prolongation, against (p + 2)^3 / 8 and TW^3 in the direct kernels, whose loads are also
// (p + 2)^3 or TW^3 gathers per row.  The first pass applies the input's Jacobi scale
// (FP32 V-cycle: fine d before the restriction, coarse s before the prolongation), the last
// the output's scale, the zeros of inactive rows and the fused update (restriction:
// xc = gamma dinv_c rc; prolongation: x += e).
enum XferEpi { XF_MID = 0, XF_RESTRICT = 1, XF_PROLONG = 2 };

template <typename TI, typename TO, typename T, int AXIS, int EPI>
__global__ void __launch_bounds__(TPB) k_xfer_pass(const TI* __restrict__ in, TO* __restrict__ out, int nx, int ny,
                                                   int nz, int n_out, const int32_t* __restrict__ first,
                                                   const T* __restrict__ w, int nt, const TI* __restrict__ pre,
                                                   const TO* __restrict__ post, const int32_t* __restrict__ rowinfo,
                                                   const TO* __restrict__ dinv, TO gamma, TO* __restrict__ upd,
                                                   const int* done) {
    pdl_begin();
    if (done && *done) return;
    // output dims: the input's with the AXIS extent replaced by n_out
    const int ox = AXIS == 0 ? n_out : nx, oy = AXIS == 1 ? n_out : ny, oz = AXIS == 2 ? n_out : nz;
    const int64_t total = (int64_t)ox * oy * oz;
    const int64_t istride = AXIS == 0 ? 1 : (AXIS == 1 ? (int64_t)nx : (int64_t)nx * ny);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % ox);
        const int64_t q = i / ox;
        const int iy = (int)(q % oy), iz = (int)(q / oy);
        const int o = AXIS == 0 ? ix : (AXIS == 1 ? iy : iz);
        const int64_t base = (AXIS == 0 ? 0 : ix) + (AXIS == 1 ? 0 : (int64_t)nx * iy) +
                             (AXIS == 2 ? 0 : (int64_t)nx * ny * iz);
        const int64_t src0 = base + (int64_t)ro(first + o) * istride;
        const T* __restrict__ wo = w + (int64_t)o * nt;
        T acc = T(0);
#pragma unroll 4
        for (int k = 0; k < nt; ++k) {
            const int64_t src = src0 + (int64_t)k * istride;
            const T v = pre ? (T)in[src] * (T)ro(pre + src) : (T)in[src];
            acc = fmaT(ro(wo + k), v, acc);
        }
        if (EPI == XF_MID) {
            out[i] = (TO)acc;
        } else {
            if (post) acc *= (T)ro(post + i);
            const bool inactive = rowinfo[i] == -2;
            const TO v = inactive ? TO(0) : (TO)acc;
            out[i] = v;
            if (EPI == XF_RESTRICT && upd) upd[i] = gamma * ro(dinv + i) * v;
            if (EPI == XF_PROLONG && upd && !inactive) upd[i] += v;
        }
    }
}

// one warp per kept coarse row
template <typename T>
__device__ __forceinline__ void coarse_warps(const int32_t* __restrict__ rows, const T* __restrict__ Cinv, int nc,
                                             const T* __restrict__ r, T* __restrict__ x, int64_t warp0, int64_t nwarps,
                                             int lane) {
    for (int64_t a = warp0; a < nc; a += nwarps) {
        const T* row = Cinv + a * nc;
        double acc = 0.0;
        for (int b = lane; b < nc; b += 32) acc = fma((double)ro(row + b), (double)r[ro(rows + b)], acc);
        acc = warp_sum(acc);
        if (lane == 0) x[ro(rows + a)] = (T)acc;
    }
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_coarse(const int32_t* __restrict__ rows, const T* __restrict__ Cinv, int nc,
                                                const T* __restrict__ r, T* __restrict__ x, const int* done) {
    pdl_begin();
    if (done && *done) return;
    coarse_warps<T>(rows, Cinv, nc, r, x, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                    ((int64_t)gridDim.x * blockDim.x) >> 5, threadIdx.x & 31);
}

// V-cycle input from an FP64 residual: r_lo = (TZ)(rs .* r) (or (TZ) r), xv = gamma dinv .* r_lo
template <typename TZ>
__global__ void __launch_bounds__(TPB) k_vcycle_in(int64_t N, const double* __restrict__ r, const TZ* __restrict__ rs,
                                                   const TZ* __restrict__ dinv, TZ gamma, TZ* __restrict__ rlo,
                                                   TZ* __restrict__ xv, const int* done) {
    pdl_begin();
    if (done && *done) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const TZ rv = rs ? (TZ)(r[i] * (double)rs[i]) : (TZ)r[i];
        rlo[i] = rv;
        xv[i] = gamma * dinv[i] * rv;
    }
}

// V-cycle output to FP64: out = zs .* z (or z)
template <typename TZ>
__global__ void __launch_bounds__(TPB) k_vcycle_out(int64_t N, const TZ* __restrict__ z, const TZ* __restrict__ zs,
                                                    double* __restrict__ out) {
    pdl_begin();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        out[i] = zs ? (double)z[i] * (double)zs[i] : (double)z[i];
}

// z as the CG sees it: z_i = zs_i * z^_i in the scaled FP32 path, z_i otherwise
template <typename TZ>
__device__ __forceinline__ double zval(const TZ* z, const TZ* zs, int64_t i) {
    return zs ? (double)z[i] * (double)zs[i] : (double)z[i];
}

template <typename TZ>
__global__ void __launch_bounds__(TPB) k_pcg_update(int64_t N, const TZ* __restrict__ dinv, const TZ* __restrict__ rs,
                                                    double* __restrict__ x, double* __restrict__ r,
                                                    const double* __restrict__ p, const double* __restrict__ q,
                                                    TZ* __restrict__ xv, TZ* __restrict__ rlo, double gamma,
                                                    double* partial, PcgState* st, double* hist) {
    pdl_begin();
    if (st->done) return;
    const double alpha = st->alpha;
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * TPB;
    for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < N; i += stride) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
        // the V-cycle's residual: r itself (FP64) or r^ = s .* r (scaled FP32)
        const TZ rv = rs ? (TZ)(ri * (double)rs[i]) : (TZ)ri;
        if (rlo) rlo[i] = rv;
        xv[i] = (TZ)gamma * dinv[i] * rv;
    }
    double rr;
    if (finish_reduction(acc, partial, &st->ticket[1], &rr) && threadIdx.x == 0) {
        st->rr = rr;
        const int it = ++st->iter;
        if (hist) hist[it] = sqrt(rr / st->bb);
        if (!isfinite(rr)) {
            st->done = 1;
            st->status = -5;
        } else if (rr <= st->tol2 * st->bb) {
            st->done = 1;
            st->status = 0;
        } else if (it >= st->maxit) {
            st->done = 1;
            st->status = 1;
        }
    }
}

// rz_new = r^T z; flexible CG (Polak-Ribiere) also needs r^T z_prev
template <typename TZ>
__global__ void __launch_bounds__(TPB) k_pcg_rz(int64_t N, const double* __restrict__ r, const TZ* __restrict__ z,
                                                const TZ* __restrict__ zs, const TZ* __restrict__ zprev,
                                                double* partial, PcgState* st, const double* __restrict__ qprev) {
    pdl_begin();
    if (st->done) return;
    double acc = 0.0, accp = 0.0;
    const int64_t stride = (int64_t)gridDim.x * TPB;
    for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < N; i += stride) {
        acc = fma(r[i], zval(z, zs, i), acc);
        if (zprev) accp = fma(r[i], zval(zprev, zs, i), accp);
        else if (qprev) accp = fma(zval(z, zs, i), qprev[i], accp);
    }
    double rz, rzp;
    if (finish_reduction2(acc, accp, partial, &st->ticket[2], &rz, &rzp) && threadIdx.x == 0) {
        const double num = zprev ? rz - rzp : (qprev ? -st->alpha * rzp : rz);
        st->beta = num / st->rz;
        st->rz = rz;
        if (!isfinite(rz)) {
            st->done = 1;
            st->status = -5;
        }
    }
}

template <typename TZ>
__global__ void __launch_bounds__(TPB) k_pcg_xpay(int64_t N, const TZ* __restrict__ z, const TZ* __restrict__ zs,
                                                  double* __restrict__ p, TZ* __restrict__ zprev, PcgState* st) {
    pdl_begin();
    if (st->done) return;
    const double beta = st->beta;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        p[i] = fma(beta, p[i], zval(z, zs, i));
        if (zprev) zprev[i] = z[i];
    }
}

// the sums of NV values over the grid (partials at [k G, (k+1) G)); the last block adds
// each in block order and returns true with the totals in tot[0..NV) (thread 0)
template <int NV>
__device__ __forceinline__ bool finish_reduction_n(const double* v, double* partial, unsigned int* ticket,
                                                   double* tot) {
    __shared__ double ws[32];
    __shared__ bool last;
#pragma unroll 1
    for (int k = 0; k < NV; ++k) {
        const double bs = block_sum(v[k], ws);
        if (threadIdx.x == 0) partial[(int64_t)k * gridDim.x + blockIdx.x] = bs;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll 1
    for (int k = 0; k < NV; ++k) {
        double s = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += TPB) s += ((volatile double*)partial)[(int64_t)k * gridDim.x + b];
        s = block_sum(s, ws);
        if (threadIdx.x == 0) tot[k] = s;
        __syncthreads();
    }
    if (threadIdx.x == 0) *ticket = 0u;
    return true;
}

__global__ void __launch_bounds__(TPB) k_fcg_push_dots(int64_t N, int m, const double* __restrict__ z,
                                                       const double* __restrict__ p, const double* __restrict__ q,
                                                       double* __restrict__ Pring, double* __restrict__ Qring,
                                                       double* partial, PcgState* st) {
    pdl_begin();
    if (st->done) return;
    const int it = st->iter;                      // steps taken, >= 1 here
    const int slot = (it - 1) % m, nv = min(it, m);
    double acc[FCG_MAX];
#pragma unroll
    for (int j = 0; j < FCG_MAX; ++j) acc[j] = 0.0;
    const int64_t stride = (int64_t)gridDim.x * TPB;
    for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < N; i += stride) {
        const double zi = z[i], qi = q[i];
        Pring[(int64_t)slot * N + i] = p[i];
        Qring[(int64_t)slot * N + i] = qi;
#pragma unroll
        for (int j = 0; j < FCG_MAX; ++j)
            if (j < nv) acc[j] = fma(zi, j == slot ? qi : Qring[(int64_t)j * N + i], acc[j]);
    }
    double tot[FCG_MAX];
    if (finish_reduction_n<FCG_MAX>(acc, partial, &st->ticket[2], tot) && threadIdx.x == 0) {
        st->fcg_pq[slot] = st->pq;
        for (int j = 0; j < FCG_MAX; ++j) st->fcg_c[j] = (j < nv && st->fcg_pq[j] > 0.0) ? tot[j] / st->fcg_pq[j] : 0.0;
        if (!isfinite(tot[0])) {
            st->done = 1;
            st->status = -5;
        }
    }
}

__global__ void __launch_bounds__(TPB) k_fcg_dir(int64_t N, int m, const double* __restrict__ z,
                                                 const double* __restrict__ r, double* __restrict__ p,
                                                 const double* __restrict__ Pring, double* partial, PcgState* st) {
    pdl_begin();
    if (st->done) return;
    const int nv = min(st->iter, m);
    double c[FCG_MAX];
#pragma unroll
    for (int j = 0; j < FCG_MAX; ++j) c[j] = st->fcg_c[j];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * TPB;
    for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < N; i += stride) {
        double pi = z[i];
#pragma unroll
        for (int j = 0; j < FCG_MAX; ++j)
            if (j < nv) pi = fma(-c[j], Pring[(int64_t)j * N + i], pi);
        p[i] = pi;
        acc = fma(r[i], pi, acc);
    }
    double rp;
    if (finish_reduction(acc, partial, &st->ticket[2], &rp) && threadIdx.x == 0) {
        st->rz = rp;
        if (!isfinite(rp)) {
            st->done = 1;
            st->status = -5;
        }
    }
}

__global__ void __launch_bounds__(TPB) k_init_norms(int64_t N, const double* __restrict__ r, const double* __restrict__ b,
                                                    double* partial, PcgState* st, double* hist) {
    pdl_begin();
    double a = 0.0, c = 0.0;
    const int64_t stride = (int64_t)gridDim.x * TPB;
    for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < N; i += stride) {
        a = fma(r[i], r[i], a);
        c = fma(b[i], b[i], c);
    }
    double rr, bb;
    if (finish_reduction2(a, c, partial, &st->ticket[3], &rr, &bb) && threadIdx.x == 0) {
        st->rr = rr;
        st->bb = bb;
        st->iter = 0;
        st->status = 0;
        st->done = 0;
        if (hist) hist[0] = (bb > 0.0) ? sqrt(rr / bb) : 0.0;
        if (bb == 0.0 || rr <= st->tol2 * bb) {
            st->done = 1;
        } else if (st->maxit <= 0) {
            st->done = 1;
            st->status = 1;
        }
        if (!isfinite(rr) || !isfinite(bb)) {
            st->done = 1;
            st->status = -5;
        }
    }
}

template <typename TZ>
__global__ void __launch_bounds__(TPB) k_init_dir(int64_t N, const double* __restrict__ r, const TZ* __restrict__ z,
                                                  const TZ* __restrict__ zs, double* __restrict__ p,
                                                  TZ* __restrict__ zprev, double* partial, PcgState* st) {
    pdl_begin();
    if (st->done) return;
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * TPB;
    for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < N; i += stride) {
        const double zi = zval(z, zs, i);
        acc = fma(r[i], zi, acc);
        p[i] = zi;
        if (zprev) zprev[i] = z[i];
    }
    double rz;
    if (finish_reduction(acc, partial, &st->ticket[2], &rz) && threadIdx.x == 0) {
        st->rz = rz;
        if (!(rz > 0.0) || !isfinite(rz)) {
            st->done = 1;
            st->status = -5;
        }
    }
}

__global__ void __launch_bounds__(TPB) k_norm2(int64_t N, const double* __restrict__ v, double* partial, PcgState* st) {
    pdl_begin();
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * TPB;
    for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < N; i += stride) acc = fma(v[i], v[i], acc);
    double t;
    if (finish_reduction(acc, partial, &st->ticket[0], &t) && threadIdx.x == 0) st->true_rr = t;
}

__global__ void k_set_continue(PcgState* st, cudaGraphConditionalHandle handle) {
    pdl_begin();
    cudaGraphSetConditional(handle, st->done ? 0u : 1u);
}

// One row per thread.  Large levels: 256-thread blocks.  Small levels: blocks just big
// enough to give every SM about two of them, so that the work is spread over the whole
// GPU instead of a handful of SMs (FP64 issues 2 FMA/clk per SM).
struct RowLaunch {
    int grid, block;
};
inline RowLaunch row_launch(int64_t n) {
    const int64_t want = 2LL * num_sms();
    int64_t tpb = (n + want - 1) / want;
    tpb = ((tpb + 31) / 32) * 32;
    if (tpb < 32) tpb = 32;
    if (tpb > TPB) tpb = TPB;
    int64_t g = (n + tpb - 1) / tpb;
    if (g < 1) g = 1;
    if (g > 65535LL * 8) g = 65535LL * 8;
    return {(int)g, (int)tpb};
}

inline int tiles_2d(int m) { return ((m + TX - 1) / TX) * ((m + TY - 1) / TY); }
// blocks of a 2-D tile launch: one per tile, except the FP64 operator apply (the CG's A p,
// and the standalone apply), whose two blocks per SM draw tiles from the level's counter.
// In the residual modes of the V-cycle the extra loads per row favour more resident blocks.
template <typename T>
inline int tile_grid(int m, int mode) {
    const int n = tiles_2d(m);
    return (sizeof(T) == 8 && mode == APPLY) ? std::min(n, 2 * num_sms()) : n;
}

// 2-D y-marching apply: strips of 32 - 2P columns x chunks of rows (the autotuner's, else a
// rule like the 3-D one), stored rows in tasks of 32.  Only with IMGM_YM2D=1: on the 512^2
// levels it measures slower than the tile kernel (finest FP64 apply 28.6 against 21.8 us),
// since a 2-D row carries no y pass to save and the short walks are latency-bound.
ZmShape ym_shape(int m, int64_t nb, int P, int zc_set) {
    ZmShape s{};
    const int xs = 32 - 2 * P;
    s.sx = (m + xs - 1) / xs;
    s.sy = 1;
    const int want = (ZM_TASKS + s.sx - 1) / s.sx;
    int zc = std::max(2, std::min(64, (m + want - 1) / want));
    if (zc_set > 0) zc = zc_set;
    const int nz = (m + zc - 1) / zc;
    s.zc = (m + nz - 1) / nz;
    s.sz = (m + s.zc - 1) / s.zc;
    s.ntensor = (unsigned)((int64_t)s.sx * s.sz);
    s.ntotal = s.ntensor + (unsigned)((nb + 31) / 32);
    return s;
}
bool use_ym_2d(int) {
    const char* v = std::getenv("IMGM_YM2D");
    return v && v[0] == '1';
}

template <typename T, int P>
cudaError_t launch_ym2d(const DevLevelT<T>& L, int mode, const T* x, const T* rin, T* out, T* xs, T gamma,
                        const int* done, cudaStream_t s) {
    if (L.tile_ctr == nullptr || (L.nb > 0 && L.band_row == nullptr)) return cudaErrorInvalidValue;
    const ZmShape sh = ym_shape(L.m, L.nb, P, L.zm_zc);
    const int g = zm_grid(sh, 2 * num_sms());
    if (mode == APPLY)
        launch_pdl(k_apply_ym2d<T, P, APPLY, false>, g, TPB, 0, s, L, x, rin, out, xs, gamma, done, nullptr, nullptr, sh);
    else if (mode == RESID)
        launch_pdl(k_apply_ym2d<T, P, RESID, false>, g, TPB, 0, s, L, x, rin, out, xs, gamma, done, nullptr, nullptr, sh);
    else
        launch_pdl(k_apply_ym2d<T, P, RESID_SMOOTH, false>, g, TPB, 0, s, L, x, rin, out, xs, gamma, done, nullptr,
                   nullptr, sh);
    return cudaGetLastError();
}

template <typename T, int P>
cudaError_t launch_tile2d(const DevLevelT<T>& L, int mode, const T* x, const T* rin, T* out, T* xs, T gamma,
                          const int* done, cudaStream_t s) {
    if (sizeof(T) == 8 && L.tile_ctr == nullptr) return cudaErrorInvalidValue;
    const int g = tile_grid<T>(L.m, mode);
    if (mode == APPLY)
        launch_pdl(k_apply_tile2d<T, P, APPLY, false>, g, TPB, 0, s, L, x, rin, out, xs, gamma, done, nullptr, nullptr);
    else if (mode == RESID)
        launch_pdl(k_apply_tile2d<T, P, RESID, false>, g, TPB, 0, s, L, x, rin, out, xs, gamma, done, nullptr, nullptr);
    else
        launch_pdl(k_apply_tile2d<T, P, RESID_SMOOTH, false>, g, TPB, 0, s, L, x, rin, out, xs, gamma, done, nullptr, nullptr);
    return cudaGetLastError();
}

}  // namespace

thread_local bool t_pdl = true;
thread_local int64_t t_launches = 0;   // kernels issued by this host thread

bool ym_applies(int m) { return use_ym_2d(m); }
void set_programmatic_launch(bool on) { t_pdl = on; }
int64_t launch_count() { return t_launches; }
void add_launches(int64_t k) { t_launches += k; }

int reduction_blocks() {
    if (g_red_blocks == 0) g_red_blocks = num_sms() * 4;
    return g_red_blocks;
}

#define IMGM_DISPATCH(DIM_, P_, CALL)                                  \
    do {                                                               \
        if ((DIM_) == 2 && (P_) == 1) { constexpr int D = 2, Q = 1; CALL; } \
        else if ((DIM_) == 2 && (P_) == 2) { constexpr int D = 2, Q = 2; CALL; } \
        else if ((DIM_) == 2 && (P_) == 3) { constexpr int D = 2, Q = 3; CALL; } \
        else if ((DIM_) == 3 && (P_) == 1) { constexpr int D = 3, Q = 1; CALL; } \
        else if ((DIM_) == 3 && (P_) == 2) { constexpr int D = 3, Q = 2; CALL; } \
        else if ((DIM_) == 3 && (P_) == 3) { constexpr int D = 3, Q = 3; CALL; } \
        else return cudaErrorInvalidValue;                             \
    } while (0)

template <typename T>
cudaError_t launch_apply(const DevLevelT<T>& L, int mode, const T* x, const T* rin, T* out, T* xs, double gamma,
                         const int* done, cudaStream_t s) {
    // tiles when there are enough of them to fill the GPU; one row per thread otherwise
    if (L.dim == 3 && zm_applies(L.m)) return apply_zm3d(L, mode, x, rin, out, xs, (T)gamma, done, s);
    if (L.dim == 2 && use_ym_2d(L.m)) {
        if (L.p == 1) return launch_ym2d<T, 1>(L, mode, x, rin, out, xs, (T)gamma, done, s);
        if (L.p == 2) return launch_ym2d<T, 2>(L, mode, x, rin, out, xs, (T)gamma, done, s);
        if (L.p == 3) return launch_ym2d<T, 3>(L, mode, x, rin, out, xs, (T)gamma, done, s);
    }
    if (L.dim == 2 && tiles_2d(L.m) >= num_sms()) {
        if (L.p == 1) return launch_tile2d<T, 1>(L, mode, x, rin, out, xs, (T)gamma, done, s);
        if (L.p == 2) return launch_tile2d<T, 2>(L, mode, x, rin, out, xs, (T)gamma, done, s);
        if (L.p == 3) return launch_tile2d<T, 3>(L, mode, x, rin, out, xs, (T)gamma, done, s);
    }
    const RowLaunch rl = row_launch(L.N);
    IMGM_DISPATCH(L.dim, L.p,
                  (launch_pdl(k_apply<T, D, Q>, rl.grid, rl.block, 0, s, L, mode, x, rin, out, xs, (T)gamma, done)));
    return cudaGetLastError();
}

cudaError_t launch_apply_pq(const DevLevel& L, const double* p, double* q, double* partial, PcgState* st,
                            cudaStream_t s) {
    if (L.dim == 2 && use_ym_2d(L.m)) {
        if (L.tile_ctr == nullptr || (L.nb > 0 && L.band_row == nullptr)) return cudaErrorInvalidValue;
        const ZmShape sh = ym_shape(L.m, L.nb, L.p, L.zm_zc);
        const int g = zm_grid(sh, std::min(2 * num_sms(), reduction_blocks()));
        if (L.p == 1)
            launch_pdl(k_apply_ym2d<double, 1, APPLY, true>, g, TPB, 0, s, L, p, nullptr, q, nullptr, 0.0, &st->done, partial, st, sh);
        else if (L.p == 2)
            launch_pdl(k_apply_ym2d<double, 2, APPLY, true>, g, TPB, 0, s, L, p, nullptr, q, nullptr, 0.0, &st->done, partial, st, sh);
        else if (L.p == 3)
            launch_pdl(k_apply_ym2d<double, 3, APPLY, true>, g, TPB, 0, s, L, p, nullptr, q, nullptr, 0.0, &st->done, partial, st, sh);
        else
            return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
    if (L.dim == 2) {
        if (L.tile_ctr == nullptr) return cudaErrorInvalidValue;
        const int g = std::min(tile_grid<double>(L.m, APPLY), reduction_blocks());
        if (L.p == 1)
            launch_pdl(k_apply_tile2d<double, 1, APPLY, true>, g, TPB, 0, s, L, p, nullptr, q, nullptr, 0.0, &st->done, partial, st);
        else if (L.p == 2)
            launch_pdl(k_apply_tile2d<double, 2, APPLY, true>, g, TPB, 0, s, L, p, nullptr, q, nullptr, 0.0, &st->done, partial, st);
        else if (L.p == 3)
            launch_pdl(k_apply_tile2d<double, 3, APPLY, true>, g, TPB, 0, s, L, p, nullptr, q, nullptr, 0.0, &st->done, partial, st);
        else
            return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
    if (L.dim == 3 && zm_applies(L.m)) return apply_zm3d_pq(L, p, q, partial, st, s);
    IMGM_DISPATCH(L.dim, L.p, (launch_pdl(k_apply_pq<D, Q>, reduction_blocks(), TPB, 0, s, L, p, q, partial, st)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale_diag(const DevLevelT<T>& L, const T* r, T* x, double gamma, const int* done, cudaStream_t s) {
    const RowLaunch rl = row_launch(L.N);
    launch_pdl(k_scale_diag<T>, rl.grid, rl.block, 0, s, L.N, L.dinv, r, x, (T)gamma, done);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_blocks(const DevLevelT<T>& L, const T* r, T* x, double gamma, const int* done, cudaStream_t s) {
    if (L.nblk == 0) return cudaSuccess;
    if (L.blk_of == nullptr || L.npair <= 0) return cudaErrorInvalidValue;
    const RowLaunch rl = row_launch(L.npair);
    launch_pdl(k_blocks_pairs<T>, rl.grid, rl.block, 0, s, L, L.npair, r, x, (T)gamma, done);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_colour_smooth(const DevLevelT<T>& L, int64_t b_first, int64_t b_end, const int32_t* sg_row,
                                 const T* sg_inv, int64_t ns, const T* r, T* x, const int* done, cudaStream_t s) {
    const int64_t nb = b_end - b_first;
    if (nb <= 0 && ns <= 0) return cudaSuccess;
    const int64_t warps = ((ns + 31) >> 5) + std::max<int64_t>(nb, 0);
    const int64_t g = (warps * 32 + TPB - 1) / TPB;
    if (g > 65535LL * 16) return cudaErrorInvalidValue;
    const size_t smem = (size_t)(TPB / 32) * L.max_block * sizeof(T);
    launch_pdl(k_colour_smooth<T>, (unsigned)g, TPB, smem, s, L, b_first, b_end, sg_row, sg_inv, ns, r, x, done);
    return cudaGetLastError();
}

// the three passes of the sum-factorised 3-D restriction (fine type TF, coarse type TC,
// arithmetic in TF): x (fine z, y; coarse x), y, then z into the coarse level
template <typename TF, typename TC>
void restrict_passes(const DevLevelT<TF>& F, const DevLevelT<TC>& C, const TF* rf, TC* rc, TC* xc, double gamma,
                     const int* done, cudaStream_t s) {
    const int mf = F.m, mc = C.m, nt = F.p + 2;
    TF* u1 = reinterpret_cast<TF*>(F.xs1);          // [mf][mf][mc]
    TF* u2 = reinterpret_cast<TF*>(F.xs2);          // [mf][mc][mc]
    const RowLaunch l1 = row_launch((int64_t)mf * mf * mc), l2 = row_launch((int64_t)mf * mc * mc),
                    l3 = row_launch(C.N);
    launch_pdl(k_xfer_pass<TF, TF, TF, 0, XF_MID>, l1.grid, l1.block, 0, s, rf, u1, mf, mf, mf, mc, F.r_first, F.r_w,
               nt, F.d, (const TF*)nullptr, (const int32_t*)nullptr, (const TF*)nullptr, TF(0), (TF*)nullptr, done);
    launch_pdl(k_xfer_pass<TF, TF, TF, 1, XF_MID>, l2.grid, l2.block, 0, s, (const TF*)u1, u2, mc, mf, mf, mc,
               F.r_first, F.r_w, nt, (const TF*)nullptr, (const TF*)nullptr, (const int32_t*)nullptr,
               (const TF*)nullptr, TF(0), (TF*)nullptr, done);
    launch_pdl(k_xfer_pass<TF, TC, TF, 2, XF_RESTRICT>, l3.grid, l3.block, 0, s, (const TF*)u2, rc, mc, mc, mf, mc,
               F.r_first, F.r_w, nt, (const TF*)nullptr, C.s, C.rowinfo, C.dinv, (TC)gamma, xc, done);
}

// the three passes of the sum-factorised 3-D prolongation: x (coarse z, y; fine x), y,
// then z onto the fine level
template <typename TF, typename TC>
void prolong_passes(const DevLevelT<TF>& F, const DevLevelT<TC>& C, const TC* xc, TF* e, TF* x, const int* done,
                    cudaStream_t s) {
    const int mf = F.m, mc = C.m, nt = F.TW;
    TF* v1 = reinterpret_cast<TF*>(F.xs2);          // [mc][mc][mf]
    TF* v2 = reinterpret_cast<TF*>(F.xs1);          // [mc][mf][mf]
    const RowLaunch l1 = row_launch((int64_t)mc * mc * mf), l2 = row_launch((int64_t)mc * mf * mf),
                    l3 = row_launch(F.N);
    launch_pdl(k_xfer_pass<TC, TF, TF, 0, XF_MID>, l1.grid, l1.block, 0, s, xc, v1, mc, mc, mc, mf, F.t_first, F.t_w,
               nt, C.s, (const TF*)nullptr, (const int32_t*)nullptr, (const TF*)nullptr, TF(0), (TF*)nullptr, done);
    launch_pdl(k_xfer_pass<TF, TF, TF, 1, XF_MID>, l2.grid, l2.block, 0, s, (const TF*)v1, v2, mf, mc, mc, mf,
               F.t_first, F.t_w, nt, (const TF*)nullptr, (const TF*)nullptr, (const int32_t*)nullptr,
               (const TF*)nullptr, TF(0), (TF*)nullptr, done);
    launch_pdl(k_xfer_pass<TF, TF, TF, 2, XF_PROLONG>, l3.grid, l3.block, 0, s, (const TF*)v2, e, mf, mf, mc, mf,
               F.t_first, F.t_w, nt, (const TF*)nullptr, F.d, F.rowinfo, (const TF*)nullptr, TF(0), x, done);
}

template <typename T>
cudaError_t launch_restrict(const DevLevelT<T>& F, const DevLevelT<T>& C, const T* rf, T* rc, T* xc, double gamma,
                            const int* done, cudaStream_t s) {
    if (F.dim == 3 && F.xs1 && F.xs2) {
        restrict_passes<T, T>(F, C, rf, rc, xc, gamma, done, s);
        return cudaGetLastError();
    }
    const RowLaunch rl = row_launch(C.N);
    IMGM_DISPATCH(F.dim, F.p, (launch_pdl(k_restrict<T, T, D, Q>, rl.grid, rl.block, 0, s, F, C, rf, rc, xc, (T)gamma, done)));
    return cudaGetLastError();
}

cudaError_t launch_restrict_64to32(const DevLevel& F, const DevLevelT<float>& C, const double* rf, float* rc, float* xc,
                                   double gamma, cudaStream_t s) {
    const int* done = nullptr;
    if (F.dim == 3 && F.xs1 && F.xs2) {
        restrict_passes<double, float>(F, C, rf, rc, xc, gamma, done, s);
        return cudaGetLastError();
    }
    const RowLaunch rl = row_launch(C.N);
    IMGM_DISPATCH(F.dim, F.p,
                  (launch_pdl(k_restrict<double, float, D, Q>, rl.grid, rl.block, 0, s, F, C, rf, rc, xc, (float)gamma, done)));
    return cudaGetLastError();
}

cudaError_t launch_prolong_32to64(const DevLevel& F, const DevLevelT<float>& C, const float* xc, double* e, double* x,
                                  cudaStream_t s) {
    const RowLaunch rl = row_launch(F.N);
    const int* done = nullptr;
    IMGM_DISPATCH(F.dim, F.p, (launch_pdl(k_prolong<double, float, D, Q>, rl.grid, rl.block, 0, s, F, C, xc, e, x, done)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong(const DevLevelT<T>& F, const DevLevelT<T>& C, const T* xc, T* e, T* x, const int* done,
                           cudaStream_t s) {
    if (F.dim == 3 && F.xs1 && F.xs2) {
        prolong_passes<T, T>(F, C, xc, e, x, done, s);
        return cudaGetLastError();
    }
    const RowLaunch rl = row_launch(F.N);
    IMGM_DISPATCH(F.dim, F.p, (launch_pdl(k_prolong<T, T, D, Q>, rl.grid, rl.block, 0, s, F, C, xc, e, x, done)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse(const int32_t* rows, const T* Cinv, int nc, const T* r, T* x, const int* done,
                          cudaStream_t s) {
    if (nc == 0) return cudaSuccess;
    const int warps = 2;
    launch_pdl(k_coarse<T>, (nc + warps - 1) / warps, 32 * warps, 0, s, rows, Cinv, nc, r, x, done);
    return cudaGetLastError();
}



template <typename TZ>
cudaError_t launch_vcycle_in(int64_t N, const double* r, const TZ* rs, const TZ* dinv, double gamma, TZ* r_lo, TZ* xv,
                             const int* done, cudaStream_t s) {
    const RowLaunch rl = row_launch(N);
    launch_pdl(k_vcycle_in<TZ>, rl.grid, rl.block, 0, s, N, r, rs, dinv, (TZ)gamma, r_lo, xv, done);
    return cudaGetLastError();
}

template <typename TZ>
cudaError_t launch_vcycle_out(int64_t N, const TZ* z, const TZ* zs, double* out, cudaStream_t s) {
    const RowLaunch rl = row_launch(N);
    launch_pdl(k_vcycle_out<TZ>, rl.grid, rl.block, 0, s, N, z, zs, out);
    return cudaGetLastError();
}

template <typename TZ>
cudaError_t launch_pcg_update(const DevLevel& L, const TZ* dinv_z, double* x, double* r, const double* p,
                              const double* q, TZ* xv, TZ* r_lo, const TZ* rs, double gamma, double* partial,
                              PcgState* st, double* hist, cudaStream_t s) {
    launch_pdl(k_pcg_update<TZ>, reduction_blocks(), TPB, 0, s, L.N, dinv_z, rs, x, r, p, q, xv, r_lo, gamma, partial, st, hist);
    return cudaGetLastError();
}

template <typename TZ>
cudaError_t launch_pcg_rz(int64_t N, const double* r, const TZ* z, const TZ* zs, const TZ* zprev, double* partial,
                          PcgState* st, cudaStream_t s, const double* qprev) {
    launch_pdl(k_pcg_rz<TZ>, reduction_blocks(), TPB, 0, s, N, r, z, zs, zprev, partial, st, qprev);
    return cudaGetLastError();
}

cudaError_t launch_fcg_push_dots(int64_t N, int m, const double* z, const double* p, const double* q, double* Pring,
                                 double* Qring, double* partial, PcgState* st, cudaStream_t s) {
    if (m < 1 || m > FCG_MAX) return cudaErrorInvalidValue;
    launch_pdl(k_fcg_push_dots, reduction_blocks(), TPB, 0, s, N, m, z, p, q, Pring, Qring, partial, st);
    return cudaGetLastError();
}

cudaError_t launch_fcg_dir(int64_t N, int m, const double* z, const double* r, double* p, const double* Pring,
                           double* partial, PcgState* st, cudaStream_t s) {
    if (m < 1 || m > FCG_MAX) return cudaErrorInvalidValue;
    launch_pdl(k_fcg_dir, reduction_blocks(), TPB, 0, s, N, m, z, r, p, Pring, partial, st);
    return cudaGetLastError();
}

template <typename TZ>
cudaError_t launch_pcg_xpay(int64_t N, const TZ* z, const TZ* zs, double* p, TZ* zprev, PcgState* st,
                            cudaStream_t s) {
    const RowLaunch rl = row_launch(N);
    launch_pdl(k_pcg_xpay<TZ>, rl.grid, rl.block, 0, s, N, z, zs, p, zprev, st);
    return cudaGetLastError();
}

cudaError_t launch_pcg_init_norms(int64_t N, const double* r, const double* b, double* partial, PcgState* st,
                                  double* hist, cudaStream_t s) {
    launch_pdl(k_init_norms, reduction_blocks(), TPB, 0, s, N, r, b, partial, st, hist);
    return cudaGetLastError();
}

template <typename TZ>
cudaError_t launch_pcg_init_dir(int64_t N, const double* r, const TZ* z, const TZ* zs, double* p, TZ* zprev,
                                double* partial, PcgState* st, cudaStream_t s) {
    launch_pdl(k_init_dir<TZ>, reduction_blocks(), TPB, 0, s, N, r, z, zs, p, zprev, partial, st);
    return cudaGetLastError();
}

cudaError_t launch_true_residual_norm(int64_t N, const double* v, double* partial, PcgState* st, cudaStream_t s) {
    launch_pdl(k_norm2, reduction_blocks(), TPB, 0, s, N, v, partial, st);
    return cudaGetLastError();
}

cudaError_t launch_set_continue(PcgState* st, unsigned long long handle, cudaStream_t s) {
    launch_pdl(k_set_continue, 1, 1, 0, s, st, (cudaGraphConditionalHandle)handle);
    return cudaGetLastError();
}

// explicit instantiations: FP64 path and mixed-precision (FP32) V-cycle
#define IMGM_INST(T)                                                                                              \
    template cudaError_t launch_apply<T>(const DevLevelT<T>&, int, const T*, const T*, T*, T*, double, const int*, \
                                         cudaStream_t);                                                            \
    template cudaError_t launch_scale_diag<T>(const DevLevelT<T>&, const T*, T*, double, const int*, cudaStream_t); \
    template cudaError_t launch_blocks<T>(const DevLevelT<T>&, const T*, T*, double, const int*, cudaStream_t);     \
    template cudaError_t launch_colour_smooth<T>(const DevLevelT<T>&, int64_t, int64_t, const int32_t*, const T*,   \
                                                 int64_t, const T*, T*, const int*, cudaStream_t);                 \
    template cudaError_t launch_restrict<T>(const DevLevelT<T>&, const DevLevelT<T>&, const T*, T*, T*, double,     \
                                            const int*, cudaStream_t);                                             \
    template cudaError_t launch_prolong<T>(const DevLevelT<T>&, const DevLevelT<T>&, const T*, T*, T*, const int*,  \
                                           cudaStream_t);                                                          \
    template cudaError_t launch_coarse<T>(const int32_t*, const T*, int, const T*, T*, const int*, cudaStream_t);   \
    template cudaError_t launch_pcg_update<T>(const DevLevel&, const T*, double*, double*, const double*,           \
                                              const double*, T*, T*, const T*, double, double*, PcgState*,          \
                                              double*, cudaStream_t);                                              \
    template cudaError_t launch_pcg_rz<T>(int64_t, const double*, const T*, const T*, const T*, double*, PcgState*, \
                                          cudaStream_t, const double*);                                            \
    template cudaError_t launch_pcg_xpay<T>(int64_t, const T*, const T*, double*, T*, PcgState*, cudaStream_t);     \
    template cudaError_t launch_pcg_init_dir<T>(int64_t, const double*, const T*, const T*, double*, T*, double*,   \
                                                PcgState*, cudaStream_t);                                          \
    template cudaError_t launch_vcycle_in<T>(int64_t, const double*, const T*, const T*, double, T*, T*, const int*, \
                                             cudaStream_t);                                                        \
    template cudaError_t launch_vcycle_out<T>(int64_t, const T*, const T*, double*, cudaStream_t);
IMGM_INST(double)
IMGM_INST(float)

}  // namespace imgm
