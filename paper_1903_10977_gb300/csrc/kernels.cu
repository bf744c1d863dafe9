// FP64 hot-path kernels of the immersed multigrid-preconditioned CG solve.
//
//   operator apply   A_l x            (Eq. systemMulti; Galerkin rows of Remark 3.1)
//   Schwarz smoother gamma M^{-1} r   (Sec. 3.4, additive Schwarz with stored block inverses)
//   restriction      R_l r            (Eq. coarsening)
//   prolongation     R_l^T x          (Sec. 3.3)
//   coarsest solve   A_1^{-1} r       (Algorithm 1, direct solve on level 1)
//   CG updates and dot products       (Sec. 3.2, the V-cycle as CG preconditioner)
//
// Rows of a level are either "tensor" rows, whose whole support lies in full
// elements, where A = K (x) M + M (x) K [+ ...] with the 1-D stiffness/mass rows K1/M1,
// or "stored" rows (support touching a cut, empty or partly active element) whose
// (2p+1)^d coefficients were assembled at setup.  Vectors hold 0 on inactive rows.
// Reductions are deterministic: fixed grid, per-block partials summed in a fixed order
// by the last block to finish.
#include "kernels.cuh"

#include <algorithm>

namespace imgm {
namespace {

constexpr int TPB = 256;
int g_red_blocks = 0;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// sum over the block (result valid in thread 0); blockDim.x == TPB
__device__ __forceinline__ double block_sum(double v, double* ws) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) ws[w] = v;
    __syncthreads();
    v = (threadIdx.x < TPB / 32) ? ws[threadIdx.x] : 0.0;
    if (w == 0) v = warp_sum(v);
    return v;
}

// Writes this block's partial and returns true in the block that finishes last, which
// then holds the sum of all partials (summed in block order) in *total (thread 0).
__device__ __forceinline__ bool finish_reduction(double v, double* partial, unsigned int* ticket, double* total) {
    __shared__ double ws[32];
    __shared__ bool last;
    double bs = block_sum(v, ws);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = bs;
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += TPB) s += ((volatile double*)partial)[b];
    s = block_sum(s, ws);
    if (threadIdx.x == 0) {
        *total = s;
        *ticket = 0u;
    }
    return true;
}

// (A x)_i for one row
template <int DIM, int P>
__device__ __forceinline__ double row_apply(const DevLevel& L, int64_t i, const double* __restrict__ x) {
    constexpr int W = 2 * P + 1;
    const int ri = L.rowinfo[i];
    if (ri == -2) return 0.0;
    const int m = L.m;
    const int ix = (int)(i % m);
    const int iy = (int)((i / m) % m);
    const int iz = (DIM == 3) ? (int)(i / ((int64_t)m * m)) : 0;
    const int64_t sy = m, sz = (int64_t)m * m;
    double y = 0.0;
    if (ri >= 0) {
        const double* __restrict__ c = L.band_coef + ri;
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
                    y = fma(c[(int64_t)ci * nb], x[i + ox + oy * sy + (DIM == 3 ? oz * sz : 0)], y);
                }
            }
        }
        return y;
    }
    const double* __restrict__ Kx = L.K1 + (int64_t)ix * W + P;
    const double* __restrict__ Mx = L.M1 + (int64_t)ix * W + P;
    const double* __restrict__ Ky = L.K1 + (int64_t)iy * W + P;
    const double* __restrict__ My = L.M1 + (int64_t)iy * W + P;
    double kx[W], mx[W];
#pragma unroll
    for (int ox = -P; ox <= P; ++ox) {
        kx[ox + P] = Kx[ox];
        mx[ox + P] = Mx[ox];
    }
    if (DIM == 2) {
#pragma unroll
        for (int oy = -P; oy <= P; ++oy) {
            if ((unsigned)(iy + oy) >= (unsigned)m) continue;
            double a = 0.0, b = 0.0;
            const double* xr = x + i + oy * sy;
#pragma unroll
            for (int ox = -P; ox <= P; ++ox) {
                if ((unsigned)(ix + ox) >= (unsigned)m) continue;
                const double xv = xr[ox];
                a = fma(kx[ox + P], xv, a);
                b = fma(mx[ox + P], xv, b);
            }
            y = fma(My[oy], a, y);
            y = fma(Ky[oy], b, y);
        }
        return y;
    }
    const double* __restrict__ Kz = L.K1 + (int64_t)iz * W + P;
    const double* __restrict__ Mz = L.M1 + (int64_t)iz * W + P;
#pragma unroll
    for (int oz = -P; oz <= P; ++oz) {
        if ((unsigned)(iz + oz) >= (unsigned)m) continue;
        const double mz = Mz[oz], kz = Kz[oz];
#pragma unroll
        for (int oy = -P; oy <= P; ++oy) {
            if ((unsigned)(iy + oy) >= (unsigned)m) continue;
            const double my = My[oy], ky = Ky[oy];
            double a = 0.0, b = 0.0;
            const double* xr = x + i + oy * sy + oz * sz;
#pragma unroll
            for (int ox = -P; ox <= P; ++ox) {
                if ((unsigned)(ix + ox) >= (unsigned)m) continue;
                const double xv = xr[ox];
                a = fma(kx[ox + P], xv, a);
                b = fma(mx[ox + P], xv, b);
            }
            // sum_ox (kx my mz + mx ky mz + mx my kz) x = my mz a + (ky mz + my kz) b
            y = fma(my * mz, a, y);
            y = fma(fma(ky, mz, my * kz), b, y);
        }
    }
    return y;
}

template <int DIM, int P>
__global__ void __launch_bounds__(TPB) k_apply(DevLevel L, int mode, const double* __restrict__ x,
                                               const double* rin, double* out, double* __restrict__ xs,
                                               double gamma, const int* done) {
    if (done && *done) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.N; i += stride) {
        const double ax = row_apply<DIM, P>(L, i, x);
        if (mode == APPLY) {
            out[i] = ax;
        } else {
            const double v = (L.rowinfo[i] == -2) ? 0.0 : rin[i] - ax;
            out[i] = v;
            if (mode == RESID_SMOOTH) xs[i] = fma(gamma * L.dinv[i], v, xs[i]);
        }
    }
}


// ---------------------------------------------------------------------------------
// 2-D operator apply on TX x TY tiles with sum factorisation.  The x values of the tile
// and a p-wide halo are staged in shared memory; the tensor rows then cost
//   u = M_y x, v = K_y x  on the (TX+2p) x TY strip   (2 (2p+1) FMA per point)
//   y = K_x u + M_x v     on the TX x TY outputs      (2 (2p+1) FMA per point)
// i.e. about 4(2p+1) FMA per row instead of 2(2p+1)^2 + 2(2p+1) for the direct sum.
// Stored rows read their (2p+1)^2 coefficients and take x from the same staged tile.
// MODE: APPLY, RESID, RESID_SMOOTH as in k_apply; DOT also accumulates sum_i x_i (A x)_i
// and finishes with alpha = rz / (p^T A p) (the CG step length).
constexpr int TX = 32, TY = 16;

template <int P, int MODE, bool DOT>
__global__ void __launch_bounds__(TPB) k_apply_tile2d(DevLevel L, const double* __restrict__ x,
                                                      const double* rin, double* out, double* __restrict__ xs,
                                                      double gamma, const int* done, double* partial, PcgState* st) {
    constexpr int W = 2 * P + 1;
    constexpr int SX = TX + 2 * P, SY = TY + 2 * P;
    __shared__ double sx[SY][SX];
    __shared__ double su[TY][SX];
    __shared__ double sv[TY][SX];
    if (done && *done) return;
    const int m = L.m;
    const int tiles_x = (m + TX - 1) / TX, tiles_y = (m + TY - 1) / TY;
    const int ntiles = tiles_x * tiles_y;
    double acc = 0.0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
        __syncthreads();   // the previous tile's smem reads are done
        for (int k = threadIdx.x; k < SX * SY; k += TPB) {
            const int ly = k / SX, lx = k % SX;
            const int gx = x0 + lx - P, gy = y0 + ly - P;
            sx[ly][lx] = ((unsigned)gx < (unsigned)m && (unsigned)gy < (unsigned)m) ? x[(int64_t)gy * m + gx] : 0.0;
        }
        __syncthreads();
        // stage 1: along y, for all columns of the strip
        for (int k = threadIdx.x; k < TY * SX; k += TPB) {
            const int ly = k / SX, lx = k % SX;
            const int gy = y0 + ly;
            double u = 0.0, v = 0.0;
            if (gy < m) {
                const double* My = L.M1 + (int64_t)gy * W;
                const double* Ky = L.K1 + (int64_t)gy * W;
#pragma unroll
                for (int o = 0; o < W; ++o) {
                    const double xv = sx[ly + o][lx];
                    u = fma(My[o], xv, u);
                    v = fma(Ky[o], xv, v);
                }
            }
            su[ly][lx] = u;
            sv[ly][lx] = v;
        }
        __syncthreads();
        // stage 2: along x, one output per thread and step
        for (int k = threadIdx.x; k < TX * TY; k += TPB) {
            const int ly = k / TX, lx = k % TX;
            const int gx = x0 + lx, gy = y0 + ly;
            if (gx >= m || gy >= m) continue;
            const int64_t i = (int64_t)gy * m + gx;
            const int ri = L.rowinfo[i];
            double y = 0.0;
            if (ri == -1) {
                const double* Kx = L.K1 + (int64_t)gx * W;
                const double* Mx = L.M1 + (int64_t)gx * W;
#pragma unroll
                for (int o = 0; o < W; ++o) {
                    y = fma(Kx[o], su[ly][lx + o], y);
                    y = fma(Mx[o], sv[ly][lx + o], y);
                }
            } else if (ri >= 0) {
                const double* __restrict__ c = L.band_coef + ri;
                const int64_t nb = L.nb;
#pragma unroll
                for (int oy = 0; oy < W; ++oy)
#pragma unroll
                    for (int ox = 0; ox < W; ++ox) y = fma(c[(int64_t)(ox + W * oy) * nb], sx[ly + oy][lx + ox], y);
            }
            if (MODE == APPLY) {
                out[i] = y;
            } else {
                const double r = (ri == -2) ? 0.0 : rin[i] - y;
                out[i] = r;
                if (MODE == RESID_SMOOTH) xs[i] = fma(gamma * L.dinv[i], r, xs[i]);
            }
            if (DOT) acc = fma(sx[ly + P][lx + P], y, acc);
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

template <int DIM, int P>
__global__ void __launch_bounds__(TPB) k_apply_pq(DevLevel L, const double* __restrict__ p, double* __restrict__ q,
                                                  double* partial, PcgState* st) {
    if (st->done) return;
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * TPB;
    for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < L.N; i += stride) {
        const double ax = row_apply<DIM, P>(L, i, p);
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

__global__ void __launch_bounds__(TPB) k_scale_diag(int64_t N, const double* __restrict__ dinv,
                                                    const double* __restrict__ r, double* __restrict__ x, double gamma,
                                                    const int* done) {
    if (done && *done) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) x[i] = gamma * dinv[i] * r[i];
}

// one warp per stored block: gather r_j, z_j = A_j^{-1} r_j, x[idx_j] += gamma z_j
__global__ void __launch_bounds__(TPB) k_blocks(DevLevel L, const double* __restrict__ r, double* x, double gamma,
                                                const int* done) {
    extern __shared__ double sm[];
    if (done && *done) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double* rs = sm + (int64_t)wib * L.max_block;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); b < L.nblk; b += nwarps) {
        const int64_t s = L.blk_ptr[b];
        const int nj = (int)(L.blk_ptr[b + 1] - s);
        const double* __restrict__ A = L.blk_val + L.blk_vptr[b];
        for (int a = lane; a < nj; a += 32) rs[a] = r[L.blk_idx[s + a]];
        __syncwarp();
        for (int a = lane; a < nj; a += 32) {
            double acc = 0.0;
            for (int c = 0; c < nj; ++c) acc = fma(A[(int64_t)c * nj + a], rs[c], acc);
            atomicAdd(&x[L.blk_idx[s + a]], gamma * acc);
        }
        __syncwarp();
    }
}

template <int DIM, int P>
__global__ void __launch_bounds__(TPB) k_restrict(DevLevel F, DevLevel C, const double* __restrict__ rf,
                                                  double* __restrict__ rc, double* __restrict__ xc, double gamma,
                                                  const int* done) {
    if (done && *done) return;
    constexpr int P2 = P + 2;
    const int mc = C.m, mf = F.m;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < C.N; i += stride) {
        if (C.rowinfo[i] == -2) {
            rc[i] = 0.0;
            if (xc) xc[i] = 0.0;
            continue;
        }
        const int cx = (int)(i % mc), cy = (int)((i / mc) % mc), cz = (DIM == 3) ? (int)(i / ((int64_t)mc * mc)) : 0;
        const int fx = F.r_first[cx], fy = F.r_first[cy], fz = (DIM == 3) ? F.r_first[cz] : 0;
        const double* wx = F.r_w + (int64_t)cx * P2;
        const double* wy = F.r_w + (int64_t)cy * P2;
        const double* wz = F.r_w + (int64_t)cz * P2;
        double s = 0.0;
#pragma unroll
        for (int kz = 0; kz < (DIM == 3 ? P2 : 1); ++kz) {
            const double wzk = (DIM == 3) ? wz[kz] : 1.0;
#pragma unroll
            for (int ky = 0; ky < P2; ++ky) {
                const double wyz = wy[ky] * wzk;
                const double* rr = rf + (int64_t)(fx) + (int64_t)mf * ((fy + ky) + (DIM == 3 ? (int64_t)mf * (fz + kz) : 0));
                double t = 0.0;
#pragma unroll
                for (int kx = 0; kx < P2; ++kx) t = fma(wx[kx], rr[kx], t);
                s = fma(wyz, t, s);
            }
        }
        rc[i] = s;
        if (xc) xc[i] = gamma * C.dinv[i] * s;
    }
}

template <int DIM, int P>
__global__ void __launch_bounds__(TPB) k_prolong(DevLevel F, DevLevel C, const double* __restrict__ xc,
                                                 double* __restrict__ e, double* __restrict__ x, const int* done) {
    if (done && *done) return;
    const int mc = C.m, mf = F.m, TW = F.TW;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < F.N; a += stride) {
        if (F.rowinfo[a] == -2) {
            e[a] = 0.0;
            continue;
        }
        const int ax = (int)(a % mf), ay = (int)((a / mf) % mf), az = (DIM == 3) ? (int)(a / ((int64_t)mf * mf)) : 0;
        const int cx = F.t_first[ax], cy = F.t_first[ay], cz = (DIM == 3) ? F.t_first[az] : 0;
        const double* wx = F.t_w + (int64_t)ax * TW;
        const double* wy = F.t_w + (int64_t)ay * TW;
        const double* wz = F.t_w + (int64_t)az * TW;
        double s = 0.0;
        for (int tz = 0; tz < (DIM == 3 ? TW : 1); ++tz) {
            const double wzk = (DIM == 3) ? wz[tz] : 1.0;
            for (int ty = 0; ty < TW; ++ty) {
                const double wyz = wy[ty] * wzk;
                const double* xr = xc + (int64_t)cx + (int64_t)mc * ((cy + ty) + (DIM == 3 ? (int64_t)mc * (cz + tz) : 0));
                double t = 0.0;
                for (int tx = 0; tx < TW; ++tx) t = fma(wx[tx], xr[tx], t);
                s = fma(wyz, t, s);
            }
        }
        e[a] = s;
        if (x) x[a] += s;
    }
}

// one warp per kept coarse row
__global__ void __launch_bounds__(TPB) k_coarse(const int32_t* __restrict__ rows, const double* __restrict__ Cinv,
                                                int nc, const double* __restrict__ r, double* __restrict__ x,
                                                const int* done) {
    if (done && *done) return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); a < nc; a += nwarps) {
        const double* row = Cinv + a * nc;
        double acc = 0.0;
        for (int b = lane; b < nc; b += 32) acc = fma(row[b], r[rows[b]], acc);
        acc = warp_sum(acc);
        if (lane == 0) x[rows[a]] = acc;
    }
}

__global__ void __launch_bounds__(TPB) k_pcg_update(int64_t N, const double* __restrict__ dinv, double* __restrict__ x,
                                                    double* __restrict__ r, const double* __restrict__ p,
                                                    const double* __restrict__ q, double* __restrict__ xv, double gamma,
                                                    double* partial, PcgState* st, double* hist) {
    if (st->done) return;
    const double alpha = st->alpha;
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * TPB;
    for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < N; i += stride) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
        xv[i] = gamma * dinv[i] * ri;
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

__global__ void __launch_bounds__(TPB) k_pcg_rz(int64_t N, const double* __restrict__ r, const double* __restrict__ z,
                                                double* partial, PcgState* st) {
    if (st->done) return;
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * TPB;
    for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < N; i += stride) acc = fma(r[i], z[i], acc);
    double rz;
    if (finish_reduction(acc, partial, &st->ticket[2], &rz) && threadIdx.x == 0) {
        st->beta = rz / st->rz;
        st->rz = rz;
        if (!isfinite(rz)) {
            st->done = 1;
            st->status = -5;
        }
    }
}

__global__ void __launch_bounds__(TPB) k_pcg_xpay(int64_t N, const double* __restrict__ z, double* __restrict__ p,
                                                  PcgState* st) {
    if (st->done) return;
    const double beta = st->beta;
    const int64_t stride = (int64_t)gridDim.x * TPB;
    for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < N; i += stride) p[i] = fma(beta, p[i], z[i]);
}

__global__ void __launch_bounds__(TPB) k_init_norms(int64_t N, const double* __restrict__ r, const double* __restrict__ b,
                                                    double* partial, PcgState* st, double* hist) {
    __shared__ double ws[32];
    double a = 0.0, c = 0.0;
    const int64_t stride = (int64_t)gridDim.x * TPB;
    for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < N; i += stride) {
        a = fma(r[i], r[i], a);
        c = fma(b[i], b[i], c);
    }
    // two partial arrays: [0, G) for ||r||^2 and [G, 2G) for ||b||^2
    double sb = block_sum(c, ws);
    if (threadIdx.x == 0) partial[gridDim.x + blockIdx.x] = sb;
    double rr;
    if (finish_reduction(a, partial, &st->ticket[3], &rr) && threadIdx.x == 0) {
        double bb = 0.0;
        for (int k = 0; k < (int)gridDim.x; ++k) bb += ((volatile double*)partial)[gridDim.x + k];
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

__global__ void __launch_bounds__(TPB) k_init_dir(int64_t N, const double* __restrict__ r, const double* __restrict__ z,
                                                  double* __restrict__ p, double* partial, PcgState* st) {
    if (st->done) return;
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * TPB;
    for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < N; i += stride) {
        acc = fma(r[i], z[i], acc);
        p[i] = z[i];
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
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * TPB;
    for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < N; i += stride) acc = fma(v[i], v[i], acc);
    double t;
    if (finish_reduction(acc, partial, &st->ticket[0], &t) && threadIdx.x == 0) st->true_rr = t;
}

__global__ void k_set_continue(PcgState* st, cudaGraphConditionalHandle handle) {
    cudaGraphSetConditional(handle, st->done ? 0u : 1u);
}

inline int grid_for(int64_t n) {
    int64_t g = (n + TPB - 1) / TPB;
    if (g < 1) g = 1;
    if (g > 65535LL * 8) g = 65535LL * 8;
    return (int)g;
}

int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    return sms;
}

// One row per thread.  Large levels: 256-thread blocks.  Small levels: blocks just big
// enough to give every SM about two of them, so that FP64 work (2 FMA/clk per SM) is
// spread over the whole GPU instead of a handful of SMs.
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

}  // namespace

int reduction_blocks() {
    if (g_red_blocks == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g_red_blocks = (sms > 0 ? sms : 148) * 4;
    }
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

template <int P>
cudaError_t launch_tile2d(const DevLevel& L, int mode, const double* x, const double* rin, double* out, double* xs,
                          double gamma, const int* done, cudaStream_t s) {
    const int g = tiles_2d(L.m);
    if (mode == APPLY)
        k_apply_tile2d<P, APPLY, false><<<g, TPB, 0, s>>>(L, x, rin, out, xs, gamma, done, nullptr, nullptr);
    else if (mode == RESID)
        k_apply_tile2d<P, RESID, false><<<g, TPB, 0, s>>>(L, x, rin, out, xs, gamma, done, nullptr, nullptr);
    else
        k_apply_tile2d<P, RESID_SMOOTH, false><<<g, TPB, 0, s>>>(L, x, rin, out, xs, gamma, done, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_apply(const DevLevel& L, int mode, const double* x, const double* rin, double* out, double* xs,
                         double gamma, const int* done, cudaStream_t s) {
    // tiles when there are enough of them to fill the GPU; one row per thread otherwise
    if (L.dim == 2 && tiles_2d(L.m) >= num_sms()) {
        if (L.p == 1) return launch_tile2d<1>(L, mode, x, rin, out, xs, gamma, done, s);
        if (L.p == 2) return launch_tile2d<2>(L, mode, x, rin, out, xs, gamma, done, s);
        if (L.p == 3) return launch_tile2d<3>(L, mode, x, rin, out, xs, gamma, done, s);
    }
    const RowLaunch rl = row_launch(L.N);
    IMGM_DISPATCH(L.dim, L.p, (k_apply<D, Q><<<rl.grid, rl.block, 0, s>>>(L, mode, x, rin, out, xs, gamma, done)));
    return cudaGetLastError();
}

cudaError_t launch_apply_pq(const DevLevel& L, const double* p, double* q, double* partial, PcgState* st,
                            cudaStream_t s) {
    if (L.dim == 2) {
        const int g = std::min(tiles_2d(L.m), reduction_blocks());
        if (L.p == 1) k_apply_tile2d<1, APPLY, true><<<g, TPB, 0, s>>>(L, p, nullptr, q, nullptr, 0.0, &st->done, partial, st);
        else if (L.p == 2) k_apply_tile2d<2, APPLY, true><<<g, TPB, 0, s>>>(L, p, nullptr, q, nullptr, 0.0, &st->done, partial, st);
        else if (L.p == 3) k_apply_tile2d<3, APPLY, true><<<g, TPB, 0, s>>>(L, p, nullptr, q, nullptr, 0.0, &st->done, partial, st);
        else return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
    IMGM_DISPATCH(L.dim, L.p, (k_apply_pq<D, Q><<<reduction_blocks(), TPB, 0, s>>>(L, p, q, partial, st)));
    return cudaGetLastError();
}

cudaError_t launch_scale_diag(const DevLevel& L, const double* r, double* x, double gamma, const int* done,
                              cudaStream_t s) {
    const RowLaunch rl = row_launch(L.N);
    k_scale_diag<<<rl.grid, rl.block, 0, s>>>(L.N, L.dinv, r, x, gamma, done);
    return cudaGetLastError();
}

cudaError_t launch_blocks(const DevLevel& L, const double* r, double* x, double gamma, const int* done,
                          cudaStream_t s) {
    if (L.nblk == 0) return cudaSuccess;
    const int warps = 2;                        // small blocks: spread the FP64 work over all SMs
    int64_t g = (L.nblk + warps - 1) / warps;
    if (g > 65535) g = 65535;
    size_t smem = (size_t)warps * L.max_block * sizeof(double);
    k_blocks<<<(int)g, 32 * warps, smem, s>>>(L, r, x, gamma, done);
    return cudaGetLastError();
}

cudaError_t launch_restrict(const DevLevel& F, const DevLevel& C, const double* rf, double* rc, double* xc,
                            double gamma, const int* done, cudaStream_t s) {
    const RowLaunch rl = row_launch(C.N);
    IMGM_DISPATCH(F.dim, F.p, (k_restrict<D, Q><<<rl.grid, rl.block, 0, s>>>(F, C, rf, rc, xc, gamma, done)));
    return cudaGetLastError();
}

cudaError_t launch_prolong(const DevLevel& F, const DevLevel& C, const double* xc, double* e, double* x,
                           const int* done, cudaStream_t s) {
    const RowLaunch rl = row_launch(F.N);
    IMGM_DISPATCH(F.dim, F.p, (k_prolong<D, Q><<<rl.grid, rl.block, 0, s>>>(F, C, xc, e, x, done)));
    return cudaGetLastError();
}

cudaError_t launch_coarse(const int32_t* rows, const double* Cinv, int nc, const double* r, double* x,
                          const int* done, cudaStream_t s) {
    if (nc == 0) return cudaSuccess;
    const int warps = 2;
    k_coarse<<<(nc + warps - 1) / warps, 32 * warps, 0, s>>>(rows, Cinv, nc, r, x, done);
    return cudaGetLastError();
}

cudaError_t launch_pcg_update(const DevLevel& L, double* x, double* r, const double* p, const double* q, double* xv,
                              double gamma, double* partial, PcgState* st, double* hist, cudaStream_t s) {
    k_pcg_update<<<reduction_blocks(), TPB, 0, s>>>(L.N, L.dinv, x, r, p, q, xv, gamma, partial, st, hist);
    return cudaGetLastError();
}

cudaError_t launch_pcg_rz(int64_t N, const double* r, const double* z, double* partial, PcgState* st, cudaStream_t s) {
    k_pcg_rz<<<reduction_blocks(), TPB, 0, s>>>(N, r, z, partial, st);
    return cudaGetLastError();
}

cudaError_t launch_pcg_xpay(int64_t N, const double* z, double* p, PcgState* st, cudaStream_t s) {
    k_pcg_xpay<<<grid_for(N), TPB, 0, s>>>(N, z, p, st);
    return cudaGetLastError();
}

cudaError_t launch_pcg_init_norms(int64_t N, const double* r, const double* b, double* partial, PcgState* st,
                                  double* hist, cudaStream_t s) {
    k_init_norms<<<reduction_blocks(), TPB, 0, s>>>(N, r, b, partial, st, hist);
    return cudaGetLastError();
}

cudaError_t launch_pcg_init_dir(int64_t N, const double* r, const double* z, double* p, double* partial,
                                PcgState* st, cudaStream_t s) {
    k_init_dir<<<reduction_blocks(), TPB, 0, s>>>(N, r, z, p, partial, st);
    return cudaGetLastError();
}

cudaError_t launch_true_residual_norm(int64_t N, const double* v, double* partial, PcgState* st, cudaStream_t s) {
    k_norm2<<<reduction_blocks(), TPB, 0, s>>>(N, v, partial, st);
    return cudaGetLastError();
}

cudaError_t launch_set_continue(PcgState* st, unsigned long long handle, cudaStream_t s) {
    k_set_continue<<<1, 1, 0, s>>>(st, (cudaGraphConditionalHandle)handle);
    return cudaGetLastError();
}

}  // namespace imgm
