// The 3-D z-marching operator apply (kernels and launchers), instantiated for FP64 in
// apply3d_f64.cu and for FP32 in apply3d_f32.cu.
#pragma once
#include "common.cuh"

namespace imgm {
namespace {

// ---------------------------------------------------------------------------------
// 3-D operator apply by z-marching warps.  A warp owns a column of outputs: 32 - 2P
// consecutive x positions (its lanes, plus P halo lanes on each side), YT (1 or 2) consecutive
// y rows and a chunk of z planes, and walks the input planes z' of that chunk (with a
// P-plane halo at each end).  For each plane every lane loads its x-column segment of
// YT + 2P values and forms, for its own YT rows,
//   m = M_y v, k = K_y v                              (along y, in registers)
//   a = M_x m, b = M_x k + K_x m                       (along x, neighbours by shuffles)
// which are the plane's (M_y M_x) and (K_y M_x + M_y K_x) images; an output at plane z then
// collects  y_z = sum_o K_z[z][o] a(z - P + o) + M_z[z][o] b(z - P + o)  in a ring of
// 2P + 1 register accumulators, and is written when its last plane has passed.  That is
// 2(2P+1) + 3(2P+1) FMA per row in the plane (times 32/(32-2P) for the halo lanes) plus
// 2(2P+1) along z: about 39 FMA per row for P = 2, with no shared memory and no block
// barrier.  Stored rows are not formed here: the same launch runs them as tasks of 32
// stored rows (one per lane, (2P+1)^3 coefficients each), so no warp of the tensor tasks
// waits on a lane with a stored row.  Warps draw tasks (tensor tasks first) from the
// level's counter; the last warp to finish re-arms it.  Modes as k_apply_tile2d.
// output rows (y) per lane: a template parameter of the kernel (1 or 2), chosen per level

// FP32 marching applies: the output row's table entry, Jacobi scale and input residual,
// loaded at the start of the step that writes the row, so that these DRAM reads travel together
// and their latency overlaps the step's plane arithmetic (read after it, behind the table entry,
// they were two dependent DRAM round trips per step; the smoothing's diagonal and iterate stay
// at the end, where keeping them across the step would spill registers).  ri = 0 (the id of a
// stored row, written by the stored-row tasks) where the lane writes nothing.
template <typename T, int MODE>
struct OutRow {
    int ri;
    T s, rin;
    __device__ __forceinline__ void load(const DevLevelT<T>& L, const T* rin_, bool w, int64_t oi) {
        ri = w ? L.rowinfo[oi] : 0;
        s = w ? ro(L.s + oi) : T(0);
        rin = (MODE != APPLY && w) ? rin_[oi] : T(0);
    }
    // the row's output from its accumulated sum r (in scaled variables); returns y = (A x)_i
    __device__ __forceinline__ T store(const DevLevelT<T>& L, T r, T* out, T* xs_, T gamma, int64_t oi) const {
        const T y = (ri == -1) ? r * s : T(0);
        if (MODE == APPLY) {
            out[oi] = y;
        } else {
            const T rr = (ri == -2) ? T(0) : rin - y;
            out[oi] = rr;
            if (MODE == RESID_SMOOTH && ri == -1) xs_[oi] = fmaT(gamma * ro(L.dinv + oi), rr, xs_[oi]);
        }
        return y;
    }
};

// blocks per SM the z-marching apply is compiled for: two in FP64 (its FP64 pipe is the
// bound), four in FP32 (latency-bound: more resident warps hide the plane loads)
template <typename T>
constexpr int zm_blocks_per_sm() { return sizeof(T) == 4 ? 4 : 2; }

template <typename T, int P, int MODE, bool DOT, int YT, bool STG>
__global__ void __launch_bounds__(TPB, zm_blocks_per_sm<T>()) k_apply_zm3d(DevLevelT<T> L, const T* __restrict__ x, const T* rin, T* out,
                                                    T* __restrict__ xs, T gamma, const int* done, double* partial,
                                                    PcgState* st, ZmShape sh) {
    pdl_begin();
    if (done && *done) return;
    constexpr int W = 2 * P + 1, XS = 32 - 2 * P, NV = YT + 2 * P;
    constexpr bool SC = sizeof(T) == 4;              // FP32 path: Jacobi-scaled variables
    extern __shared__ __align__(16) float zm_stage[];   // FP32: [warp][W planes][x, s][NV][32]
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int m = L.m;
    const int64_t mm = (int64_t)m * m;
    double acc = 0.0;
    for (;;) {
        unsigned int t = 0;
        if (lane == 0) t = atomicAdd(&L.tile_ctr[0], 1u);
        t = __shfl_sync(FULL, t, 0);
        if (t >= sh.ntotal) break;
        if (t < sh.ntensor) {
            // ---------------- tensor task: strip sxi, rows y0.., planes zc0..zend-1
            const int sxi = (int)(t % (unsigned)sh.sx);
            const int syi = (int)((t / (unsigned)sh.sx) % (unsigned)sh.sy);
            const int szi = (int)(t / ((unsigned)sh.sx * (unsigned)sh.sy));
            const int gx = sxi * XS - P + lane;
            const int y0 = syi * YT;
            const int zc0 = szi * sh.zc;
            const int zend = min(zc0 + sh.zc, m);
            const bool xin = (unsigned)gx < (unsigned)m;
            const bool own = lane >= P && lane < 32 - P && xin;      // this lane writes outputs
            T kx[W], mx[W];
#pragma unroll
            for (int o = 0; o < W; ++o) {
                kx[o] = xin ? ro(L.K1 + (int64_t)gx * W + o) : T(0);
                mx[o] = xin ? ro(L.M1 + (int64_t)gx * W + o) : T(0);
            }
            // Away from the open-knot ends the 1-D rows are symmetric (c[o] = c[2P - o]): the sums
            // along x and y then pair the neighbours first, 2P adds and 3(P+1) FMA instead of
            // 3(2P+1) FMA along x, P adds and 2(P+1) FMA instead of 2(2P+1) along y.  The test
            // is per warp (x) and per row (y), so no lane diverges.
            bool symx = true;
#pragma unroll
            for (int o = 0; o < P; ++o) symx = symx && kx[o] == kx[2 * P - o] && mx[o] == mx[2 * P - o];
            symx = __all_sync(FULL, symx);
            bool symy[YT];
#pragma unroll
            for (int j = 0; j < YT; ++j) {
                const int gy = y0 + j;
                bool sy = gy < m;
#pragma unroll
                for (int o = 0; o < P; ++o)
                    sy = sy && ro(L.K1 + (int64_t)gy * W + o) == ro(L.K1 + (int64_t)gy * W + 2 * P - o) &&
                         ro(L.M1 + (int64_t)gy * W + o) == ro(L.M1 + (int64_t)gy * W + 2 * P - o);
                symy[j] = sy;
            }
            T ring[YT][W];
#pragma unroll
            for (int j = 0; j < YT; ++j)
#pragma unroll
                for (int q = 0; q < W; ++q) ring[j][q] = T(0);
            const int nplanes = (zend - zc0) + 2 * P;
            // the column segment of input plane zp in registers, the next plane's loads issued
            // before the current plane's arithmetic (zero outside the grid): FP64, and FP32 where
            // the autotuner found it faster than staging (L2-resident levels)
            auto load_plane = [&](int zp, T* v) {
                const bool zin = (unsigned)zp < (unsigned)m;
#pragma unroll
                for (int i = 0; i < NV; ++i) {
                    const int gy = y0 - P + i;
                    const bool in = zin && xin && (unsigned)gy < (unsigned)m;
                    const int64_t g = (int64_t)zp * mm + (int64_t)gy * m + gx;
                    v[i] = in ? (SC ? x[g] * ro(L.s + g) : x[g]) : T(0);
                }
            };
            // FP32 (latency-bound, not ALU-bound): the segments of x and of the Jacobi scale s of
            // the next W - 1 planes are in flight at once, copied by cp.async into this warp's ring
            // of W plane buffers in shared memory.  A lane copies and later reads only its own
            // column, so its own cp.async.wait_group orders them and no warp barrier is needed.
            float* stg = nullptr;
            constexpr bool staged = SC && STG;
            if constexpr (SC) stg = zm_stage + (threadIdx.x >> 5) * (W * 2 * NV * 32);
            auto stage_plane = [&](int k) {
                if constexpr (SC) {
                    const int zp = zc0 - P + k;
                    const bool zin = k < nplanes && (unsigned)zp < (unsigned)m;
                    float* bx = stg + (k % W) * (2 * NV * 32);
#pragma unroll
                    for (int i = 0; i < NV; ++i) {
                        const int gy = y0 - P + i;
                        const bool in = zin && xin && (unsigned)gy < (unsigned)m;
                        const int64_t g = in ? (int64_t)zp * mm + (int64_t)gy * m + gx : 0;
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                                         (uint32_t)__cvta_generic_to_shared(bx + i * 32 + lane)),
                                     "l"(x + g), "r"(in ? 4 : 0)
                                     : "memory");
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                                         (uint32_t)__cvta_generic_to_shared(bx + (NV + i) * 32 + lane)),
                                     "l"(L.s + g), "r"(in ? 4 : 0)
                                     : "memory");
                    }
                    asm volatile("cp.async.commit_group;" ::: "memory");
                }
            };
            T v[NV];
            if constexpr (staged) {
#pragma unroll
                for (int k = 0; k < W - 1; ++k) stage_plane(k);
            } else {
                load_plane(zc0 - P, v);
            }
            for (int base = 0; base < nplanes; base += W) {
#pragma unroll
                for (int u = 0; u < W; ++u) {
                    const int k = base + u;
                    if (k >= nplanes) break;
                    const int zp = zc0 - P + k;                      // input plane
                    OutRow<T, MODE> orow[YT];                        // FP32: this step's output rows
                    if constexpr (SC) {
#pragma unroll
                        for (int j = 0; j < YT; ++j) {
                            const int gy = y0 + j, zo = zp - P;
                            const bool w = own && zo >= zc0 && zo < zend && gy < m;
                            orow[j].load(L, rin, w, w ? (int64_t)zo * mm + (int64_t)gy * m + gx : 0);
                        }
                    }
                    T vn[NV];
                    if constexpr (staged) {
                        stage_plane(k + W - 1);                      // into the buffer of plane k - 1
                        asm volatile("cp.async.wait_group %0;" ::"n"(W - 1) : "memory");   // plane k is in
                        const float* bx = stg + (k % W) * (2 * NV * 32);
#pragma unroll
                        for (int i = 0; i < NV; ++i) v[i] = bx[i * 32 + lane] * bx[(NV + i) * 32 + lane];
                    } else {
                        // the next plane's loads go out before this plane's arithmetic
                        if (k + 1 < nplanes) load_plane(zp + 1, vn);
                    }
                    T a[YT], b[YT];
#pragma unroll
                    for (int j = 0; j < YT; ++j) {
                        const int gy = y0 + j;
                        const T* __restrict__ My = L.M1 + (int64_t)gy * W;
                        const T* __restrict__ Ky = L.K1 + (int64_t)gy * W;
                        T my = T(0), ky = T(0);
                        if (symy[j]) {
                            my = ro(My + P) * v[j + P];
                            ky = ro(Ky + P) * v[j + P];
#pragma unroll
                            for (int o = 0; o < P; ++o) {
                                const T pv = v[j + o] + v[j + 2 * P - o];
                                my = fmaT(ro(My + o), pv, my);
                                ky = fmaT(ro(Ky + o), pv, ky);
                            }
                        } else if (gy < m) {
#pragma unroll
                            for (int o = 0; o < W; ++o) {
                                my = fmaT(ro(My + o), v[j + o], my);
                                ky = fmaT(ro(Ky + o), v[j + o], ky);
                            }
                        }
                        T aa = T(0), bb = T(0);
                        if (symx) {
                            aa = mx[P] * my;
                            bb = fmaT(kx[P], my, mx[P] * ky);
#pragma unroll
                            for (int o = 0; o < P; ++o) {
                                const T sm = __shfl_sync(FULL, my, (lane - P + o) & 31) +
                                             __shfl_sync(FULL, my, (lane + P - o) & 31);
                                const T sk = __shfl_sync(FULL, ky, (lane - P + o) & 31) +
                                             __shfl_sync(FULL, ky, (lane + P - o) & 31);
                                aa = fmaT(mx[o], sm, aa);
                                bb = fmaT(mx[o], sk, bb);
                                bb = fmaT(kx[o], sm, bb);
                            }
                        } else {
#pragma unroll
                            for (int o = 0; o < W; ++o) {
                                const T mo = __shfl_sync(FULL, my, (lane - P + o) & 31);
                                const T ko = __shfl_sync(FULL, ky, (lane - P + o) & 31);
                                aa = fmaT(mx[o], mo, aa);
                                bb = fmaT(mx[o], ko, bb);
                                bb = fmaT(kx[o], mo, bb);
                            }
                        }
                        a[j] = aa;
                        b[j] = bb;
                    }
                    // outputs z = zp - P + jz receive K_z[z][2P - jz] a + M_z[z][2P - jz] b;
                    // output z keeps ring slot (z - zc0 + 2P + 1) mod W, here (u + 1 + jz) mod W
                    // (base is a multiple of W)
#pragma unroll
                    for (int jz = 0; jz < W; ++jz) {
                        const int z = zp - P + jz;
                        if ((unsigned)z < (unsigned)m) {
                            const T kz = ro(L.K1 + (int64_t)z * W + (2 * P - jz));
                            const T mz = ro(L.M1 + (int64_t)z * W + (2 * P - jz));
#pragma unroll
                            for (int j = 0; j < YT; ++j) {
                                T& r = ring[j][(u + 1 + jz) % W];
                                r = fmaT(kz, a[j], r);
                                r = fmaT(mz, b[j], r);
                            }
                        }
                    }
                    // output zp - P has seen its last plane (slot (u + 1) mod W)
                    const int zo = zp - P;
#pragma unroll
                    for (int j = 0; j < YT; ++j) {
                        T& r = ring[j][(u + 1) % W];
                        const int gy = y0 + j;
                        if (own && zo >= zc0 && zo < zend && gy < m) {
                            const int64_t oi = (int64_t)zo * mm + (int64_t)gy * m + gx;
                            if constexpr (SC) {
                                if (orow[j].ri < 0) {
                                    const T y = orow[j].store(L, r, out, xs, gamma, oi);
                                    if (DOT && orow[j].ri == -1) acc = fma((double)x[oi], (double)y, acc);
                                }
                            } else if (const int ri = L.rowinfo[oi]; ri < 0) {   // tensor or inactive row
                                T y = T(0);
                                if (ri == -1) y = r;
                                if (MODE == APPLY) {
                                    out[oi] = y;
                                } else {
                                    const T rr = (ri == -2) ? T(0) : rin[oi] - y;
                                    out[oi] = rr;
                                    if (MODE == RESID_SMOOTH && ri == -1)
                                        xs[oi] = fmaT(gamma * ro(L.dinv + oi), rr, xs[oi]);
                                }
                                if (DOT && ri == -1) acc = fma((double)x[oi], (double)y, acc);
                            }
                        }
                        r = T(0);
                    }
                    if constexpr (!staged) {
#pragma unroll
                        for (int i = 0; i < NV; ++i) v[i] = vn[i];
                    }
                }
            }
            if constexpr (staged) asm volatile("cp.async.wait_group 0;" ::: "memory");   // the ring is free again
        } else {
            // ---------------- stored rows: 32 consecutive stored row ids, one per lane
            const int64_t k = (int64_t)(t - sh.ntensor) * 32 + lane;
            if (k < L.nb) {
                const int64_t oi = L.band_row[k];
                const int ix = (int)(oi % m), iy = (int)((oi / m) % m), iz = (int)(oi / mm);
                const T* __restrict__ c = L.band_coef + k;
                const int64_t nb = L.nb;
                T y = T(0);
#pragma unroll
                for (int oz = 0; oz < W; ++oz) {
                    const bool zin = (unsigned)(iz + oz - P) < (unsigned)m;
#pragma unroll
                    for (int oy = 0; oy < W; ++oy) {
                        const bool yin = zin && (unsigned)(iy + oy - P) < (unsigned)m;
#pragma unroll
                        for (int ox = 0; ox < W; ++ox) {
                            const bool in = yin && (unsigned)(ix + ox - P) < (unsigned)m;
                            const int64_t g = oi + (ox - P) + (int64_t)(oy - P) * m + (int64_t)(oz - P) * mm;
                            const T xv = in ? x[g] : T(0);
                            y = fmaT(ro(c + (int64_t)(ox + W * (oy + W * oz)) * nb), xv, y);
                        }
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
    // every warp has drawn past the end once; the last one re-arms the counter for the next
    // launch (which starts only after this grid has completed)
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

// ---------------------------------------------------------------------------------
// FP32 form of the z-marching apply for levels that stream from HBM: the 8 warps of a CTA
// march together through one x strip, 8 YT rows and a z chunk, and the CTA stages each input
// plane's region (32 columns x (8 YT + 2P) rows of x and of the Jacobi scale s) once in a
// shared-memory ring, ZMC_DEPTH - 1 planes ahead by cp.async, so the y halo of a warp's rows
// is read from shared memory instead of again from L2, and the CTA keeps three planes of its
// tile in flight.  One CTA barrier per plane.  The per-warp arithmetic is that of
// k_apply_zm3d.  Stored rows are CTA tasks of 256 rows.
constexpr int ZMC_DEPTH = 4;

template <int P, int YT>
constexpr size_t zmc_smem() {
    return (size_t)ZMC_DEPTH * 2 * (8 * YT + 2 * P) * 32 * sizeof(float);
}

template <int P, int MODE, int YT>
__global__ void __launch_bounds__(TPB, 3) k_apply_zmc3d(DevLevelT<float> L, const float* __restrict__ x,
                                                        const float* rin, float* out, float* __restrict__ xs,
                                                        float gamma, const int* done, ZmShape sh) {
    pdl_begin();
    using T = float;
    if (done && *done) return;
    constexpr int W = 2 * P + 1, XS = 32 - 2 * P, NV = YT + 2 * P, RY = 8 * YT + 2 * P;
    constexpr int BUF = 2 * RY * 32;                     // floats of one plane buffer (x, then s)
    extern __shared__ __align__(16) float zc_ring[];     // [ZMC_DEPTH][2][RY][32]
    __shared__ unsigned int s_task;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m = L.m;
    const int64_t mm = (int64_t)m * m;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_task = atomicAdd(&L.tile_ctr[0], 1u);
        __syncthreads();
        const unsigned int t = s_task;
        if (t >= sh.ntotal) break;
        if (t < sh.ntensor) {
            const int sxi = (int)(t % (unsigned)sh.sx);
            const int syi = (int)((t / (unsigned)sh.sx) % (unsigned)sh.sy);
            const int szi = (int)(t / ((unsigned)sh.sx * (unsigned)sh.sy));
            const int gx = sxi * XS - P + lane;
            const int yc = syi * 8 * YT;                     // the CTA's first row
            const int y0 = yc + warp * YT;                   // this warp's first row
            const int zc0 = szi * sh.zc;
            const int zend = min(zc0 + sh.zc, m);
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
            bool symy[YT];
#pragma unroll
            for (int j = 0; j < YT; ++j) {
                const int gy = y0 + j;
                bool sy = gy < m;
#pragma unroll
                for (int o = 0; o < P; ++o)
                    sy = sy && ro(L.K1 + (int64_t)gy * W + o) == ro(L.K1 + (int64_t)gy * W + 2 * P - o) &&
                         ro(L.M1 + (int64_t)gy * W + o) == ro(L.M1 + (int64_t)gy * W + 2 * P - o);
                symy[j] = sy;
            }
            T ring[YT][W];
#pragma unroll
            for (int j = 0; j < YT; ++j)
#pragma unroll
                for (int q = 0; q < W; ++q) ring[j][q] = T(0);
            const int nplanes = (zend - zc0) + 2 * P;
            // the CTA copies plane k's region (x and s, zero outside the grid) into buffer k mod D
            auto stage = [&](int k) {
                const int zp = zc0 - P + k;
                const bool zin = k < nplanes && (unsigned)zp < (unsigned)m;
                float* b = zc_ring + (k % ZMC_DEPTH) * BUF;
                for (int e = threadIdx.x; e < 2 * RY * 32; e += TPB) {
                    const int arr = e / (RY * 32), r = (e >> 5) % RY, c = e & 31;
                    const int cx = sxi * XS - P + c, cy = yc - P + r;
                    const bool in = zin && (unsigned)cx < (unsigned)m && (unsigned)cy < (unsigned)m;
                    const int64_t g = in ? (int64_t)zp * mm + (int64_t)cy * m + cx : 0;
                    const float* src = (arr ? L.s : x) + g;
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                                     (uint32_t)__cvta_generic_to_shared(b + e)),
                                 "l"(src), "r"(in ? 4 : 0)
                                 : "memory");
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
            };
#pragma unroll
            for (int k = 0; k < ZMC_DEPTH - 1; ++k) stage(k);
            for (int base = 0; base < nplanes; base += W) {
#pragma unroll
                for (int u = 0; u < W; ++u) {
                    const int k = base + u;
                    if (k >= nplanes) break;
                    const int zp = zc0 - P + k;
                    OutRow<T, MODE> orow[YT];
#pragma unroll
                    for (int j = 0; j < YT; ++j) {
                        const int gy = y0 + j, zo = zp - P;
                        const bool w = own && zo >= zc0 && zo < zend && gy < m;
                        orow[j].load(L, rin, w, w ? (int64_t)zo * mm + (int64_t)gy * m + gx : 0);
                    }
                    asm volatile("cp.async.wait_group %0;" ::"n"(ZMC_DEPTH - 2) : "memory");   // own copies of k
                    __syncthreads();                 // everyone's copies of k; everyone done with k - 1
                    stage(k + ZMC_DEPTH - 1);        // into the buffer of plane k - 1
                    const float* b = zc_ring + (k % ZMC_DEPTH) * BUF;
                    T v[NV];
#pragma unroll
                    for (int i = 0; i < NV; ++i)
                        v[i] = b[(warp * YT + i) * 32 + lane] * b[(RY + warp * YT + i) * 32 + lane];
                    T a[YT], bb2[YT];
#pragma unroll
                    for (int j = 0; j < YT; ++j) {
                        const int gy = y0 + j;
                        const T* __restrict__ My = L.M1 + (int64_t)gy * W;
                        const T* __restrict__ Ky = L.K1 + (int64_t)gy * W;
                        T my = T(0), ky = T(0);
                        if (symy[j]) {
                            my = ro(My + P) * v[j + P];
                            ky = ro(Ky + P) * v[j + P];
#pragma unroll
                            for (int o = 0; o < P; ++o) {
                                const T pv = v[j + o] + v[j + 2 * P - o];
                                my = fmaT(ro(My + o), pv, my);
                                ky = fmaT(ro(Ky + o), pv, ky);
                            }
                        } else if (gy < m) {
#pragma unroll
                            for (int o = 0; o < W; ++o) {
                                my = fmaT(ro(My + o), v[j + o], my);
                                ky = fmaT(ro(Ky + o), v[j + o], ky);
                            }
                        }
                        T aa = T(0), bb = T(0);
                        if (symx) {
                            aa = mx[P] * my;
                            bb = fmaT(kx[P], my, mx[P] * ky);
#pragma unroll
                            for (int o = 0; o < P; ++o) {
                                const T sm = __shfl_sync(FULL, my, (lane - P + o) & 31) +
                                             __shfl_sync(FULL, my, (lane + P - o) & 31);
                                const T sk = __shfl_sync(FULL, ky, (lane - P + o) & 31) +
                                             __shfl_sync(FULL, ky, (lane + P - o) & 31);
                                aa = fmaT(mx[o], sm, aa);
                                bb = fmaT(mx[o], sk, bb);
                                bb = fmaT(kx[o], sm, bb);
                            }
                        } else {
#pragma unroll
                            for (int o = 0; o < W; ++o) {
                                const T mo = __shfl_sync(FULL, my, (lane - P + o) & 31);
                                const T ko = __shfl_sync(FULL, ky, (lane - P + o) & 31);
                                aa = fmaT(mx[o], mo, aa);
                                bb = fmaT(mx[o], ko, bb);
                                bb = fmaT(kx[o], mo, bb);
                            }
                        }
                        a[j] = aa;
                        bb2[j] = bb;
                    }
#pragma unroll
                    for (int jz = 0; jz < W; ++jz) {
                        const int z = zp - P + jz;
                        if ((unsigned)z < (unsigned)m) {
                            const T kz = ro(L.K1 + (int64_t)z * W + (2 * P - jz));
                            const T mz = ro(L.M1 + (int64_t)z * W + (2 * P - jz));
#pragma unroll
                            for (int j = 0; j < YT; ++j) {
                                T& r = ring[j][(u + 1 + jz) % W];
                                r = fmaT(kz, a[j], r);
                                r = fmaT(mz, bb2[j], r);
                            }
                        }
                    }
                    const int zo = zp - P;
#pragma unroll
                    for (int j = 0; j < YT; ++j) {
                        T& r = ring[j][(u + 1) % W];
                        const int gy = y0 + j;
                        if (own && zo >= zc0 && zo < zend && gy < m && orow[j].ri < 0)
                            orow[j].store(L, r, out, xs, gamma, (int64_t)zo * mm + (int64_t)gy * m + gx);
                        r = T(0);
                    }
                }
            }
            asm volatile("cp.async.wait_group 0;" ::: "memory");   // the ring is free for the next task
        } else {
            // ---------------- stored rows: 256 consecutive stored row ids, one per thread
            const int64_t k = (int64_t)(t - sh.ntensor) * TPB + threadIdx.x;
            if (k < L.nb) {
                const int64_t oi = L.band_row[k];
                const int ix = (int)(oi % m), iy = (int)((oi / m) % m), iz = (int)(oi / mm);
                const T* __restrict__ c = L.band_coef + k;
                const int64_t nb = L.nb;
                T y = T(0);
#pragma unroll
                for (int oz = 0; oz < W; ++oz) {
                    const bool zin = (unsigned)(iz + oz - P) < (unsigned)m;
#pragma unroll
                    for (int oy = 0; oy < W; ++oy) {
                        const bool yin = zin && (unsigned)(iy + oy - P) < (unsigned)m;
#pragma unroll
                        for (int ox = 0; ox < W; ++ox) {
                            const bool in = yin && (unsigned)(ix + ox - P) < (unsigned)m;
                            const int64_t g = oi + (ox - P) + (int64_t)(oy - P) * m + (int64_t)(oz - P) * mm;
                            y = fmaT(ro(c + (int64_t)(ox + W * (oy + W * oz)) * nb), in ? x[g] : T(0), y);
                        }
                    }
                }
                if (MODE == APPLY) {
                    out[oi] = y;
                } else {
                    const T rr = rin[oi] - y;
                    out[oi] = rr;
                    if (MODE == RESID_SMOOTH) xs[oi] = fmaT(gamma * ro(L.dinv + oi), rr, xs[oi]);
                }
            }
        }
    }
    // every CTA has drawn past the end once; the last one re-arms the counter
    if (threadIdx.x == 0 && atomicAdd(&L.tile_ctr[1], 1u) == gridDim.x - 1) {
        L.tile_ctr[0] = 0u;
        L.tile_ctr[1] = 0u;
    }
}

// 3-D operator apply: the z-marching warp kernel on levels with enough work to fill the
// GPU (IMGM_TILE3D=1: on every level, for testing it on small grids; IMGM_ZM_BLOCKS=k
// caps its grid at k blocks, so that warps draw many tasks on small grids)
// Task shape of a level: strips of 32 - 2P columns, segments of yt rows, and z chunks of
// equal size, as long as possible (each chunk recomputes the plane passes of 2P halo
// planes) while there are at least ZM_TASKS tensor tasks to spread over the warps (a
// task is one warp's sequential walk, so too few tasks leave the SMs latency-bound),
// and no shorter than ZM_ZMIN planes.  IMGM_ZM_ZC / IMGM_ZM_ZMIN override the two limits.
constexpr int ZM_ZMIN = 4, ZM_ZMAX = 32;
ZmShape zm_shape(int m, int64_t nb, int P, int yt, int zc_set) {
    ZmShape s{};
    const int xs = 32 - 2 * P;
    s.sx = (m + xs - 1) / xs;
    s.sy = (m + yt - 1) / yt;
    int zmin = ZM_ZMIN, zmax = ZM_ZMAX;
    if (const char* v = std::getenv("IMGM_ZM_ZMIN")) zmin = std::max(1, std::atoi(v));
    const int want = (ZM_TASKS + s.sx * s.sy - 1) / (s.sx * s.sy);     // chunks for enough tasks
    int zc = std::max(zmin, std::min(zmax, (m + want - 1) / want));
    if (zc_set > 0) zc = zc_set;
    if (const char* v = std::getenv("IMGM_ZM_ZC")) zc = std::max(1, std::atoi(v));
    const int nz = (m + zc - 1) / zc;
    s.zc = (m + nz - 1) / nz;
    s.sz = (m + s.zc - 1) / s.zc;
    s.ntensor = (unsigned)((int64_t)s.sx * s.sy * s.sz);
    s.ntotal = s.ntensor + (unsigned)((nb + 31) / 32);
    return s;
}
bool use_zm_3d(int m) {
    const char* v = std::getenv("IMGM_TILE3D");
    static const int mmin = [] {
        const char* w = std::getenv("IMGM_ZM_MIN_M");
        return w ? std::atoi(w) : 18;
    }();
    return (v && v[0] == '1') || m >= mmin;
}
// rows per lane: two on large levels (fewer loads per row), one where the level needs the
// extra tasks (IMGM_ZM_YT overrides)
int zm_yt(int m, int yt_set) {
    if (const char* v = std::getenv("IMGM_ZM_YT")) return std::atoi(v) == 1 ? 1 : 2;
    if (yt_set == 1 || yt_set == 2) return yt_set;
    return m >= 100 ? 2 : 1;
}
// dynamic shared memory of the z-marching apply: the FP32 instances' plane rings
template <typename T, int P, int YT, bool STG>
constexpr size_t zm_smem() {
    return (sizeof(T) == 4 && STG) ? (size_t)(TPB / 32) * (2 * P + 1) * 2 * (YT + 2 * P) * 32 * sizeof(float) : 0;
}

template <typename T, int P, int YT, bool STG>
void launch_zm3d_stg(const DevLevelT<T>& L, int mode, const T* x, const T* rin, T* out, T* xs, T gamma,
                     const int* done, cudaStream_t s) {
    const ZmShape sh = zm_shape(L.m, L.nb, P, YT, L.zm_zc);
    const int g = zm_grid(sh, zm_blocks_per_sm<T>() * num_sms());
    constexpr size_t smem = zm_smem<T, P, YT, STG>();
    if (smem > 48 * 1024) {
        static bool attr = false;                      // opted in once per instantiation
        if (!attr) {
            cudaFuncSetAttribute(k_apply_zm3d<T, P, APPLY, false, YT, STG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
            cudaFuncSetAttribute(k_apply_zm3d<T, P, RESID, false, YT, STG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
            cudaFuncSetAttribute(k_apply_zm3d<T, P, RESID_SMOOTH, false, YT, STG>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr = true;
        }
    }
    if (mode == APPLY)
        launch_pdl(k_apply_zm3d<T, P, APPLY, false, YT, STG>, g, TPB, smem, s, L, x, rin, out, xs, gamma, done, nullptr,
                   nullptr, sh);
    else if (mode == RESID)
        launch_pdl(k_apply_zm3d<T, P, RESID, false, YT, STG>, g, TPB, smem, s, L, x, rin, out, xs, gamma, done, nullptr,
                   nullptr, sh);
    else
        launch_pdl(k_apply_zm3d<T, P, RESID_SMOOTH, false, YT, STG>, g, TPB, smem, s, L, x, rin, out, xs, gamma, done,
                   nullptr, nullptr, sh);
}

// the CTA form (FP32): strips x CTA row blocks of 8 YT rows x z chunks, stored rows in tasks of 256
template <int P, int YT>
void launch_zmc3d(const DevLevelT<float>& L, int mode, const float* x, const float* rin, float* out, float* xs,
                  float gamma, const int* done, cudaStream_t s) {
    ZmShape sh = zm_shape(L.m, L.nb, P, 8 * YT, L.zm_zc);
    sh.ntotal = sh.ntensor + (unsigned)((L.nb + TPB - 1) / TPB);
    int64_t g = std::min<int64_t>(sh.ntotal, 3 * num_sms());
    if (const char* v = std::getenv("IMGM_ZM_BLOCKS")) {
        const int k = std::atoi(v);
        if (k > 0) g = std::min<int64_t>(g, k);
    }
    g = std::max<int64_t>(g, 1);
    constexpr size_t smem = zmc_smem<P, YT>();
    static_assert(zmc_smem<P, YT>() <= 48 * 1024, "CTA ring within the default shared memory");
    if (mode == APPLY)
        launch_pdl(k_apply_zmc3d<P, APPLY, YT>, (int)g, TPB, smem, s, L, x, rin, out, xs, gamma, done, sh);
    else if (mode == RESID)
        launch_pdl(k_apply_zmc3d<P, RESID, YT>, (int)g, TPB, smem, s, L, x, rin, out, xs, gamma, done, sh);
    else
        launch_pdl(k_apply_zmc3d<P, RESID_SMOOTH, YT>, (int)g, TPB, smem, s, L, x, rin, out, xs, gamma, done, sh);
}

// FP32 levels take the form the autotuner chose (0 registers, 1 warp-staged, 2 CTA-staged);
// FP64 the register form
template <typename T, int P, int YT>
void launch_zm3d_yt(const DevLevelT<T>& L, int mode, const T* x, const T* rin, T* out, T* xs, T gamma, const int* done,
                    cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (L.zm_stage == 2) {
            launch_zmc3d<P, YT>(L, mode, x, rin, out, xs, gamma, done, s);
            return;
        }
    }
    if (sizeof(T) == 4 && L.zm_stage)
        launch_zm3d_stg<T, P, YT, true>(L, mode, x, rin, out, xs, gamma, done, s);
    else
        launch_zm3d_stg<T, P, YT, false>(L, mode, x, rin, out, xs, gamma, done, s);
}

template <typename T, int P>
cudaError_t launch_zm3d(const DevLevelT<T>& L, int mode, const T* x, const T* rin, T* out, T* xs, T gamma,
                        const int* done, cudaStream_t s) {
    if (L.tile_ctr == nullptr || (L.nb > 0 && L.band_row == nullptr)) return cudaErrorInvalidValue;
    if (zm_yt(L.m, L.zm_yt) == 2)
        launch_zm3d_yt<T, P, 2>(L, mode, x, rin, out, xs, gamma, done, s);
    else
        launch_zm3d_yt<T, P, 1>(L, mode, x, rin, out, xs, gamma, done, s);
    return cudaGetLastError();
}

}  // namespace
}  // namespace imgm
