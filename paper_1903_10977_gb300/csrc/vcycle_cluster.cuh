// The coarse part of the FP32 V-cycle as one thread-block-cluster launch, the levels resident
// in distributed shared memory (Algorithm 1 on levels 1..top: the same arithmetic, in the
// same order, as the separate level kernels).  Instantiated for 2-D levels in
// vcycle_cluster_2d.cu and for 3-D levels in vcycle_cluster_3d.cu.
#pragma once
#include "common.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace imgm {
namespace {

// ---------------------------------------------------------------------------------
// Coarse part of the FP32 V-cycle with the levels resident in distributed shared memory
// (see DsLevel).  Same arithmetic, in the same order, as the separate kernels above; only
// where the data lives differs.
namespace ds {

struct Ctx {
    unsigned char* sm;
    unsigned char* const* bases;   // generic address of every block's shared memory
    unsigned rank;
};

// row j of the common per-row vector at `off` of level L (any block's chunk)
__device__ __forceinline__ float* at(const Ctx& c, const DsLevel& L, uint32_t off, int64_t j) {
    const int64_t l = j - (int64_t)c.rank * L.ch;
    if ((uint64_t)l < (uint64_t)L.ch) return reinterpret_cast<float*>(c.sm + off) + l;
    const unsigned owner = (unsigned)((uint32_t)j / (uint32_t)L.ch);
    return reinterpret_cast<float*>(c.bases[owner] + off) + (j - (int64_t)owner * L.ch);
}

template <typename U>
__device__ __forceinline__ const U* tab(const Ctx& c, uint32_t off) {
    return reinterpret_cast<const U*>(c.sm + off);
}

// A row segment [j0, j0 + len) of a common vector: a plain shared-memory pointer when the
// segment lies in this block's chunk (the usual case), else nullptr (element-wise path).
__device__ __forceinline__ const float* seg(const Ctx& c, const DsLevel& L, uint32_t off, int j0, int len) {
    const int l = j0 - (int)c.rank * L.ch;
    return (l >= 0 && l + len <= L.ch) ? reinterpret_cast<const float*>(c.sm + off) + l : nullptr;
}

// (A v)_i in scaled variables for own row i (local index il); v = the vector at off_v.
// Indices are 32-bit (levels on the cluster hold far fewer than 2^31 rows); the (2p+1)
// values of one grid line are read through one segment pointer.
template <int DIM, int P>
__device__ __forceinline__ float row_apply(const Ctx& c, const DsLevel& L, int64_t i64, int il, uint32_t off_v) {
    constexpr int W = 2 * P + 1;
    constexpr int NC = (DIM == 2) ? W * W : W * W * W;
    const int ri = tab<int32_t>(c, L.off_ri)[il];
    if (ri == -2) return 0.f;
    const int i = (int)i64;
    const int m = L.m;
    const int ix = i % m, iy = (i / m) % m, iz = (DIM == 3) ? i / (m * m) : 0;
    const int sy = m, sz = m * m;
    // valid x offsets of the row's lines
    const int ox0 = max(-P, -ix), ox1 = min(P, m - 1 - ix);
    float y = 0.f;
    if (ri >= 0) {
        const float* cf = tab<float>(c, L.off_coef) + ri * NC;
#pragma unroll
        for (int oz = (DIM == 3 ? -P : 0); oz <= (DIM == 3 ? P : 0); ++oz) {
            if (DIM == 3 && (unsigned)(iz + oz) >= (unsigned)m) continue;
#pragma unroll
            for (int oy = -P; oy <= P; ++oy) {
                if ((unsigned)(iy + oy) >= (unsigned)m) continue;
                const int jc = i + oy * sy + (DIM == 3 ? oz * sz : 0);
                const float* v = seg(c, L, off_v, jc - P, W);
                const float* crow = cf + W * ((oy + P) + (DIM == 3 ? W * (oz + P) : 0)) + P;
#pragma unroll
                for (int ox = -P; ox <= P; ++ox) {
                    if (ox < ox0 || ox > ox1) continue;
                    const float xv = v ? v[ox + P] : *at(c, L, off_v, jc + ox);
                    y = fmaf(crow[ox], xv, y);
                }
            }
        }
        return y;
    }
    const float* K1 = tab<float>(c, L.off_K1);
    const float* M1 = tab<float>(c, L.off_M1);
    float kx[W], mx[W];
#pragma unroll
    for (int o = 0; o < W; ++o) {
        kx[o] = K1[ix * W + o];
        mx[o] = M1[ix * W + o];
    }
#pragma unroll
    for (int oz = (DIM == 3 ? -P : 0); oz <= (DIM == 3 ? P : 0); ++oz) {
        if (DIM == 3 && (unsigned)(iz + oz) >= (unsigned)m) continue;
        const float mz = (DIM == 3) ? M1[iz * W + oz + P] : 1.f, kz = (DIM == 3) ? K1[iz * W + oz + P] : 0.f;
#pragma unroll
        for (int oy = -P; oy <= P; ++oy) {
            if ((unsigned)(iy + oy) >= (unsigned)m) continue;
            const float my = M1[iy * W + oy + P], ky = K1[iy * W + oy + P];
            const int jc = i + oy * sy + (DIM == 3 ? oz * sz : 0);
            const float* v = seg(c, L, off_v, jc - P, W);
            const float* sv = seg(c, L, L.off_s, jc - P, W);
            float a = 0.f, b = 0.f;
#pragma unroll
            for (int ox = -P; ox <= P; ++ox) {
                if (ox < ox0 || ox > ox1) continue;
                const float xv = (v ? v[ox + P] : *at(c, L, off_v, jc + ox)) *
                                 (sv ? sv[ox + P] : *at(c, L, L.off_s, jc + ox));
                a = fmaf(kx[ox + P], xv, a);
                b = fmaf(mx[ox + P], xv, b);
            }
            if (DIM == 2) {
                y = fmaf(my, a, y);
                y = fmaf(ky, b, y);
            } else {
                y = fmaf(my * mz, a, y);
                y = fmaf(fmaf(ky, mz, my * kz), b, y);
            }
        }
    }
    return y * reinterpret_cast<const float*>(c.sm + L.off_s)[il];
}

// x += gamma A_j^{-1} r on the Schwarz blocks this block owns, one warp per block
__device__ __forceinline__ void blocks(const Ctx& c, const DsLevel& L, uint32_t off_r, float gamma, float* rs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t* bptr = tab<int32_t>(c, L.off_bptr);
    const int32_t* bvptr = tab<int32_t>(c, L.off_bvptr);
    const int32_t* bidx = tab<int32_t>(c, L.off_bidx);
    const float* bval = tab<float>(c, L.off_bval);
    for (int b = warp; b < L.nblk; b += DS_TPB / 32) {
        const int s0 = bptr[b], nj = bptr[b + 1] - s0;
        const float* A = bval + bvptr[b];
        for (int a = lane; a < nj; a += 32) rs[a] = *at(c, L, off_r, bidx[s0 + a]);
        __syncwarp();
        for (int a = lane; a < nj; a += 32) {
            float acc = 0.f;
            for (int q = 0; q < nj; ++q) acc = fmaf(A[q * nj + a], rs[q], acc);
            atomicAdd(at(c, L, L.off_x, bidx[s0 + a]), gamma * acc);
        }
        __syncwarp();
    }
}

// own rows: out = rin - A v (and x += gamma dinv out when smooth)
template <int DIM, int P>
__device__ __forceinline__ void resid(const Ctx& c, const DsLevel& L, uint32_t off_v, uint32_t off_rin,
                                      uint32_t off_out, bool smooth, float gamma) {
    const int64_t lo = (int64_t)c.rank * L.ch;
    const int32_t* ri = tab<int32_t>(c, L.off_ri);
    const float* dinv = tab<float>(c, L.off_dinv);
    float* rin = reinterpret_cast<float*>(c.sm + off_rin);
    float* out = reinterpret_cast<float*>(c.sm + off_out);
    float* x = reinterpret_cast<float*>(c.sm + L.off_x);
    for (int l = threadIdx.x; l < L.ch && lo + l < L.N; l += DS_TPB) {
        const float ax = row_apply<DIM, P>(c, L, lo + l, l, off_v);
        const float v = (ri[l] == -2) ? 0.f : rin[l] - ax;
        out[l] = v;
        if (smooth) x[l] = fmaf(gamma * dinv[l], v, x[l]);
    }
}

// own coarse rows of C: r_C = R t_F (scaled), x_C = gamma dinv_C r_C (or 0 on level 1)
template <int DIM, int P>
__device__ __forceinline__ void restrict_(const Ctx& c, const DsLevel& F, const DsLevel& C, float gamma, bool diag) {
    constexpr int P2 = P + 2;
    const int64_t lo = (int64_t)c.rank * C.ch;
    const int mc = C.m, mf = F.m;
    const int32_t* rfirst = tab<int32_t>(c, F.off_rfirst);
    const float* rw = tab<float>(c, F.off_rw);
    const int32_t* cri = tab<int32_t>(c, C.off_ri);
    const float* cdinv = tab<float>(c, C.off_dinv);
    float* rc = reinterpret_cast<float*>(c.sm + C.off_r);
    float* xc = reinterpret_cast<float*>(c.sm + C.off_x);
    const float* cs = reinterpret_cast<const float*>(c.sm + C.off_s);
    for (int l = threadIdx.x; l < C.ch && lo + l < C.N; l += DS_TPB) {
        const int64_t i = lo + l;
        const int cx = (int)(i % mc), cy = (int)((i / mc) % mc), cz = (DIM == 3) ? (int)(i / ((int64_t)mc * mc)) : 0;
        const int fx = rfirst[cx], fy = rfirst[cy], fz = (DIM == 3) ? rfirst[cz] : 0;
        const float* wx = rw + cx * P2;
        const float* wy = rw + cy * P2;
        const float* wz = rw + cz * P2;
        float s = 0.f;
#pragma unroll
        for (int kz = 0; kz < (DIM == 3 ? P2 : 1); ++kz) {
            const float wzk = (DIM == 3) ? wz[kz] : 1.f;
#pragma unroll
            for (int ky = 0; ky < P2; ++ky) {
                const float wyz = wy[ky] * wzk;
                const int64_t rb = (int64_t)fx + (int64_t)mf * ((fy + ky) + (DIM == 3 ? (int64_t)mf * (fz + kz) : 0));
                float t = 0.f;
#pragma unroll
                for (int kx = 0; kx < P2; ++kx)
                    t = fmaf(wx[kx], *at(c, F, F.off_t, rb + kx) * *at(c, F, F.off_d, rb + kx), t);
                s = fmaf(wyz, t, s);
            }
        }
        s *= cs[l];
        if (cri[l] == -2) s = 0.f;
        rc[l] = s;
        xc[l] = diag ? gamma * cdinv[l] * s : 0.f;
    }
}

// own fine rows of F: e_F = R^T x_C (scaled), x_F += e_F
template <int DIM>
__device__ __forceinline__ void prolong(const Ctx& c, const DsLevel& F, const DsLevel& C) {
    const int64_t lo = (int64_t)c.rank * F.ch;
    const int mc = C.m, mf = F.m, TW = F.TW;
    const int32_t* tfirst = tab<int32_t>(c, F.off_tfirst);
    const float* tw = tab<float>(c, F.off_tw);
    const int32_t* fri = tab<int32_t>(c, F.off_ri);
    float* e = reinterpret_cast<float*>(c.sm + F.off_e);
    float* x = reinterpret_cast<float*>(c.sm + F.off_x);
    const float* fd = reinterpret_cast<const float*>(c.sm + F.off_d);
    for (int l = threadIdx.x; l < F.ch && lo + l < F.N; l += DS_TPB) {
        const int64_t a = lo + l;
        const int ax = (int)(a % mf), ay = (int)((a / mf) % mf), az = (DIM == 3) ? (int)(a / ((int64_t)mf * mf)) : 0;
        const int cx = tfirst[ax], cy = tfirst[ay], cz = (DIM == 3) ? tfirst[az] : 0;
        const float* wx = tw + ax * TW;
        const float* wy = tw + ay * TW;
        const float* wz = tw + az * TW;
        float s = 0.f;
        for (int tz = 0; tz < (DIM == 3 ? TW : 1); ++tz) {
            const float wzk = (DIM == 3) ? wz[tz] : 1.f;
            for (int ty = 0; ty < TW; ++ty) {
                const float wyz = wy[ty] * wzk;
                const int64_t rb = (int64_t)cx + (int64_t)mc * ((cy + ty) + (DIM == 3 ? (int64_t)mc * (cz + tz) : 0));
                float t = 0.f;
                for (int tx = 0; tx < TW; ++tx)
                    t = fmaf(wx[tx], *at(c, C, C.off_x, rb + tx) * *at(c, C, C.off_s, rb + tx), t);
                s = fmaf(wyz, t, s);
            }
        }
        s *= fd[l];
        const bool inactive = fri[l] == -2;
        if (inactive) s = 0.f;
        e[l] = s;
        if (!inactive) x[l] += s;
    }
}

// x_0 = C r_0 on the kept rows of level 1, rows spread over the warps of the cluster
__device__ __forceinline__ void coarse(const Ctx& c, const DsLevel& L, const int32_t* rows, const float* Cinv, int nc,
                                       unsigned cs) {
    const int lane = threadIdx.x & 31;
    const int w = (int)c.rank * (DS_TPB / 32) + (threadIdx.x >> 5), nw = (int)cs * (DS_TPB / 32);
    for (int a = w; a < nc; a += nw) {
        const float* row = Cinv + (int64_t)a * nc;
        double acc = 0.0;
        for (int b = lane; b < nc; b += 32) acc = fma((double)ro(row + b), (double)*at(c, L, L.off_r, ro(rows + b)), acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) *at(c, L, L.off_x, ro(rows + a)) = (float)acc;
    }
}

}  // namespace ds

template <int DIM, int P>
__global__ void __launch_bounds__(DS_TPB) k_vcycle_dsmem(const DsVcycle V) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ unsigned char* bases[32];
    cg::cluster_group cl = cg::this_cluster();
    const unsigned rank = cl.block_rank();
    const int tid = threadIdx.x;
    // static data first: this block's image and its rows' scales (independent of the
    // kernels before this one, so read before waiting on them)
    {
        const uint4* src = reinterpret_cast<const uint4*>(V.images + (size_t)rank * V.image_bytes);
        uint4* dst = reinterpret_cast<uint4*>(sm + V.vec_bytes);
        for (uint32_t k = tid; k < V.image_bytes / 16; k += DS_TPB) dst[k] = __ldg(src + k);
        if (tid < V.cs) bases[tid] = reinterpret_cast<unsigned char*>(cl.map_shared_rank(reinterpret_cast<void*>(sm), tid));
    }
    __syncthreads();
    const DsImage& I = *reinterpret_cast<const DsImage*>(sm + V.vec_bytes);
    const ds::Ctx c{sm, bases, rank};
    const int top = V.top;
    for (int li = 0; li <= top; ++li) {
        const DsLevel& L = I.lv[li];
        const int64_t lo = (int64_t)rank * L.ch;
        float* s = reinterpret_cast<float*>(sm + L.off_s);
        float* d = reinterpret_cast<float*>(sm + L.off_d);
        for (int l = tid; l < L.ch; l += DS_TPB) {
            const bool in = lo + l < L.N;
            s[l] = in ? __ldg(V.s_glob[li] + lo + l) : 0.f;
            d[l] = in ? __ldg(V.d_glob[li] + lo + l) : 0.f;
        }
        if (li == 0) {
            float* x0 = reinterpret_cast<float*>(sm + L.off_x);
            for (int l = tid; l < L.ch; l += DS_TPB) x0[l] = 0.f;
        }
    }
    pdl_begin();
    {
        const DsLevel& T = I.lv[top];
        const int64_t lo = (int64_t)rank * T.ch;
        float* x = reinterpret_cast<float*>(sm + T.off_x);
        float* r = reinterpret_cast<float*>(sm + T.off_r);
        for (int l = tid; l < T.ch; l += DS_TPB) {
            const bool in = lo + l < T.N;
            x[l] = in ? V.x_top[lo + l] : 0.f;
            r[l] = in ? V.r_top[lo + l] : 0.f;
        }
    }
    float* rs = reinterpret_cast<float*>(sm + I.scratch_off) + (tid >> 5) * I.max_block;
    const float g = I.gamma;
    cl.sync();
    for (int li = top; li >= 1; --li) {
        const DsLevel& F = I.lv[li];
        ds::blocks(c, F, F.off_r, g, rs);
        cl.sync();
        ds::resid<DIM, P>(c, F, F.off_x, F.off_r, F.off_t, false, g);
        cl.sync();
        ds::restrict_<DIM, P>(c, F, I.lv[li - 1], g, li - 1 >= 1);
        cl.sync();
    }
    ds::coarse(c, I.lv[0], V.c_rows, V.c_inv, V.nc, (unsigned)V.cs);
    for (int li = 1; li <= top; ++li) {
        const DsLevel& F = I.lv[li];
        cl.sync();
        ds::prolong<DIM>(c, F, I.lv[li - 1]);
        cl.sync();
        ds::resid<DIM, P>(c, F, F.off_e, F.off_t, F.off_t, true, g);
        cl.sync();
        ds::blocks(c, F, F.off_t, g, rs);
    }
    cl.sync();     // every block's scatter into the top level is done
    {
        const DsLevel& T = I.lv[top];
        const int64_t lo = (int64_t)rank * T.ch;
        const float* x = reinterpret_cast<const float*>(sm + T.off_x);
        for (int l = tid; l < T.ch && lo + l < T.N; l += DS_TPB) V.x_top[lo + l] = x[l];
    }
    cl.sync();     // no block leaves while others may still read its shared memory
}

}  // namespace
}  // namespace imgm
