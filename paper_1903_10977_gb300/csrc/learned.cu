// Kernels of the learned correction stage (declarations and conventions in learned.cuh).
//
// Convolutions: one thread per output voxel, all output channels in registers, the
// layer's weights converted to FP32 in shared memory (read as warp-wide broadcasts), the
// input channels of a neighbour read as one or two 16-byte loads (bf16, channels
// innermost).  The input gradient of a layer is the forward convolution of the output
// gradient with the transposed, tap-reversed weights, gated by the ReLU of the layer's
// input.  Weight gradients: each thread owns one (out, in) channel pair and a slice of
// the voxels, keeps the 27 tap sums in registers, the block adds its slices in shared
// memory and issues one atomic add per weight.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdlib>

#include "kernels.cuh"
#include "learned.cuh"

namespace imgm {
namespace {

constexpr int CTPB = 128;     // convolution threads per block
constexpr int WTPB = 256;     // weight-gradient threads per block
constexpr int RTPB = 256;     // reduction threads per block (= NET_PARTIALS)
static_assert(RTPB == NET_PARTIALS, "one partial per reduction block");

enum ConvEpilogue { EPI_RELU = 0, EPI_GATE = 1, EPI_OUT = 2 };

__device__ __forceinline__ float bf(uint16_t u) { return __uint_as_float((uint32_t)u << 16); }
__device__ __forceinline__ uint32_t bf_bits(float f) { return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(f)); }

// the CI channels of voxel u as floats
template <int CI, typename TIN>
__device__ __forceinline__ void load_channels(const TIN* __restrict__ x, int64_t u, float* out) {
    if constexpr (CI == 1) {
        if constexpr (sizeof(TIN) == 2) out[0] = bf(x[u]);
        else out[0] = x[u];
    } else if constexpr (sizeof(TIN) == 2) {
        static_assert(CI % 8 == 0, "bf16 channels come in 16-byte groups");
        const uint4* p = reinterpret_cast<const uint4*>(x + u * CI);
#pragma unroll
        for (int q = 0; q < CI / 8; ++q) {
            const uint4 a = p[q];
            const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                out[8 * q + 2 * k] = __uint_as_float(w[k] << 16);
                out[8 * q + 2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
            }
        }
    } else {
        static_assert(CI % 4 == 0, "float channels come in 16-byte groups");
        const float4* p = reinterpret_cast<const float4*>(x + u * CI);
#pragma unroll
        for (int q = 0; q < CI / 4; ++q) {
            const float4 a = p[q];
            out[4 * q] = a.x;
            out[4 * q + 1] = a.y;
            out[4 * q + 2] = a.z;
            out[4 * q + 3] = a.w;
        }
    }
}

// y[v][o] = sum_tap sum_i W[tap][o][i] x[v + off_tap][i], zero outside the grid, then
// EPI_RELU: yb = bf16(max(y, 0)); EPI_GATE: yf = y where gate > 0, else 0;
// EPI_OUT (one channel): yd = y (FP64) and/or yf = y on the mask, 0 elsewhere.
template <int CI, int CO, typename TIN, int EPI>
__global__ void __launch_bounds__(CTPB) k_conv(const TIN* __restrict__ x, const uint16_t* __restrict__ w,
                                               const uint16_t* __restrict__ gate, const uint8_t* __restrict__ mask,
                                               uint16_t* __restrict__ yb, float* __restrict__ yf,
                                               double* __restrict__ yd, int nx, int ny, int nz) {
    __shared__ __align__(16) float ws[27 * CO * CI];
    for (int i = threadIdx.x; i < 27 * CO * CI; i += blockDim.x) ws[i] = bf(w[i]);
    __syncthreads();
    const int64_t nvox = (int64_t)nx * ny * nz;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(v % nx);
        const int64_t q = v / nx;
        const int iy = (int)(q % ny);
        const int iz = (int)(q / ny);
        float acc[CO];
#pragma unroll
        for (int o = 0; o < CO; ++o) acc[o] = 0.f;
#pragma unroll 1
        for (int dz = -1; dz <= 1; ++dz) {
            const int jz = iz + dz;
            if (jz < 0 || jz >= nz) continue;
#pragma unroll 1
            for (int dy = -1; dy <= 1; ++dy) {
                const int jy = iy + dy;
                if (jy < 0 || jy >= ny) continue;
                const int64_t row = (int64_t)nx * (jy + (int64_t)ny * jz);
                const float* wrow = ws + (9 * (dz + 1) + 3 * (dy + 1)) * CO * CI;
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    const int jx = ix + dx;
                    if (jx < 0 || jx >= nx) continue;
                    float xin[CI];
                    load_channels<CI, TIN>(x, row + jx, xin);
                    const float* wt = wrow + (dx + 1) * CO * CI;
#pragma unroll
                    for (int o = 0; o < CO; ++o)
#pragma unroll
                        for (int i = 0; i < CI; ++i) acc[o] = fmaf(wt[o * CI + i], xin[i], acc[o]);
                }
            }
        }
        if constexpr (EPI == EPI_RELU) {
            static_assert(CO % 8 == 0, "bf16 output in 16-byte groups");
            uint4* p = reinterpret_cast<uint4*>(yb + v * CO);
#pragma unroll
            for (int g = 0; g < CO / 8; ++g) {
                uint32_t wv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    wv[k] = bf_bits(fmaxf(acc[8 * g + 2 * k], 0.f)) | (bf_bits(fmaxf(acc[8 * g + 2 * k + 1], 0.f)) << 16);
                p[g] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            }
        } else if constexpr (EPI == EPI_GATE) {
            static_assert(CO % 4 == 0, "float output in 16-byte groups");
            float gv[CO];
            load_channels<CO, uint16_t>(gate, v, gv);
            float4* p = reinterpret_cast<float4*>(yf + v * CO);
#pragma unroll
            for (int g = 0; g < CO / 4; ++g)
                p[g] = make_float4(gv[4 * g] > 0.f ? acc[4 * g] : 0.f, gv[4 * g + 1] > 0.f ? acc[4 * g + 1] : 0.f,
                                   gv[4 * g + 2] > 0.f ? acc[4 * g + 2] : 0.f, gv[4 * g + 3] > 0.f ? acc[4 * g + 3] : 0.f);
        } else {
            static_assert(CO == 1, "one output channel");
            const bool on = !mask || mask[v];
            if (yd) yd[v] = on ? (double)acc[0] : 0.0;
            if (yf) yf[v] = on ? acc[0] : 0.f;
        }
    }
}

// ---------------------------------------------------------------------------------
// The 16 -> 16 layer's forward convolution on the tensor cores (tcgen05, kind::f16 with
// bf16 operands and an FP32 accumulator in tensor memory).  It is an implicit GEMM: the
// 128 output voxels of an 8 x 16 patch of one z plane are the M = 128 rows, the 16 output
// channels N = 16, and each of the 27 taps one K = 16 step (the 16 input channels of the
// neighbour in that direction): y = sum_tap X_tap W_tap^T, 27 MMAs per output plane.
//
// A CTA walks a column of patches along z.  Its input planes (the patch plus a one-voxel
// halo, 10 x 18 voxels, zero outside the grid) sit in a ring of three shared-memory
// slots, each stored as two planes of 8-channel groups (16 bytes per voxel, x fastest).
// In that layout the operand of tap (dx, dy, dz) is a canonical K-major matrix without
// swizzling: 8-row core matrices are 8 consecutive voxels of an x line (16-byte rows), the
// next 8 rows the next y line (stride 10 x 16 B), the second 8 channels one group-plane
// further; its start moves by 16 bytes per voxel of shift, so all 27 operands are views
// of the same ring.  The weights of tap t, W_t[out][in], are the K-major B operand in the
// same layout (16-byte rows per output channel).
//
// Per output plane: the CTA waits for the previous plane's MMAs (an mbarrier the MMA
// commit arrives on), starts the copy of the input plane two ahead into the ring slot
// those MMAs no longer read (cp.async, so that it overlaps this plane's work; four slots
// hold planes z - 1 .. z + 2), waits for the plane one ahead, and one thread issues the
// plane's 27 MMAs into one of two accumulators while the four warps read the previous
// plane's accumulator (tcgen05.ld, one warp per 32 rows) and store it through the
// layer's epilogue.  Every wait is bounded: after about a second the CTA sets *err and
// stops (the host reports the error), never hanging the GPU.
constexpr int TC_PX = 8, TC_PY = 16;                 // output patch of one plane: 128 voxels
constexpr int TC_RX = TC_PX + 2, TC_RY = TC_PY + 2;  // its input region with the halo
constexpr int TC_RV = TC_RX * TC_RY;                 // 180 voxels
constexpr int TC_GROUP = TC_RV * 16;                 // one 8-channel group-plane of a slot (bytes)
constexpr int TC_SLOT = 2 * TC_GROUP;                // one input plane: 5,760 bytes
constexpr int TC_WBYTES = 27 * 512;                  // B operands of the 27 taps
constexpr int TC_ZC = 16;                            // output planes per CTA
constexpr int TC_THREADS = 128;
constexpr int TC_SLOTS = 4;                          // ring slots: planes z - 1 .. z + 2
// shared memory: weights, ring, two mbarriers and the TMEM address
constexpr int TC_SMEM = TC_WBYTES + TC_SLOTS * TC_SLOT + 64;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor: start address, leading (K-direction) and
// stride (M/N-direction) byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B bf16
// (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// waits until the mbarrier's phase of the given parity has completed; false after ~1 s
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = globaltimer();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (globaltimer() - t0 > 1000000000ull) return false;
    }
}

// Instances: the forward 16 -> 16 layer (bf16 input, ReLU, bf16 output), the forward
// 16 -> 1 layer (CO = 1: the one output channel is column 0 of a 16-column accumulator whose
// other weights are zero; FP64 and/or FP32 output on the mask), and the 16 -> 16 layer's
// input gradient (FP32 output gradient rounded to bf16 as it enters shared memory, the
// transposed weights, FP32 result where the layer's input gate is positive).
template <typename TIN, int CI, int CO, int EPI>
__global__ void __launch_bounds__(TC_THREADS) k_conv16_tc(const TIN* __restrict__ x, const uint16_t* __restrict__ w,
                                                          const uint16_t* __restrict__ gate,
                                                          const uint8_t* __restrict__ mask, uint16_t* __restrict__ yb,
                                                          float* __restrict__ yf, double* __restrict__ yd, int nx,
                                                          int ny, int nz, int* err) {
    static_assert(CO == 16 || CO == 1, "16 output channels or one");
    static_assert(CI == 16 || (CI == 1 && sizeof(TIN) == 2), "16 input channels, or one bf16 channel");
    constexpr bool ASYNC = CI == 16 && sizeof(TIN) == 2;       // bf16 planes copied by cp.async
    extern __shared__ __align__(1024) unsigned char tsm[];
    unsigned char* wsm = tsm;                                    // [27][2 groups][16 out][8 in] bf16
    unsigned char* ring = tsm + TC_WBYTES;                       // [4 slots][2 groups][180 voxels][8] bf16
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + TC_SLOTS * TC_SLOT);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int npx = (nx + TC_PX - 1) / TC_PX, npy = (ny + TC_PY - 1) / TC_PY;
    const int bx = blockIdx.x % npx, by = (blockIdx.x / npx) % npy, bz = blockIdx.x / (npx * npy);
    const int x0 = bx * TC_PX, y0 = by * TC_PY, z0 = bz * TC_ZC, z1 = min(z0 + TC_ZC, nz);

    // B operands: W_t[o][i] -> group i / 8, row o, column i % 8
    uint16_t* wsm16 = reinterpret_cast<uint16_t*>(wsm);
    for (int q = tid; q < 27 * 256; q += TC_THREADS) {
        const int t = q >> 8, o = (q >> 4) & 15, i = q & 15;
        // layouts [tap][out][in]: 16 x 16, 1 x 16 (CO = 1) or 16 x 1 (CI = 1), zero-padded
        const uint16_t v = CI == 1 ? (i == 0 ? w[t * 16 + o] : (uint16_t)0)
                                   : (CO == 16 ? w[q] : (o == 0 ? w[t * 16 + i] : (uint16_t)0));
        wsm16[t * 256 + (i >> 3) * 128 + o * 8 + (i & 7)] = v;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {                                 // 32 columns: two 16-column accumulators
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // one input plane into its slot: 180 voxels x 2 groups of 16 bytes (zero outside the
    // grid); bf16 16-channel planes by cp.async (a group per plane; the caller commits and
    // waits), the others with plain loads and stores
    auto load_plane = [&](int zp) {
        unsigned char* slot = ring + ((zp - z0 + 1) & (TC_SLOTS - 1)) * TC_SLOT;
        for (int q = tid; q < 2 * TC_RV; q += TC_THREADS) {
            const int vox = q >> 1, g = q & 1;
            const int gx = x0 - 1 + vox % TC_RX, gy = y0 - 1 + vox / TC_RX;
            const bool in = (unsigned)gx < (unsigned)nx && (unsigned)gy < (unsigned)ny && (unsigned)zp < (unsigned)nz;
            const int64_t v = in ? (int64_t)gx + (int64_t)nx * (gy + (int64_t)ny * zp) : 0;
            unsigned char* dst = slot + g * TC_GROUP + vox * 16;
            if constexpr (ASYNC) {
                const TIN* src = x + v * 16 + g * 8;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
                             "r"(in ? 16 : 0)
                             : "memory");
            } else {
                uint4 val = make_uint4(0u, 0u, 0u, 0u);
                if (in) {
                    if constexpr (CI == 1) {
                        if (g == 0) val.x = (uint32_t)x[v];          // channel 0 of 16, the rest zero
                    } else if constexpr (sizeof(TIN) == 2) {
                        val = *reinterpret_cast<const uint4*>(x + v * 16 + g * 8);
                    } else {                              // FP32 channels, rounded to bf16 here
                        const float4 a = *reinterpret_cast<const float4*>(x + v * 16 + g * 8);
                        const float4 b = *reinterpret_cast<const float4*>(x + v * 16 + g * 8 + 4);
                        val = make_uint4(bf_bits(a.x) | (bf_bits(a.y) << 16), bf_bits(a.z) | (bf_bits(a.w) << 16),
                                         bf_bits(b.x) | (bf_bits(b.y) << 16), bf_bits(b.z) | (bf_bits(b.w) << 16));
                    }
                }
                *reinterpret_cast<uint4*>(dst) = val;
            }
        }
        if constexpr (ASYNC) asm volatile("cp.async.commit_group;" ::: "memory");
    };
    load_plane(z0 - 1);
    load_plane(z0);
    if constexpr (ASYNC) {
        load_plane(z0 + 1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");   // planes z0 - 1 and z0 are in
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t wbase = smem_u32(wsm), rbase = smem_u32(ring);

    // accumulator of plane k -> ReLU -> bf16 -> y (row = warp * 32 + lane)
    auto epilogue = [&](int k) {
        uint32_t v[16];
        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((k & 1) * 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int row = warp * 32 + lane;
        const int gx = x0 + row % TC_PX, gy = y0 + row / TC_PX, gz = z0 + k;
        if (gx < nx && gy < ny) {
            const int64_t vox = (int64_t)gx + (int64_t)nx * (gy + (int64_t)ny * gz);
            if constexpr (EPI == EPI_RELU) {
                uint32_t pk[8];
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    pk[c] = bf_bits(fmaxf(__uint_as_float(v[2 * c]), 0.f)) |
                            (bf_bits(fmaxf(__uint_as_float(v[2 * c + 1]), 0.f)) << 16);
                uint4* out = reinterpret_cast<uint4*>(yb + vox * 16);
                out[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                out[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            } else if constexpr (EPI == EPI_GATE) {
                float gv[16];
                load_channels<16, uint16_t>(gate, vox, gv);
                float4* out = reinterpret_cast<float4*>(yf + vox * 16);
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    out[c] = make_float4(gv[4 * c] > 0.f ? __uint_as_float(v[4 * c]) : 0.f,
                                         gv[4 * c + 1] > 0.f ? __uint_as_float(v[4 * c + 1]) : 0.f,
                                         gv[4 * c + 2] > 0.f ? __uint_as_float(v[4 * c + 2]) : 0.f,
                                         gv[4 * c + 3] > 0.f ? __uint_as_float(v[4 * c + 3]) : 0.f);
            } else {
                const bool on = !mask || mask[vox];
                const float o0 = __uint_as_float(v[0]);
                if (yd) yd[vox] = on ? (double)o0 : 0.0;
                if (yf) yf[vox] = on ? o0 : 0.f;
            }
        }
    };

    bool ok = true;
    const int nk = z1 - z0;
    for (int k = 0; k < nk && ok; ++k) {
        const int z = z0 + k;
        if (k > 0) ok = __syncthreads_and(mbar_wait(smem_u32(&bars[(k - 1) & 1]), ((k - 1) >> 1) & 1));
        if (!ok) break;
        if constexpr (ASYNC) {
            load_plane(z + 2);                        // the slot of plane z - 2, no longer read
            asm volatile("cp.async.wait_group 1;" ::: "memory");   // plane z + 1 is in
        } else {
            load_plane(z + 1);                        // the slot of plane z - 3, no longer read
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t d = tmem + (uint32_t)((k & 1) * 16);
#pragma unroll 1
            for (int t = 0; t < 27; ++t) {
                const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
                const uint32_t a = rbase + ((z + dz - z0 + 1) & (TC_SLOTS - 1)) * TC_SLOT + 16 * ((dx + 1) + TC_RX * (dy + 1));
                const uint64_t ad = tc_desc(a, TC_GROUP, 16 * TC_RX);
                const uint64_t bd = tc_desc(wbase + t * 512, 256, 128);
                const uint32_t acc = t > 0 ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                    ::"r"(d), "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bars[k & 1]))
                         : "memory");
        }
        if (k > 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            epilogue(k - 1);
        }
    }
    if (ok && nk > 0) {
        ok = __syncthreads_and(mbar_wait(smem_u32(&bars[(nk - 1) & 1]), ((nk - 1) >> 1) & 1));
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            epilogue(nk - 1);
        }
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    if constexpr (ASYNC) asm volatile("cp.async.wait_group 0;" ::: "memory");   // no copy outlives the CTA
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
}

// ---------------------------------------------------------------------------------
// The same convolutions with the z taps folded into the MMA's N dimension.  An input plane
// zp feeds the output planes zp + 1, zp and zp - 1 (taps dz = -1, 0, +1) through the same
// shifted operand, so each of its nine (dx, dy) shifts is ONE MMA of N = 48: B holds
// W(dx, dy, +1), W(dx, dy, 0) and W(dx, dy, -1) one below the other, and the accumulator
// columns [16 (o - z0 + 2), +16) belong to output plane o, so the 48 columns of input zp's
// MMAs land on the accumulators of planes zp - 1, zp and zp + 1, which slide along z with
// the input plane.  Nine MMAs per plane instead of 27 of N = 16 (the tensor pipe's issue
// rate, not its math, bounds the narrow ones); each input plane is read by its own MMAs
// only, so three ring slots hold the plane being multiplied and the two being copied.
// Accumulators: TCZ_ZC + 4 groups of 16 columns (one per output plane of the chunk, plus
// the neighbours of its first and last), cleared with tcgen05.st before the first MMA.
constexpr int TCZ_ZC = 4;                            // output planes per CTA
constexpr int TCZ_COLS = 128;                        // TMEM columns: 16 (TCZ_ZC + 4) rounded up
constexpr int TCZ_SLOTS = 3;
constexpr int TCZ_WBYTES = 9 * 1536;                 // 9 B operands of 48 rows x 16 bf16
constexpr int TCZ_SMEM_USED = TCZ_WBYTES + TCZ_SLOTS * TC_SLOT + 64;
// requested per CTA: enough that at most four CTAs share an SM, whose 512 TMEM columns then
// hold all their accumulators (a fifth CTA's tcgen05.alloc would wait for one to finish)
constexpr int TCZ_SMEM = TCZ_SMEM_USED > 56 * 1024 ? TCZ_SMEM_USED : 56 * 1024;
static_assert(16 * (TCZ_ZC + 4) <= TCZ_COLS, "accumulators exceed the allocation");
// kind::f16, FP32 accumulator, bf16 A and B, K-major, N = 48, M = 128
constexpr uint32_t TCZ_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((48u >> 3) << 17) | ((128u >> 4) << 24);

template <typename TIN, int CI, int CO, int EPI>
__global__ void __launch_bounds__(TC_THREADS) k_conv_tcz(const TIN* __restrict__ x, const uint16_t* __restrict__ w,
                                                         const uint16_t* __restrict__ gate,
                                                         const uint8_t* __restrict__ mask, uint16_t* __restrict__ yb,
                                                         float* __restrict__ yf, double* __restrict__ yd, int nx,
                                                         int ny, int nz, int* err) {
    static_assert(CO == 16 || CO == 1, "16 output channels or one");
    static_assert(CI == 16 || (CI == 1 && sizeof(TIN) == 2), "16 input channels, or one bf16 channel");
    constexpr bool ASYNC = CI == 16 && sizeof(TIN) == 2;
    extern __shared__ __align__(1024) unsigned char tsm[];
    unsigned char* wsm = tsm;                                    // [9][2 groups][48 rows][8 in] bf16
    unsigned char* ring = tsm + TCZ_WBYTES;                      // [3 slots][2 groups][180 voxels][8] bf16
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + TCZ_SLOTS * TC_SLOT);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int npx = (nx + TC_PX - 1) / TC_PX, npy = (ny + TC_PY - 1) / TC_PY;
    const int bx = blockIdx.x % npx, by = (blockIdx.x / npx) % npy, bz = blockIdx.x / (npx * npy);
    const int x0 = bx * TC_PX, y0 = by * TC_PY, z0 = bz * TCZ_ZC, z1 = min(z0 + TCZ_ZC, nz);

    // B operand of shift (dx, dy): row n = 16 q + o holds W(dx, dy, dz = 1 - q)[o][.]
    uint16_t* wsm16 = reinterpret_cast<uint16_t*>(wsm);
    for (int e = tid; e < 9 * 48 * 16; e += TC_THREADS) {
        const int s9 = e / 768, n = (e / 16) % 48, i = e % 16;
        const int q = n / 16, o = n % 16;
        const int dz = 1 - q, t = 9 * (dz + 1) + (s9 / 3) * 3 + (s9 % 3);     // tap index of W[t]
        const uint16_t v = CI == 1 ? (i == 0 ? w[t * 16 + o] : (uint16_t)0)
                                   : (CO == 16 ? w[(t * 16 + o) * 16 + i] : (o == 0 ? w[t * 16 + i] : (uint16_t)0));
        wsm16[s9 * 768 + (i >> 3) * 384 + n * 8 + (i & 7)] = v;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "n"(TCZ_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    auto load_plane = [&](int zp) {
        unsigned char* slot = ring + ((zp - z0 + 1) % TCZ_SLOTS) * TC_SLOT;
        for (int q = tid; q < 2 * TC_RV; q += TC_THREADS) {
            const int vox = q >> 1, g = q & 1;
            const int gx = x0 - 1 + vox % TC_RX, gy = y0 - 1 + vox / TC_RX;
            const bool in = (unsigned)gx < (unsigned)nx && (unsigned)gy < (unsigned)ny && (unsigned)zp < (unsigned)nz;
            const int64_t v = in ? (int64_t)gx + (int64_t)nx * (gy + (int64_t)ny * zp) : 0;
            unsigned char* dst = slot + g * TC_GROUP + vox * 16;
            if constexpr (ASYNC) {
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(x + v * 16 + g * 8),
                             "r"(in ? 16 : 0)
                             : "memory");
            } else {
                uint4 val = make_uint4(0u, 0u, 0u, 0u);
                if (in) {
                    if constexpr (CI == 1) {
                        if (g == 0) val.x = (uint32_t)x[v];
                    } else if constexpr (sizeof(TIN) == 2) {
                        val = *reinterpret_cast<const uint4*>(x + v * 16 + g * 8);
                    } else {
                        const float4 a = *reinterpret_cast<const float4*>(x + v * 16 + g * 8);
                        const float4 b = *reinterpret_cast<const float4*>(x + v * 16 + g * 8 + 4);
                        val = make_uint4(bf_bits(a.x) | (bf_bits(a.y) << 16), bf_bits(a.z) | (bf_bits(a.w) << 16),
                                         bf_bits(b.x) | (bf_bits(b.y) << 16), bf_bits(b.z) | (bf_bits(b.w) << 16));
                    }
                }
                *reinterpret_cast<uint4*>(dst) = val;
            }
        }
        if constexpr (ASYNC) asm volatile("cp.async.commit_group;" ::: "memory");
    };
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t wbase = smem_u32(wsm), rbase = smem_u32(ring);
    {   // clear this warp's 32 lanes of every accumulator column
        const uint32_t z = 0u;
        for (int c = 0; c < TCZ_COLS; c += 16)
            asm volatile(
                "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
                "%1, %1};" ::"r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c),
                "r"(z)
                : "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    if constexpr (ASYNC) {
        load_plane(z0 - 1);
        load_plane(z0);
    }

    // output plane o: accumulator group o - z0 + 2 -> epilogue -> y
    auto epilogue = [&](int o) {
        uint32_t v[16];
        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(16 * (o - z0 + 2));
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int row = warp * 32 + lane;
        const int gx = x0 + row % TC_PX, gy = y0 + row / TC_PX;
        if (gx < nx && gy < ny) {
            const int64_t vox = (int64_t)gx + (int64_t)nx * (gy + (int64_t)ny * o);
            if constexpr (EPI == EPI_RELU) {
                uint32_t pk[8];
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    pk[c] = bf_bits(fmaxf(__uint_as_float(v[2 * c]), 0.f)) |
                            (bf_bits(fmaxf(__uint_as_float(v[2 * c + 1]), 0.f)) << 16);
                uint4* out = reinterpret_cast<uint4*>(yb + vox * 16);
                out[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                out[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            } else if constexpr (EPI == EPI_GATE) {
                float gv[16];
                load_channels<16, uint16_t>(gate, vox, gv);
                float4* out = reinterpret_cast<float4*>(yf + vox * 16);
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    out[c] = make_float4(gv[4 * c] > 0.f ? __uint_as_float(v[4 * c]) : 0.f,
                                         gv[4 * c + 1] > 0.f ? __uint_as_float(v[4 * c + 1]) : 0.f,
                                         gv[4 * c + 2] > 0.f ? __uint_as_float(v[4 * c + 2]) : 0.f,
                                         gv[4 * c + 3] > 0.f ? __uint_as_float(v[4 * c + 3]) : 0.f);
            } else {
                const bool on = !mask || mask[vox];
                const float o0 = __uint_as_float(v[0]);
                if (yd) yd[vox] = on ? (double)o0 : 0.0;
                if (yf) yf[vox] = on ? o0 : 0.f;
            }
        }
    };

    bool ok = true;
    const int K = (z1 - z0) + 2;                     // input planes z0 - 1 .. z1
    for (int k = 0; k < K && ok; ++k) {
        const int zp = z0 - 1 + k;
        if (k > 0) ok = __syncthreads_and(mbar_wait(smem_u32(&bars[(k - 1) & 1]), ((k - 1) >> 1) & 1));
        if (!ok) break;
        if constexpr (ASYNC) {
            load_plane(zp + 2);                       // the slot of plane zp - 1, whose MMAs are done
            asm volatile("cp.async.wait_group 2;" ::: "memory");      // plane zp is in
        } else {
            load_plane(zp);                           // the slot of plane zp - 3
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t d = tmem + (uint32_t)(16 * k);            // groups of planes zp - 1, zp, zp + 1
            const uint32_t a0 = rbase + ((zp - z0 + 1) % TCZ_SLOTS) * TC_SLOT;
#pragma unroll 1
            for (int s9 = 0; s9 < 9; ++s9) {
                const int dy = s9 / 3 - 1, dx = s9 % 3 - 1;
                const uint64_t ad = tc_desc(a0 + 16 * ((dx + 1) + TC_RX * (dy + 1)), TC_GROUP, 16 * TC_RX);
                const uint64_t bd = tc_desc(wbase + s9 * 1536, 768, 128);
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                    ::"r"(d), "l"(ad), "l"(bd), "r"(TCZ_IDESC), "r"(1u)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bars[k & 1]))
                         : "memory");
        }
        // output plane zp - 2 has received its last contribution (from plane zp - 1)
        if (k >= 3 && zp - 2 >= z0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            epilogue(zp - 2);
        }
    }
    if (ok) {
        ok = __syncthreads_and(mbar_wait(smem_u32(&bars[(K - 1) & 1]), ((K - 1) >> 1) & 1));
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            epilogue(z1 - 1);                         // the last output plane (z1 > z0)
        }
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    if constexpr (ASYNC) asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TCZ_COLS) : "memory");
}

// part[block][tap][o][i] = the block's share of sum_v dy[v][o] x[v + off_tap][i]; k_wsum adds
// the blocks' shares to gw in block order, so the gradient of given inputs is the same bits in
// every run (FP32 atomics would add them in whatever order the blocks finish)
template <int CI, int CO>
__global__ void __launch_bounds__(WTPB) k_wgrad(const float* __restrict__ dy, const uint16_t* __restrict__ x,
                                                float* __restrict__ part, int nx, int ny, int nz) {
    constexpr int P = CI * CO;
    constexpr int S = WTPB / P;
    static_assert(P * S == WTPB, "channel pairs must divide the block");
    __shared__ float red[27 * WTPB];
    const int pair = threadIdx.x % P, slice = threadIdx.x / P;
    const int co = pair / CI, ci = pair % CI;
    const int64_t nvox = (int64_t)nx * ny * nz;
    float acc[27];
#pragma unroll
    for (int t = 0; t < 27; ++t) acc[t] = 0.f;
    for (int64_t v = (int64_t)blockIdx.x * S + slice; v < nvox; v += (int64_t)gridDim.x * S) {
        const float g = dy[v * CO + co];
        if (g == 0.f) continue;
        const int ix = (int)(v % nx);
        const int64_t q = v / nx;
        const int iy = (int)(q % ny);
        const int iz = (int)(q / ny);
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
#pragma unroll
            for (int dy_ = -1; dy_ <= 1; ++dy_) {
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    const int jx = ix + dx, jy = iy + dy_, jz = iz + dz;
                    if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz) continue;
                    const int64_t u = jx + (int64_t)nx * (jy + (int64_t)ny * jz);
                    const int t = 9 * (dz + 1) + 3 * (dy_ + 1) + (dx + 1);
                    acc[t] = fmaf(g, bf(x[u * CI + ci]), acc[t]);
                }
            }
        }
    }
    if constexpr (S > 1) {
#pragma unroll
        for (int t = 0; t < 27; ++t) red[t * WTPB + threadIdx.x] = acc[t];
        __syncthreads();
        if (slice == 0) {
#pragma unroll
            for (int t = 0; t < 27; ++t) {
                float s = 0.f;
                for (int k = 0; k < S; ++k) s += red[t * WTPB + k * P + pair];
                acc[t] = s;
            }
        }
    }
    if (slice == 0) {
        float* __restrict__ out = part + (int64_t)blockIdx.x * (27 * P);
#pragma unroll
        for (int t = 0; t < 27; ++t) out[(t * CO + co) * CI + ci] = acc[t];
    }
}

// gw[k] += sum over the nb blocks of part[b][k], in block order
__global__ void __launch_bounds__(RTPB) k_wsum(const float* __restrict__ part, int nb, int nw, float* __restrict__ gw) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nw) return;
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += part[(int64_t)b * nw + k];
    gw[k] += s;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
    __syncthreads();
    return s;   // valid in thread 0
}

__global__ void __launch_bounds__(RTPB) k_pack(int64_t n, const double* __restrict__ in, const uint8_t* __restrict__ mask,
                                               double in_scale, uint16_t* __restrict__ a0) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        a0[v] = (!mask || mask[v]) ? (uint16_t)bf_bits((float)(in[v] * in_scale)) : (uint16_t)0;
}

__global__ void __launch_bounds__(RTPB) k_loss(int64_t n, const float* __restrict__ o, const double* __restrict__ t,
                                               const uint8_t* __restrict__ mask, double scale, float* __restrict__ d3,
                                               double* loss) {
    __shared__ double sh[RTPB / 32];
    double acc = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const double diff = (!mask || mask[v]) ? ((double)o[v] - t[v]) : 0.0;
        d3[v] = (float)(2.0 * diff * scale);
        acc = fma(diff, diff, acc);
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0 && s != 0.0) atomicAdd(loss, s * scale);
}

// weight k of the flat vector: its layer's (tap, out, in) and its places in wb and wbt
__device__ __forceinline__ void net_places(int k, int& fwd, int& bwd) {
    int off, CI, CO;
    if (k < NET_OFF2) {
        off = 0, CI = 1, CO = NET_C;
    } else if (k < NET_OFF3) {
        off = NET_OFF2, CI = NET_C, CO = NET_C;
    } else {
        off = NET_OFF3, CI = NET_C, CO = 1;
    }
    const int r = k - off;
    const int tap = r / (CO * CI), rem = r % (CO * CI);
    const int co = rem / CI, ci = rem % CI;
    fwd = k;
    bwd = off + ((26 - tap) * CI + ci) * CO + co;
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       uint16_t* __restrict__ wb, uint16_t* __restrict__ wbt, float lr, float b1, float b2, float eps,
                       float c1, float c2, int update) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NET_NW) return;
    float wk = w[k];
    if (update) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        wk -= lr * (mk * c1) / (sqrtf(vk * c2) + eps);
        w[k] = wk;
    }
    int f, b;
    net_places(k, f, b);
    const uint16_t q = (uint16_t)bf_bits(wk);
    wb[f] = q;
    wbt[b] = q;
}

// partial[2 blk] = sum a b, partial[2 blk + 1] = sum c d (c null: 0)
__global__ void __launch_bounds__(RTPB) k_dots(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                                               const double* __restrict__ c, const double* __restrict__ d,
                                               double* partial) {
    __shared__ double sh[RTPB / 32];
    double s0 = 0.0, s1 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        s0 = fma(a[i], b[i], s0);
        if (c) s1 = fma(c[i], d[i], s1);
    }
    const double t0 = block_sum(s0, sh);
    const double t1 = block_sum(s1, sh);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = t0;
        partial[2 * blockIdx.x + 1] = t1;
    }
}

// both sums of the NET_PARTIALS partials, in a fixed order (every block gets the same)
__device__ __forceinline__ void sum_partials(const double* partial, double* s0, double* s1) {
    __shared__ double a[RTPB], b[RTPB];
    a[threadIdx.x] = partial[2 * threadIdx.x];
    b[threadIdx.x] = partial[2 * threadIdx.x + 1];
    __syncthreads();
    for (int h = RTPB / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            a[threadIdx.x] += a[threadIdx.x + h];
            b[threadIdx.x] += b[threadIdx.x + h];
        }
        __syncthreads();
    }
    *s0 = a[0];
    *s1 = b[0];
}

__global__ void __launch_bounds__(RTPB) k_stage_axpy(int64_t n, double* __restrict__ z, const double* __restrict__ c,
                                                     const double* __restrict__ partial, double* omega_out) {
    double num, den;
    sum_partials(partial, &num, &den);
    double omega = 0.0;
    if (den > 0.0) {
        omega = num / den;
        if (!isfinite(omega)) omega = 0.0;
    }
    if (omega_out && blockIdx.x == 0 && threadIdx.x == 0) omega_out[0] = omega;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = fma(omega, c[i], z[i]);
}

__global__ void __launch_bounds__(RTPB) k_sub(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                                              double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] - b[i];
}

// partials hold (sum r^2, sum e^2): r, e *= k = 1 / rms(e); r_rms_out = rms(r) afterwards
__global__ void __launch_bounds__(RTPB) k_pair_scale(int64_t n, double* __restrict__ r, double* __restrict__ e,
                                                     double count, const double* __restrict__ partial,
                                                     double* r_rms_out) {
    double sr, se;
    sum_partials(partial, &sr, &se);
    const double k = (se > 0.0 && count > 0.0) ? 1.0 / sqrt(se / count) : 1.0;
    if (r_rms_out && blockIdx.x == 0 && threadIdx.x == 0) r_rms_out[0] = count > 0.0 ? k * sqrt(sr / count) : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        r[i] *= k;
        e[i] *= k;
    }
}

int sm_count() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    return sms;
}

// Which convolution kernels the network uses: 1 (default) the tensor cores with one N = 16
// MMA per tap (k_conv16_tc), 2 (IMGM_NET_TC=48) the tensor cores with the z taps folded into
// N = 48 (k_conv_tcz: a third of the MMAs, but its accumulators occupy 128 tensor-memory
// columns per CTA, which caps the CTAs per SM; measured slower on the 130^3 grid), 0
// (IMGM_NET_TC=0) the CUDA-core FP32 loops (k_conv).  The kernels' shared memory is opted in
// once per process.
int net_tc_mode() {
    static const int mode = [] {
        const char* v = std::getenv("IMGM_NET_TC");
        if (v && v[0] == '0') return 0;
        if (v && std::atoi(v) == 48) return 2;
        return 1;
    }();
    static bool attr = false;
    if (mode > 0 && !attr) {
        cudaFuncSetAttribute(k_conv16_tc<uint16_t, 1, NET_C, EPI_RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TC_SMEM);
        cudaFuncSetAttribute(k_conv16_tc<uint16_t, NET_C, NET_C, EPI_RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TC_SMEM);
        cudaFuncSetAttribute(k_conv16_tc<uint16_t, NET_C, 1, EPI_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
        cudaFuncSetAttribute(k_conv16_tc<float, NET_C, NET_C, EPI_GATE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TC_SMEM);
        cudaFuncSetAttribute(k_conv_tcz<uint16_t, 1, NET_C, EPI_RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TCZ_SMEM);
        cudaFuncSetAttribute(k_conv_tcz<uint16_t, NET_C, NET_C, EPI_RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TCZ_SMEM);
        cudaFuncSetAttribute(k_conv_tcz<uint16_t, NET_C, 1, EPI_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TCZ_SMEM);
        cudaFuncSetAttribute(k_conv_tcz<float, NET_C, NET_C, EPI_GATE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TCZ_SMEM);
        attr = true;
    }
    return mode;
}

// one tensor-core convolution over the grid of ws in the chosen form
template <typename TIN, int CI, int CO, int EPI>
cudaError_t conv_tc(int mode, const NetWorkspace& ws, const TIN* x, const uint16_t* w, const uint16_t* gate,
                    const uint8_t* mask, uint16_t* yb, float* yf, double* yd, cudaStream_t s) {
    const int zc = mode == 2 ? TCZ_ZC : TC_ZC;
    const int64_t g = (int64_t)((ws.nx + TC_PX - 1) / TC_PX) * ((ws.ny + TC_PY - 1) / TC_PY) * ((ws.nz + zc - 1) / zc);
    if (g <= 0 || g > 2147483647LL) return cudaErrorInvalidValue;
    if (mode == 2)
        k_conv_tcz<TIN, CI, CO, EPI><<<(unsigned)g, TC_THREADS, TCZ_SMEM, s>>>(x, w, gate, mask, yb, yf, yd, ws.nx, ws.ny,
                                                                             ws.nz, ws.err);
    else
        k_conv16_tc<TIN, CI, CO, EPI><<<(unsigned)g, TC_THREADS, TC_SMEM, s>>>(x, w, gate, mask, yb, yf, yd, ws.nx,
                                                                             ws.ny, ws.nz, ws.err);
    return cudaGetLastError();
}


int grid_for(int64_t work, int per_block, int max_per_sm) {
    const int64_t want = (work + per_block - 1) / per_block;
    const int64_t cap = (int64_t)max_per_sm * sm_count();
    return (int)std::max<int64_t>(1, std::min(want, cap));
}

int elementwise_grid(int64_t n) { return grid_for(n, RTPB, 8); }

}  // namespace

cudaError_t NetWorkspace::ensure(int nx_, int ny_, int nz_, bool train_) {
    const int64_t nvox = (int64_t)nx_ * ny_ * nz_;
    if (nvox > cap || (train_ && !train)) {
        release();
        const int64_t n = std::max<int64_t>(nvox, 1);
        cudaError_t e;
        if ((e = cudaMalloc(&a0, n * sizeof(uint16_t))) != cudaSuccess) return e;
        if ((e = cudaMalloc(&a1, n * NET_C * sizeof(uint16_t))) != cudaSuccess) return e;
        if ((e = cudaMalloc(&a2, n * NET_C * sizeof(uint16_t))) != cudaSuccess) return e;
        if ((e = cudaMalloc(&partial, 2 * NET_PARTIALS * sizeof(double))) != cudaSuccess) return e;
        if ((e = cudaMalloc(&err, sizeof(int))) != cudaSuccess) return e;
        if ((e = cudaMemset(err, 0, sizeof(int))) != cudaSuccess) return e;
        if (train_) {
            if ((e = cudaMalloc(&o, n * sizeof(float))) != cudaSuccess) return e;
            if ((e = cudaMalloc(&d3, n * sizeof(float))) != cudaSuccess) return e;
            if ((e = cudaMalloc(&d2, n * NET_C * sizeof(float))) != cudaSuccess) return e;
            if ((e = cudaMalloc(&d1, n * NET_C * sizeof(float))) != cudaSuccess) return e;
            // per-block weight-gradient shares: at most 4 blocks per SM (grid_for) x 27 x 16 x 16
            if ((e = cudaMalloc(&wpart, (size_t)4 * sm_count() * 27 * NET_C * NET_C * sizeof(float))) != cudaSuccess)
                return e;
        }
        cap = n;
        train = train_;
    }
    nx = nx_, ny = ny_, nz = nz_;
    return cudaSuccess;
}

void NetWorkspace::release() {
    for (void* p : {(void*)a0, (void*)a1, (void*)a2, (void*)o, (void*)d3, (void*)d2, (void*)d1, (void*)wpart,
                    (void*)partial, (void*)err})
        if (p) cudaFree(p);
    a0 = a1 = a2 = nullptr;
    err = nullptr;
    o = d3 = d2 = d1 = wpart = nullptr;
    partial = nullptr;
    cap = 0;
    train = false;
}

cudaError_t net_convert(const float* w, uint16_t* wb, uint16_t* wbt, cudaStream_t s) {
    k_adam<<<(NET_NW + 255) / 256, 256, 0, s>>>(const_cast<float*>(w), nullptr, nullptr, nullptr, wb, wbt, 0.f, 0.f,
                                                0.f, 0.f, 0.f, 0.f, 0);
    add_launches(1);
    return cudaGetLastError();
}

cudaError_t net_forward(const uint16_t* wb, NetWorkspace& ws, const double* in, const uint8_t* mask, double in_scale,
                        double* out64, float* out32, cudaStream_t s) {
    const int64_t nvox = (int64_t)ws.nx * ws.ny * ws.nz;
    if (nvox == 0) return cudaSuccess;
    const int gc = grid_for(nvox, CTPB, 16);
    k_pack<<<elementwise_grid(nvox), RTPB, 0, s>>>(nvox, in, mask, in_scale, ws.a0);
    if (const int mode = net_tc_mode()) {
        cudaError_t e;
        if ((e = conv_tc<uint16_t, 1, NET_C, EPI_RELU>(mode, ws, ws.a0, wb, nullptr, nullptr, ws.a1, nullptr, nullptr,
                                                       s)) != cudaSuccess)
            return e;
        if ((e = conv_tc<uint16_t, NET_C, NET_C, EPI_RELU>(mode, ws, ws.a1, wb + NET_OFF2, nullptr, nullptr, ws.a2,
                                                           nullptr, nullptr, s)) != cudaSuccess)
            return e;
        if ((e = conv_tc<uint16_t, NET_C, 1, EPI_OUT>(mode, ws, ws.a2, wb + NET_OFF3, nullptr, mask, nullptr, out32,
                                                      out64, s)) != cudaSuccess)
            return e;
    } else {
        k_conv<1, NET_C, uint16_t, EPI_RELU><<<gc, CTPB, 0, s>>>(ws.a0, wb, nullptr, nullptr, ws.a1, nullptr, nullptr,
                                                                 ws.nx, ws.ny, ws.nz);
        k_conv<NET_C, NET_C, uint16_t, EPI_RELU><<<gc, CTPB, 0, s>>>(ws.a1, wb + NET_OFF2, nullptr, nullptr, ws.a2,
                                                                     nullptr, nullptr, ws.nx, ws.ny, ws.nz);
        k_conv<NET_C, 1, uint16_t, EPI_OUT><<<gc, CTPB, 0, s>>>(ws.a2, wb + NET_OFF3, nullptr, mask, nullptr, out32,
                                                                out64, ws.nx, ws.ny, ws.nz);
    }
    add_launches(4);
    return cudaGetLastError();
}

cudaError_t net_backward(const uint16_t* wbt, NetWorkspace& ws, const double* target, const uint8_t* mask,
                         double scale, float* grad, double* loss, cudaStream_t s) {
    const int64_t nvox = (int64_t)ws.nx * ws.ny * ws.nz;
    if (nvox == 0) return cudaSuccess;
    const int gc = grid_for(nvox, CTPB, 16);
    k_loss<<<elementwise_grid(nvox), RTPB, 0, s>>>(nvox, ws.o, target, mask, scale, ws.d3, loss);
    // layer 3: dW3 from (d3, a2); d2 = (W3^T d3) where a2 > 0
    const int g13 = grid_for(nvox, (WTPB / NET_C) * 32, 4), g2 = grid_for(nvox, 32, 4);
    k_wgrad<NET_C, 1><<<g13, WTPB, 0, s>>>(ws.d3, ws.a2, ws.wpart, ws.nx, ws.ny, ws.nz);
    k_wsum<<<(27 * NET_C + RTPB - 1) / RTPB, RTPB, 0, s>>>(ws.wpart, g13, 27 * NET_C, grad + NET_OFF3);
    k_conv<1, NET_C, float, EPI_GATE><<<gc, CTPB, 0, s>>>(ws.d3, wbt + NET_OFF3, ws.a2, nullptr, nullptr, ws.d2,
                                                          nullptr, ws.nx, ws.ny, ws.nz);
    // layer 2: dW2 from (d2, a1); d1 = (W2^T d2) where a1 > 0
    k_wgrad<NET_C, NET_C><<<g2, WTPB, 0, s>>>(ws.d2, ws.a1, ws.wpart, ws.nx, ws.ny, ws.nz);
    k_wsum<<<(27 * NET_C * NET_C + RTPB - 1) / RTPB, RTPB, 0, s>>>(ws.wpart, g2, 27 * NET_C * NET_C, grad + NET_OFF2);
    if (const int mode = net_tc_mode()) {
        cudaError_t e = conv_tc<float, NET_C, NET_C, EPI_GATE>(mode, ws, ws.d2, wbt + NET_OFF2, ws.a1, nullptr, nullptr,
                                                               ws.d1, nullptr, s);
        if (e != cudaSuccess) return e;
    } else {
        k_conv<NET_C, NET_C, float, EPI_GATE><<<gc, CTPB, 0, s>>>(ws.d2, wbt + NET_OFF2, ws.a1, nullptr, nullptr,
                                                                  ws.d1, nullptr, ws.nx, ws.ny, ws.nz);
    }
    // layer 1: dW1 from (d1, a0)
    k_wgrad<1, NET_C><<<g13, WTPB, 0, s>>>(ws.d1, ws.a0, ws.wpart, ws.nx, ws.ny, ws.nz);
    k_wsum<<<(27 * NET_C + RTPB - 1) / RTPB, RTPB, 0, s>>>(ws.wpart, g13, 27 * NET_C, grad);
    add_launches(9);
    return cudaGetLastError();
}

cudaError_t net_adam(float* w, const float* g, float* m, float* v, uint16_t* wb, uint16_t* wbt, float lr, float beta1,
                     float beta2, float eps, float c1, float c2, cudaStream_t s) {
    k_adam<<<(NET_NW + 255) / 256, 256, 0, s>>>(w, g, m, v, wb, wbt, lr, beta1, beta2, eps, c1, c2, 1);
    add_launches(1);
    return cudaGetLastError();
}

cudaError_t stage_update(int64_t n, const double* r1, const double* c, const double* Ac, double* z, double* partial,
                         double* omega_out, cudaStream_t s) {
    k_dots<<<NET_PARTIALS, RTPB, 0, s>>>(n, r1, c, c, Ac, partial);
    k_stage_axpy<<<elementwise_grid(n), RTPB, 0, s>>>(n, z, c, partial, omega_out);
    add_launches(2);
    return cudaGetLastError();
}

cudaError_t pair_error(int64_t n, const double* e0, const double* z, double* e1, cudaStream_t s) {
    k_sub<<<elementwise_grid(n), RTPB, 0, s>>>(n, e0, z, e1);
    add_launches(1);
    return cudaGetLastError();
}

cudaError_t pair_normalise(int64_t n, double* r, double* e, double count, double* partial, double* r_rms,
                           cudaStream_t s) {
    k_dots<<<NET_PARTIALS, RTPB, 0, s>>>(n, r, r, e, e, partial);
    k_pair_scale<<<elementwise_grid(n), RTPB, 0, s>>>(n, r, e, count, partial, r_rms);
    add_launches(2);
    return cudaGetLastError();
}

}  // namespace imgm
