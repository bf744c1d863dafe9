// Device helpers and the launch path shared by the kernel translation units (kernels.cu, and
// apply3d_f64.cu / apply3d_f32.cu, which hold the instances of the 3-D z-marching apply so
// that the library compiles in parallel).  Everything below the declarations lives in an
// unnamed namespace: each unit has its own copy.
#pragma once
#include "kernels.cuh"

#include <algorithm>
#include <cstdlib>
#include <utility>

namespace imgm {

// programmatic launches allowed, and kernels issued, by this host thread (kernels.cu)
extern thread_local bool t_pdl;
extern thread_local int64_t t_launches;

// the 3-D z-marching apply of one level (mode APPLY / RESID / RESID_SMOOTH) and, FP64, the
// CG's A p with p^T A p in the same launch
cudaError_t apply_zm3d(const DevLevelT<double>& L, int mode, const double* x, const double* rin, double* out,
                       double* xs, double gamma, const int* done, cudaStream_t s);
cudaError_t apply_zm3d(const DevLevelT<float>& L, int mode, const float* x, const float* rin, float* out, float* xs,
                       float gamma, const int* done, cudaStream_t s);
cudaError_t apply_zm3d_pq(const DevLevel& L, const double* p, double* q, double* partial, PcgState* st,
                          cudaStream_t s);
// the cluster-resident coarse V-cycle kernel of degree p for 2-D and for 3-D levels
const void* ds_kernel_2d(int p);
const void* ds_kernel_3d(int p);

namespace {

constexpr int TPB = 256;

// Programmatic dependent launch: every kernel is launched with programmatic stream
// serialisation allowed, so that the blocks of the next kernel in the stream (or graph)
// are scheduled while this one drains instead of after a full launch round trip.  Each
// kernel first waits until its predecessor has completed and its writes are visible
// (griddepcontrol.wait returns at once when there is no programmatic predecessor), then
// lets its own successor launch.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Read-only data (level tables, stored coefficients, block inverses, scales): never
// written on the device after setup, so it may take the non-coherent cached path.
// The row tables are read with plain loads.
template <typename T>
__device__ __forceinline__ T ro(const T* p) {
    return __ldg(p);
}
__device__ __forceinline__ int64_t ro(const int64_t* p) {
    return (int64_t)__ldg(reinterpret_cast<const long long*>(p));
}

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

// Two sums at once (partials at [0, G) and [G, 2G)); the last block sums both in parallel.
__device__ __forceinline__ bool finish_reduction2(double v1, double v2, double* partial, unsigned int* ticket,
                                                  double* t1, double* t2) {
    __shared__ double ws[32];
    __shared__ bool last;
    double b1 = block_sum(v1, ws);
    double b2 = block_sum(v2, ws);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = b1;
        partial[gridDim.x + blockIdx.x] = b2;
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s1 = 0.0, s2 = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += TPB) {
        s1 += ((volatile double*)partial)[b];
        s2 += ((volatile double*)partial)[gridDim.x + b];
    }
    s1 = block_sum(s1, ws);
    s2 = block_sum(s2, ws);
    if (threadIdx.x == 0) {
        *t1 = s1;
        *t2 = s2;
        *ticket = 0u;
    }
    return true;
}

template <typename T>
__device__ __forceinline__ T fmaT(T a, T b, T c) {
    return fma(a, b, c);
}

struct ZmShape {
    int sx, sy, sz;                      // tensor tasks along x (strips), y (segments), z (chunks)
    int zc;                              // planes per chunk
    unsigned int ntensor, ntotal;        // tensor tasks; all tasks (tensor + stored)
};

// tensor tasks a marching apply aims for: a task is one warp's sequential walk, so too few
// leave the SMs latency-bound
constexpr int ZM_TASKS = 3600;

// Whether the next launch on s may carry the programmatic-serialisation attribute: always
// outside stream capture; under capture only when every node it will depend on is a
// kernel node (a programmatic edge joins two kernels).
bool pdl_allowed(cudaStream_t s) {
    if (!t_pdl) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, nullptr, &nd) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (cs != cudaStreamCaptureStatusActive) return true;
    for (size_t k = 0; k < nd; ++k) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(deps[k], &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) {
            cudaGetLastError();
            return false;
        }
    }
    return true;
}

// Every kernel goes through here: programmatic stream serialisation lets the kernel
// launch while its predecessor drains (each kernel starts with pdl_begin()).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_allowed(s) ? 1 : 0;
    ++t_launches;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
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

int zm_grid(const ZmShape& sh, int cap) {
    int64_t g = std::min<int64_t>((sh.ntotal + TPB / 32 - 1) / (TPB / 32), cap);
    if (const char* v = std::getenv("IMGM_ZM_BLOCKS")) {
        const int k = std::atoi(v);
        if (k > 0) g = std::min<int64_t>(g, k);
    }
    return (int)std::max<int64_t>(g, 1);
}

}  // namespace
}  // namespace imgm
