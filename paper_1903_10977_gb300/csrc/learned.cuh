// Learned correction stage: a three-layer 3-D convolutional network on the background
// grid of the finest level's basis functions, its training kernels, and the stage that
// adds its proposal to the V-cycle's output with the energy-minimising step.  The paper
// has no learned component; the network is an extra stage inside flexible CG beside the
// V-cycle of Algorithm 1.
//
// Network: 1 -> 16 -> 16 -> 1 channels, 3 x 3 x 3 kernels, no biases, zero padding, ReLU
// after the first two layers.  Weights are kept in FP32 (master copy, Adam moments) and
// read by the convolutions as bfloat16; activations are stored as bfloat16 with
// channels innermost ([voxel][channel]); sums accumulate in FP32.  Layer l has weights
// W_l[tap][out][in] with tap = 9 (dz + 1) + 3 (dy + 1) + (dx + 1) and voxel index
// v = x + nx (y + ny z), the order of the basis functions' flat index.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace imgm {

constexpr int NET_C = 16;
constexpr int NET_W1 = 27 * NET_C;            // layer 1: [27][16][1]
constexpr int NET_W2 = 27 * NET_C * NET_C;    // layer 2: [27][16][16]
constexpr int NET_W3 = 27 * NET_C;            // layer 3: [27][1][16]
constexpr int NET_OFF2 = NET_W1;
constexpr int NET_OFF3 = NET_W1 + NET_W2;
constexpr int NET_NW = NET_W1 + NET_W2 + NET_W3;   // 7776
constexpr int NET_PARTIALS = 256;                  // blocks of the stage's reductions

// Activations and gradients of one grid (device memory, bf16 stored as uint16_t).
struct NetWorkspace {
    int nx = 0, ny = 0, nz = 0;
    int64_t cap = 0;                 // voxels allocated
    bool train = false;              // gradient buffers allocated
    uint16_t *a0 = nullptr, *a1 = nullptr, *a2 = nullptr;   // input [v], hidden [v][16]
    float* o = nullptr;              // output [v] (training)
    float *d3 = nullptr, *d2 = nullptr, *d1 = nullptr;      // dL/d(out) [v], dL/d(a2), dL/d(a1) [v][16]
    float* wpart = nullptr;          // per-block weight-gradient shares [block][27 x 16 x 16] (training)
    double* partial = nullptr;       // [2 * NET_PARTIALS]
    int* err = nullptr;              // set by a tensor-core convolution whose wait gave up
    cudaError_t ensure(int nx, int ny, int nz, bool train);
    void release();
};

// wb = bf16(w) in the forward layout, wbt = the layers' transposed, tap-reversed bf16
// weights ([26 - tap][in][out]) that turn the input gradient into a forward convolution.
cudaError_t net_convert(const float* w, uint16_t* wb, uint16_t* wbt, cudaStream_t s);

// N(in_scale in) on the grid of ws: a0 = bf16(float(in_scale in)) on the mask (mask null:
// every voxel), a1, a2 stored; the output goes to out64 (FP64, zero off the mask) and/or out32.
cudaError_t net_forward(const uint16_t* wb, NetWorkspace& ws, const double* in, const uint8_t* mask, double in_scale,
                        double* out64, float* out32, cudaStream_t s);

// After net_forward(..., out32 = ws.o): grad += dL/dw of L = scale sum_v m_v (o_v - t_v)^2
// and loss[0] += L (device double).
cudaError_t net_backward(const uint16_t* wbt, NetWorkspace& ws, const double* target, const uint8_t* mask,
                         double scale, float* grad, double* loss, cudaStream_t s);

// Adam step on the FP32 master weights (c1 = 1/(1 - beta1^t), c2 = 1/(1 - beta2^t)),
// then the bf16 copies.
cudaError_t net_adam(float* w, const float* g, float* m, float* v, uint16_t* wb, uint16_t* wbt, float lr, float beta1,
                     float beta2, float eps, float c1, float c2, cudaStream_t s);

// z += omega c with omega = (r1 . c) / (c . Ac) (0 unless c . Ac > 0 and finite);
// omega_out (device, may be null) receives omega.
cudaError_t stage_update(int64_t n, const double* r1, const double* c, const double* Ac, double* z, double* partial,
                         double* omega_out, cudaStream_t s);

// e1 = e0 - z (e1 may alias neither input)
cudaError_t pair_error(int64_t n, const double* e0, const double* z, double* e1, cudaStream_t s);
// r, e /= sqrt(sum(e^2) / count); r_rms (device, may be null) = sqrt(sum(r^2) / count) afterwards
cudaError_t pair_normalise(int64_t n, double* r, double* e, double count, double* partial, double* r_rms,
                           cudaStream_t s);

}  // namespace imgm
