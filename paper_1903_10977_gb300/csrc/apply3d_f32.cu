// FP32 instances of the 3-D z-marching operator apply (the mixed-precision V-cycle's, in
// Jacobi-scaled variables): registers, per-warp staging or the CTA form, per the level's
// autotuned choice.
#include "apply3d.cuh"

namespace imgm {

cudaError_t apply_zm3d(const DevLevelT<float>& L, int mode, const float* x, const float* rin, float* out, float* xs,
                       float gamma, const int* done, cudaStream_t s) {
    if (L.p == 1) return launch_zm3d<float, 1>(L, mode, x, rin, out, xs, gamma, done, s);
    if (L.p == 2) return launch_zm3d<float, 2>(L, mode, x, rin, out, xs, gamma, done, s);
    if (L.p == 3) return launch_zm3d<float, 3>(L, mode, x, rin, out, xs, gamma, done, s);
    return cudaErrorInvalidValue;
}

}  // namespace imgm
