// FP64 instances of the 3-D z-marching operator apply (the CG's and the FP64 V-cycle's),
// with the CG's A p and p^T A p in one launch (Sec. 3.2: the V-cycle as CG preconditioner).
#include "apply3d.cuh"

namespace imgm {

bool zm_applies(int m) { return use_zm_3d(m); }

cudaError_t apply_zm3d(const DevLevelT<double>& L, int mode, const double* x, const double* rin, double* out,
                       double* xs, double gamma, const int* done, cudaStream_t s) {
    if (L.p == 1) return launch_zm3d<double, 1>(L, mode, x, rin, out, xs, gamma, done, s);
    if (L.p == 2) return launch_zm3d<double, 2>(L, mode, x, rin, out, xs, gamma, done, s);
    if (L.p == 3) return launch_zm3d<double, 3>(L, mode, x, rin, out, xs, gamma, done, s);
    return cudaErrorInvalidValue;
}

cudaError_t apply_zm3d_pq(const DevLevel& L, const double* p, double* q, double* partial, PcgState* st,
                          cudaStream_t s) {
    if (L.tile_ctr == nullptr || (L.nb > 0 && L.band_row == nullptr)) return cudaErrorInvalidValue;
    const int yt = zm_yt(L.m, L.zm_yt);
    const ZmShape sh = zm_shape(L.m, L.nb, L.p, yt, L.zm_zc);
    const int g = zm_grid(sh, std::min(2 * num_sms(), reduction_blocks()));
#define IMGM_ZM_PQ(PP, YY)                                                                                      \
    launch_pdl(k_apply_zm3d<double, PP, APPLY, true, YY, false>, g, TPB, 0, s, L, p, nullptr, q, nullptr, 0.0, \
               &st->done, partial, st, sh)
    if (L.p == 1) { if (yt == 2) IMGM_ZM_PQ(1, 2); else IMGM_ZM_PQ(1, 1); }
    else if (L.p == 2) { if (yt == 2) IMGM_ZM_PQ(2, 2); else IMGM_ZM_PQ(2, 1); }
    else if (L.p == 3) { if (yt == 2) IMGM_ZM_PQ(3, 2); else IMGM_ZM_PQ(3, 1); }
    else return cudaErrorInvalidValue;
#undef IMGM_ZM_PQ
    return cudaGetLastError();
}

}  // namespace imgm
