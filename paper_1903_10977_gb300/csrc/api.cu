// C-ABI of the immersed multigrid-preconditioned CG library (declarations in imgm.h).
//
// imgm_setup builds the hierarchy on the host (setup.cpp) and uploads it; the GPU entry
// points enqueue the kernels of kernels.cu.  The CG solve runs as one CUDA graph: the
// start-up kernels, a device-side while loop (conditional graph node) over one CG
// iteration with its V-cycle, and the final residual check.  The loop condition is set
// by a kernel from the device-held convergence flag, so the host waits only once.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>
#include <type_traits>

#include "../../include/imgm.h"
#include "kernels.cuh"
#include "learned.cuh"
#include "setup.hpp"

using imgm::DevLevel;
using imgm::PcgState;

namespace {

thread_local std::string g_setup_error;

struct LevelDev {
    DevLevel d;
    double* x = nullptr;   // V-cycle iterate (level < L) / unused on the finest level
    double* r = nullptr;   // restricted residual (level < L)
    double* t = nullptr;   // residual after smoothing
    double* e = nullptr;   // prolongated correction
    // the same in FP32 and Jacobi-scaled variables (mixed-precision V-cycle)
    imgm::DevLevelT<float> fd;
    float *fx = nullptr, *fr = nullptr, *ft = nullptr, *fe = nullptr;
    // multiplicative Schwarz: colour ranges (host) and the one-function blocks (device)
    int ncolour = 0;
    std::vector<int64_t> blk_cptr, sg_cptr;
    int32_t* sg_row = nullptr;
    double* sg_inv = nullptr;
    float* f_sg_inv = nullptr;
    imgm_level_info info{};
};

// typed access to a level's data and V-cycle vectors
template <typename T>
struct Acc;
template <>
struct Acc<double> {
    static const imgm::DevLevelT<double>& d(const LevelDev& L) { return L.d; }
    static double* x(LevelDev& L) { return L.x; }
    static double* r(LevelDev& L) { return L.r; }
    static double* t(LevelDev& L) { return L.t; }
    static double* e(LevelDev& L) { return L.e; }
    static const double* sg_inv(const LevelDev& L) { return L.sg_inv; }
};
template <>
struct Acc<float> {
    static const imgm::DevLevelT<float>& d(const LevelDev& L) { return L.fd; }
    static float* x(LevelDev& L) { return L.fx; }
    static float* r(LevelDev& L) { return L.fr; }
    static float* t(LevelDev& L) { return L.ft; }
    static float* e(LevelDev& L) { return L.fe; }
    static const float* sg_inv(const LevelDev& L) { return L.f_sg_inv; }
};

}  // namespace

// What every solve context of one problem shares: the host hierarchy and the device
// tables (operator rows, blocks, transfers, coarse inverse, right-hand side).  Freed with
// the last handle that refers to it.
struct SharedData {
    imgm::Hierarchy H;
    std::vector<void*> allocs;
    ~SharedData() {
        for (void* v : allocs) cudaFree(v);
    }
};

// The learned stage's network: FP32 master weights, gradient and Adam moments, the bf16
// copies the convolutions read, and the activations of the last standalone call.
struct imgm_net {
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    uint16_t *wb = nullptr, *wbt = nullptr;
    int64_t t = 0;                 // Adam steps taken
    int attached = 0;              // handles holding it plus batches whose graph recorded it
    imgm::NetWorkspace ws;
    ~imgm_net() {
        for (void* p : {(void*)w, (void*)g, (void*)m, (void*)v, (void*)wb, (void*)wbt})
            if (p) cudaFree(p);
        ws.release();
    }
};

struct imgm_handle {
    std::shared_ptr<SharedData> sh;
    imgm::Hierarchy& H;
    explicit imgm_handle(std::shared_ptr<SharedData> s) : sh(std::move(s)), H(sh->H) {}
    bool on_device = false;
    int dim = 2, p = 2, L = 2;
    double gamma = 0.0;
    int smoother = 0;          // 0 additive, 1 coloured multiplicative Schwarz
    double gamma_diag = 0.0;   // factor of the diagonal start x = gamma_diag dinv r (0: x starts at 0)
    std::vector<LevelDev> lv;          // index 0 = level 1
    std::vector<void*> allocs;         // this context's vectors and scratch
    int32_t* c_rows = nullptr;
    double* c_inv = nullptr;
    float* f_c_inv = nullptr;
    int nc = 0;
    int precision = 0;                 // 0: FP64 V-cycle, 1: FP32 V-cycle in the FP64 CG
    float *zf = nullptr, *rf = nullptr, *zpf = nullptr;   // finest FP32 V-cycle output, input, previous output
    // FP32 V-cycle: levels 0..ds_top on one thread-block cluster, resident in distributed
    // shared memory (-1: every level as separate launches)
    int ds_top = -1;
    imgm::DsVcycle dsv{};
    std::vector<const unsigned char*> ds_images;   // per top: the blocks' images (shared tables), or null
    std::vector<imgm::DsVcycle> ds_cand;           // per top: launch parameters of this context
    double* b = nullptr;               // built-in right-hand side
    // CG state
    double *cx = nullptr, *cr = nullptr, *cp = nullptr, *cq = nullptr, *cz = nullptr, *cb = nullptr;
    double* czp = nullptr;             // previous preconditioned residual (flexible CG, precision 2)
    double* hist = nullptr;
    int hist_cap = 0;
    double* partial = nullptr;
    PcgState* st = nullptr;
    double* partial_aux = nullptr;     // reductions outside the CG solve
    PcgState* st_aux = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph_failed = false;
    cudaStream_t capture = nullptr;    // the solve graph is captured here (the caller's stream may be the legacy one)
    int64_t graph_kernels[3] = {0, 0, 0};   // kernel nodes of the solve graph: start, loop body, finish
    // learned stage (dim 3, FP64 V-cycle output): the attached network, its activations on
    // the finest grid, the stage's vectors (r1 = r - A z, c = N(r1), A c), the active mask
    imgm_net* net = nullptr;
    // truncated flexible CG (imgm_set_fcg): m stored directions and their images, m x N each
    int fcg_m = 0, fcg_cap = 0;
    double *fcg_P = nullptr, *fcg_Q = nullptr;
    imgm::NetWorkspace lws;
    double *l_r1 = nullptr, *l_c = nullptr, *l_q = nullptr;
    uint8_t* l_mask = nullptr;
    std::string err;

    template <class T>
    cudaError_t alloc(T** p, size_t count) {
        void* v = nullptr;
        cudaError_t e = cudaMalloc(&v, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
        if (e != cudaSuccess) return e;
        allocs.push_back(v);
        *p = (T*)v;
        return cudaSuccess;
    }
    // read-only tables: shared by every context of the problem
    template <class T>
    cudaError_t upload(T** p, const std::vector<T>& h) {
        void* v = nullptr;
        cudaError_t e = cudaMalloc(&v, h.size() * sizeof(T) > 0 ? h.size() * sizeof(T) : 16);
        if (e != cudaSuccess) return e;
        sh->allocs.push_back(v);
        *p = (T*)v;
        if (h.empty()) return cudaSuccess;
        return cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    }
    ~imgm_handle() {
        if (net) net->attached -= 1;
        if (exec) cudaGraphExecDestroy(exec);
        if (capture) cudaStreamDestroy(capture);
        if (graph) cudaGraphDestroy(graph);
        lws.release();
        for (void* v : allocs) cudaFree(v);
    }
};

namespace {

// ---- scratch of imgm_residual_norm2_noalloc -------------------------------------
// Some callers cannot call cudaMalloc while they run: a process whose device memory is
// reserved up front by a caching allocator (a new cudaMalloc then fails or forces the
// cache to be released), or a latency-critical loop in which cudaMalloc's implicit
// device-wide synchronisation would stall work on other streams.  For them the residual
// norm has a variant whose scratch is this file-scope array, which exists on every GPU
// that loads the library until the process exits: a CG state record (the reduction
// ticket and the result), the per-block partial sums, and the residual vector of at
// most NOALLOC_MAX_ROWS rows (4 MiB in all).
constexpr int64_t NOALLOC_MAX_ROWS = int64_t(1) << 19;
constexpr int64_t NOALLOC_MAX_PARTIALS = 4096;
constexpr int64_t NOALLOC_STATE_DOUBLES = 32;   // 256 bytes, holds one PcgState
static_assert(sizeof(PcgState) <= NOALLOC_STATE_DOUBLES * sizeof(double), "state slot too small");
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_STATE_DOUBLES + NOALLOC_MAX_PARTIALS + NOALLOC_MAX_ROWS];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

int fail(imgm_handle* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    else g_setup_error = msg;
    return code;
}

// A tensor-core convolution whose bounded wait gave up sets the workspace's flag (it never
// hangs the GPU); a call that waits for the device reads and clears it.
int net_wait_status(imgm_handle* h, const imgm::NetWorkspace& ws) {
    if (!ws.err) return IMGM_OK;
    int flag = 0;
    if (cudaMemcpy(&flag, ws.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(h, IMGM_ERR_CUDA, "reading the network's status");
    if (!flag) return IMGM_OK;
    cudaMemset(ws.err, 0, sizeof(int));
    return fail(h, IMGM_ERR_CUDA, "a tensor-core convolution gave up waiting for its matrix multiplies");
}

int cuda_fail(imgm_handle* h, cudaError_t e, const char* where) {
    return fail(h, IMGM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                   \
    do {                                                  \
        cudaError_t _e = (call);                          \
        if (_e != cudaSuccess) return cuda_fail(h, _e, where); \
    } while (0)

int check_level(imgm_handle* h, int level, int min_level) {
    if (!h) return IMGM_ERR_INVALID;
    if (!h->on_device) return fail(h, IMGM_ERR_INVALID, "handle has no device data");
    if (level < min_level || level > h->L) return fail(h, IMGM_ERR_INVALID, "level out of range");
    return IMGM_OK;
}

template <typename T>
const T* coarse_inverse(const imgm_handle* h);
template <>
const double* coarse_inverse<double>(const imgm_handle* h) { return h->c_inv; }
template <>
const float* coarse_inverse<float>(const imgm_handle* h) { return h->f_c_inv; }

// One V-cycle (Algorithm 1) from the finest level.  On entry z = gamma * dinv .* r
// (the diagonal part of the first smoothing step); on exit z = B r.  r is not modified.
// T = float runs it in FP32 on the Jacobi-scaled data (r and z then are r^, z^).
template <typename T>
int cluster_top(const imgm_handle* h);
template <>
int cluster_top<double>(const imgm_handle*) { return -1; }
template <>
int cluster_top<float>(const imgm_handle* h) { return h->ds_top; }

// one colour c of the multiplicative Schwarz sweep on level F: x += B_c r
template <typename T>
cudaError_t colour_step(LevelDev& F, int c, const T* r, T* x, const int* done, cudaStream_t s) {
    using A = Acc<T>;
    const int64_t s0 = F.sg_cptr[c];
    return imgm::launch_colour_smooth<T>(A::d(F), F.blk_cptr[c], F.blk_cptr[c + 1], F.sg_row + s0, A::sg_inv(F) + s0,
                                         F.sg_cptr[c + 1] - s0, r, x, done, s);
}

// The V-cycle with coloured multiplicative Schwarz (Sec. 3.4).  On entry z = 0.  Each
// level: a forward sweep over the colours from x = 0, the residual recomputed after every
// colour (so that line 5 falls out of the last one), restriction, coarse correction,
// t -= A e (line 10), and the reversed sweep on the current residual (line 12).
template <typename T>
cudaError_t enqueue_vcycle_mult(imgm_handle* h, const T* r, T* z, const int*, cudaStream_t s) {
    using A = Acc<T>;
    const int* done = nullptr;   // see enqueue_vcycle
    const int L = h->L;
    cudaError_t e;
    for (int li = L - 1; li >= 1; --li) {
        LevelDev& F = h->lv[li];
        LevelDev& C = h->lv[li - 1];
        const T* rl = (li == L - 1) ? r : A::r(F);
        T* xl = (li == L - 1) ? z : A::x(F);
        for (int c = 0; c < F.ncolour; ++c) {
            if ((e = colour_step<T>(F, c, c == 0 ? rl : A::t(F), xl, done, s)) != cudaSuccess) return e;
            if ((e = imgm::launch_apply<T>(A::d(F), imgm::RESID, xl, rl, A::t(F), nullptr, 0.0, done, s)) != cudaSuccess)
                return e;
        }
        T* xc = (li - 1 >= 1) ? A::x(C) : nullptr;     // zeroed: the coarse sweep starts from 0
        if ((e = imgm::launch_restrict<T>(A::d(F), A::d(C), A::t(F), A::r(C), xc, 0.0, done, s)) != cudaSuccess) return e;
    }
    if ((e = imgm::launch_coarse<T>(h->c_rows, coarse_inverse<T>(h), h->nc, A::r(h->lv[0]), A::x(h->lv[0]), done, s)) !=
        cudaSuccess)
        return e;
    for (int li = 1; li <= L - 1; ++li) {
        LevelDev& F = h->lv[li];
        LevelDev& C = h->lv[li - 1];
        const T* rl = (li == L - 1) ? r : A::r(F);
        T* xl = (li == L - 1) ? z : A::x(F);
        if ((e = imgm::launch_prolong<T>(A::d(F), A::d(C), A::x(C), A::e(F), xl, done, s)) != cudaSuccess) return e;
        if ((e = imgm::launch_apply<T>(A::d(F), imgm::RESID, A::e(F), A::t(F), A::t(F), nullptr, 0.0, done, s)) !=
            cudaSuccess)
            return e;
        for (int c = F.ncolour - 1; c >= 0; --c) {
            if ((e = colour_step<T>(F, c, A::t(F), xl, done, s)) != cudaSuccess) return e;
            if (c > 0 &&
                (e = imgm::launch_apply<T>(A::d(F), imgm::RESID, xl, rl, A::t(F), nullptr, 0.0, done, s)) != cudaSuccess)
                return e;
        }
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t enqueue_vcycle_top(imgm_handle* h, int top, const T* r, T* z, cudaStream_t s) {
    const int* done = nullptr;
    using A = Acc<T>;
    const double g = h->gamma;
    cudaError_t e;
    const int ct = cluster_top<T>(h);
    if (ct >= 0) {
        // levels above the cluster's: separate kernels, then one cluster launch for the rest
        for (int li = top; li > ct; --li) {
            LevelDev& F = h->lv[li];
            LevelDev& C = h->lv[li - 1];
            const T* rl = (li == top) ? r : A::r(F);
            T* xl = (li == top) ? z : A::x(F);
            if ((e = imgm::launch_blocks<T>(A::d(F), rl, xl, g, done, s)) != cudaSuccess) return e;
            if ((e = imgm::launch_apply<T>(A::d(F), imgm::RESID, xl, rl, A::t(F), nullptr, g, done, s)) != cudaSuccess)
                return e;
            T* xc = (li - 1 >= 1) ? A::x(C) : nullptr;
            if ((e = imgm::launch_restrict<T>(A::d(F), A::d(C), A::t(F), A::r(C), xc, g, done, s)) != cudaSuccess)
                return e;
        }
        if ((e = imgm::launch_vcycle_dsmem(h->dim, h->p, h->dsv, s)) != cudaSuccess) return e;
        for (int li = ct + 1; li <= top; ++li) {
            LevelDev& F = h->lv[li];
            LevelDev& C = h->lv[li - 1];
            T* xl = (li == top) ? z : A::x(F);
            if ((e = imgm::launch_prolong<T>(A::d(F), A::d(C), A::x(C), A::e(F), xl, done, s)) != cudaSuccess)
                return e;
            if ((e = imgm::launch_apply<T>(A::d(F), imgm::RESID_SMOOTH, A::e(F), A::t(F), A::t(F), xl, g, done, s)) !=
                cudaSuccess)
                return e;
            if ((e = imgm::launch_blocks<T>(A::d(F), A::t(F), xl, g, done, s)) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    for (int li = top; li >= 1; --li) {
        LevelDev& F = h->lv[li];
        LevelDev& C = h->lv[li - 1];
        const T* rl = (li == top) ? r : A::r(F);
        T* xl = (li == top) ? z : A::x(F);
        // line 4: x = gamma M^{-1} r (the one-function blocks were applied by the producer of r)
        if ((e = imgm::launch_blocks<T>(A::d(F), rl, xl, g, done, s)) != cudaSuccess) return e;
        // line 5: t = r - A x
        if ((e = imgm::launch_apply<T>(A::d(F), imgm::RESID, xl, rl, A::t(F), nullptr, g, done, s)) != cudaSuccess)
            return e;
        // line 7: r_c = R t, and the diagonal part of the coarse pre-smoothing step
        T* xc = (li - 1 >= 1) ? A::x(C) : nullptr;
        if ((e = imgm::launch_restrict<T>(A::d(F), A::d(C), A::t(F), A::r(C), xc, g, done, s)) != cudaSuccess) return e;
    }
    // line 14: direct solve on level 1
    if ((e = imgm::launch_coarse<T>(h->c_rows, coarse_inverse<T>(h), h->nc, A::r(h->lv[0]), A::x(h->lv[0]), done, s)) !=
        cudaSuccess)
        return e;
    for (int li = 1; li <= top; ++li) {
        LevelDev& F = h->lv[li];
        LevelDev& C = h->lv[li - 1];
        T* xl = (li == top) ? z : A::x(F);
        // line 9: e = R^T x_c, x += e
        if ((e = imgm::launch_prolong<T>(A::d(F), A::d(C), A::x(C), A::e(F), xl, done, s)) != cudaSuccess) return e;
        // line 10: t -= A e; line 12 (one-function blocks): x += gamma dinv .* t
        if ((e = imgm::launch_apply<T>(A::d(F), imgm::RESID_SMOOTH, A::e(F), A::t(F), A::t(F), xl, g, done, s)) !=
            cudaSuccess)
            return e;
        // line 12 (stored blocks): x += gamma sum_j P_j A_j^{-1} P_j^T t
        if ((e = imgm::launch_blocks<T>(A::d(F), A::t(F), xl, g, done, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The V-cycle with its finest level in FP64 and the levels below it in FP32 on
// Jacobi-scaled data (precision 2): the finest level's residual and its restriction keep
// FP64, so the rounding of the coarse levels' input is that of a restricted FP64 residual.
// On entry z = gamma dinv .* r (FP64), as for the FP64 V-cycle.
cudaError_t enqueue_vcycle_hybrid(imgm_handle* h, const double* r, double* z, cudaStream_t s) {
    const int L = h->L;
    const double g = h->gamma;
    LevelDev& F = h->lv[L - 1];
    LevelDev& C = h->lv[L - 2];
    cudaError_t e;
    if ((e = imgm::launch_blocks<double>(F.d, r, z, g, nullptr, s)) != cudaSuccess) return e;
    if ((e = imgm::launch_apply<double>(F.d, imgm::RESID, z, r, F.t, nullptr, g, nullptr, s)) != cudaSuccess) return e;
    if ((e = imgm::launch_restrict_64to32(F.d, C.fd, F.t, C.fr, L - 2 >= 1 ? C.fx : nullptr, g, s)) != cudaSuccess)
        return e;
    if (L - 2 >= 1) {
        if ((e = enqueue_vcycle_top<float>(h, L - 2, C.fr, C.fx, s)) != cudaSuccess) return e;
    } else if ((e = imgm::launch_coarse<float>(h->c_rows, h->f_c_inv, h->nc, C.fr, C.fx, nullptr, s)) != cudaSuccess) {
        return e;
    }
    if ((e = imgm::launch_prolong_32to64(F.d, C.fd, C.fx, F.e, z, s)) != cudaSuccess) return e;
    if ((e = imgm::launch_apply<double>(F.d, imgm::RESID_SMOOTH, F.e, F.t, F.t, z, g, nullptr, s)) != cudaSuccess)
        return e;
    return imgm::launch_blocks<double>(F.d, F.t, z, g, nullptr, s);
}

template <typename T>
cudaError_t enqueue_vcycle(imgm_handle* h, const T* r, T* z, const int*, cudaStream_t s) {
    // The V-cycle kernels are not told the convergence flag: they touch only the V-cycle's
    // own vectors, so the one V-cycle after convergence is harmless, while reading the flag
    // would put a dependent memory round trip in front of every one of them.
    if (h->smoother == 1) return enqueue_vcycle_mult<T>(h, r, z, nullptr, s);
    if (std::is_same<T, double>::value && h->precision == 2)
        return enqueue_vcycle_hybrid(h, reinterpret_cast<const double*>(r), reinterpret_cast<double*>(z), s);
    return enqueue_vcycle_top<T>(h, h->L - 1, r, z, s);
}

// The learned stage on the FP64 V-cycle's output: z += omega N(r - A z) with the
// energy-minimising omega = (r1 . c) / (c . A c) (0 unless positive curvature).
cudaError_t enqueue_learned(imgm_handle* h, const double* r, double* z, double* omega_out, cudaStream_t s) {
    LevelDev& F = h->lv[h->L - 1];
    const int64_t N = F.d.N;
    cudaError_t e;
    if ((e = imgm::launch_apply<double>(F.d, imgm::RESID, z, r, h->l_r1, nullptr, h->gamma, nullptr, s)) != cudaSuccess)
        return e;
    if ((e = imgm::net_forward(h->net->wb, h->lws, h->l_r1, h->l_mask, 1.0, h->l_c, nullptr, s)) != cudaSuccess)
        return e;
    if ((e = imgm::launch_apply<double>(F.d, imgm::APPLY, h->l_c, nullptr, h->l_q, nullptr, 0.0, nullptr, s)) !=
        cudaSuccess)
        return e;
    return imgm::stage_update(N, h->l_r1, h->l_c, h->l_q, z, h->lws.partial, omega_out, s);
}

// The whole CG solve on the handle's own vectors (cb -> cx): start, loop, final check.
cudaError_t enqueue_solve_start(imgm_handle* h, cudaStream_t s) {
    LevelDev& F = h->lv[h->L - 1];
    const int* done = &h->st->done;
    const int64_t N = F.d.N;
    cudaError_t e;
    if ((e = imgm::launch_apply<double>(F.d, imgm::RESID, h->cx, h->cb, h->cr, nullptr, h->gamma, nullptr, s)) !=
        cudaSuccess)
        return e;
    if ((e = imgm::launch_pcg_init_norms(N, h->cr, h->cb, h->partial, h->st, h->hist, s)) != cudaSuccess) return e;
    if (h->precision == 1) {
        if ((e = imgm::launch_vcycle_in<float>(N, h->cr, F.fd.s, F.fd.dinv, h->gamma_diag, h->rf, h->zf, done, s)) !=
            cudaSuccess)
            return e;
        if ((e = enqueue_vcycle<float>(h, h->rf, h->zf, done, s)) != cudaSuccess) return e;
        return imgm::launch_pcg_init_dir<float>(N, h->cr, h->zf, F.fd.s, h->cp, h->zpf, h->partial, h->st, s);
    }
    if ((e = imgm::launch_scale_diag<double>(F.d, h->cr, h->cz, h->gamma_diag, done, s)) != cudaSuccess) return e;
    if ((e = enqueue_vcycle<double>(h, h->cr, h->cz, done, s)) != cudaSuccess) return e;
    if (h->net && (e = enqueue_learned(h, h->cr, h->cz, nullptr, s)) != cudaSuccess) return e;
    return imgm::launch_pcg_init_dir<double>(N, h->cr, h->cz, nullptr, h->cp, h->czp, h->partial, h->st, s);
}

cudaError_t enqueue_iteration(imgm_handle* h, cudaStream_t s) {
    LevelDev& F = h->lv[h->L - 1];
    const int* done = &h->st->done;
    const int64_t N = F.d.N;
    cudaError_t e;
    if ((e = imgm::launch_apply_pq(F.d, h->cp, h->cq, h->partial, h->st, s)) != cudaSuccess) return e;
    if (h->precision == 1) {
        if ((e = imgm::launch_pcg_update<float>(F.d, F.fd.dinv, h->cx, h->cr, h->cp, h->cq, h->zf, h->rf, F.fd.s,
                                                h->gamma_diag, h->partial, h->st, h->hist, s)) != cudaSuccess)
            return e;
        if ((e = enqueue_vcycle<float>(h, h->rf, h->zf, done, s)) != cudaSuccess) return e;
        if ((e = imgm::launch_pcg_rz<float>(N, h->cr, h->zf, F.fd.s, h->zpf, h->partial, h->st, s)) != cudaSuccess)
            return e;
        return imgm::launch_pcg_xpay<float>(N, h->zf, F.fd.s, h->cp, h->zpf, h->st, s);
    }
    if ((e = imgm::launch_pcg_update<double>(F.d, F.d.dinv, h->cx, h->cr, h->cp, h->cq, h->cz, nullptr, nullptr,
                                             h->gamma_diag, h->partial, h->st, h->hist, s)) != cudaSuccess)
        return e;
    if ((e = enqueue_vcycle<double>(h, h->cr, h->cz, done, s)) != cudaSuccess) return e;
    if (h->fcg_m > 0) {
        // FCG(m): the new direction is z (after the learned stage, if any) A-orthogonalised
        // against the last m directions
        if (h->net && (e = enqueue_learned(h, h->cr, h->cz, nullptr, s)) != cudaSuccess) return e;
        if ((e = imgm::launch_fcg_push_dots(N, h->fcg_m, h->cz, h->cp, h->cq, h->fcg_P, h->fcg_Q, h->partial, h->st,
                                            s)) != cudaSuccess)
            return e;
        return imgm::launch_fcg_dir(N, h->fcg_m, h->cz, h->cr, h->cp, h->fcg_P, h->partial, h->st, s);
    }
    if (h->net) {
        // the learned stage makes the preconditioner vary: Polak-Ribiere beta from A p (cq)
        if ((e = enqueue_learned(h, h->cr, h->cz, nullptr, s)) != cudaSuccess) return e;
        if ((e = imgm::launch_pcg_rz<double>(N, h->cr, h->cz, nullptr, nullptr, h->partial, h->st, s, h->cq)) !=
            cudaSuccess)
            return e;
        return imgm::launch_pcg_xpay<double>(N, h->cz, nullptr, h->cp, nullptr, h->st, s);
    }
    // FP64 V-cycle: standard beta (czp null); FP32 levels below an FP64 finest one: flexible
    if ((e = imgm::launch_pcg_rz<double>(N, h->cr, h->cz, nullptr, h->czp, h->partial, h->st, s)) != cudaSuccess)
        return e;
    return imgm::launch_pcg_xpay<double>(N, h->cz, nullptr, h->cp, h->czp, h->st, s);
}

cudaError_t enqueue_solve_finish(imgm_handle* h, cudaStream_t s) {
    LevelDev& F = h->lv[h->L - 1];
    cudaError_t e;
    if ((e = imgm::launch_apply<double>(F.d, imgm::RESID, h->cx, h->cb, F.t, nullptr, h->gamma, nullptr, s)) !=
        cudaSuccess)
        return e;
    return imgm::launch_true_residual_norm(F.d.N, F.t, h->partial, h->st, s);
}

// Builds the solve graph: start -> while (!done) { iteration } -> finish.
// Enqueues the whole solve of h on the capturing stream s: the start, a conditional WHILE
// node whose body is one CG iteration (captured into the node's graph on a side stream),
// and the finish.  Records the kernel counts of the three parts in h->graph_kernels.
cudaError_t capture_solve(imgm_handle* h, cudaStream_t s) {
    cudaStream_t body_stream = nullptr;
    cudaError_t ce = cudaStreamCreateWithFlags(&body_stream, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return ce;
    int64_t c0 = imgm::launch_count();
    ce = enqueue_solve_start(h, s);
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaStreamCaptureStatus cs;
    cudaGraphConditionalHandle handle = 0;
    cudaGraphNode_t cnode = nullptr;
    alignas(cudaGraphNodeParams) unsigned char cp_storage[sizeof(cudaGraphNodeParams)];
    std::memset(cp_storage, 0, sizeof(cp_storage));
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_storage);
    if (ce == cudaSuccess) ce = cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, nullptr, &ndeps);
    if (ce == cudaSuccess) ce = cudaGraphConditionalHandleCreate(&handle, cg, 0, cudaGraphCondAssignDefault);
    if (ce == cudaSuccess) ce = imgm::launch_set_continue(h->st, (unsigned long long)handle, s);
    if (ce == cudaSuccess) ce = cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, nullptr, &ndeps);
    if (ce == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ce = cudaGraphAddNode(&cnode, cg, deps, nullptr, ndeps, &cp);
    }
    if (ce == cudaSuccess) ce = cudaStreamUpdateCaptureDependencies(s, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (ce == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        ce = cudaStreamBeginCaptureToGraph(body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            h->graph_kernels[0] = imgm::launch_count() - c0;
            c0 = imgm::launch_count();
            cudaError_t be = enqueue_iteration(h, body_stream);
            if (be == cudaSuccess) be = imgm::launch_set_continue(h->st, (unsigned long long)handle, body_stream);
            h->graph_kernels[1] = imgm::launch_count() - c0;
            c0 = imgm::launch_count();
            cudaGraph_t outb = nullptr;
            cudaError_t ee = cudaStreamEndCapture(body_stream, &outb);
            ce = (be != cudaSuccess) ? be : ee;
        }
    }
    if (ce == cudaSuccess) ce = enqueue_solve_finish(h, s);
    h->graph_kernels[2] = imgm::launch_count() - c0;
    cudaStreamDestroy(body_stream);
    return ce;
}

// Captures start, conditional WHILE loop over one iteration, and finish into h->exec.
// Capture runs on a stream of the handle (capturing the legacy default stream is not
// allowed); the graph is then launched on the caller's stream.
cudaError_t build_solve_graph(imgm_handle* h) {
    cudaError_t e = cudaSuccess;
    if (!h->capture && (e = cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking)) != cudaSuccess) return e;
    cudaStream_t s = h->capture;
    cudaGraph_t g = nullptr;
    do {
        if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) break;
        const cudaError_t ce = capture_solve(h, s);
        e = cudaStreamEndCapture(s, &g);
        if (ce != cudaSuccess) e = ce;
        if (e != cudaSuccess) break;
        e = cudaGraphInstantiate(&h->exec, g, 0);
    } while (0);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        g = nullptr;
        cudaGetLastError();
    }
    h->graph = g;
    return e;
}

// Images of the cluster-resident coarse levels 0..top for a cluster of cs blocks (see
// DsLevel): the common per-row vector layout, and per block its own rows' tables and the
// Schwarz blocks it applies (the block of its first member's owner).  Returns false when
// the levels do not fit the shared memory of one block.
bool build_ds_images(const imgm_handle* h, int top, int cs, std::vector<unsigned char>& images, imgm::DsImage& hdr0) {
    using imgm::DsLevel;
    const imgm::Hierarchy& H = h->H;
    const int dim = H.dim, p = H.p, W = 2 * p + 1, NC = H.ncoef;
    auto al16 = [](size_t v) { return (v + 15) & ~size_t(15); };
    std::vector<int> ch(top + 1);
    uint32_t off = 0;
    imgm::DsImage hdr{};
    hdr.top = top;
    hdr.dim = dim;
    hdr.p = p;
    hdr.gamma = (float)h->gamma;
    int mb = 1;
    for (int li = 0; li <= top; ++li) {
        const imgm::LevelData& L = H.lv[li];
        ch[li] = (int)(((L.N + cs - 1) / cs + 3) & ~int64_t(3));
        DsLevel& d = hdr.lv[li];
        d.m = L.m;
        d.N = (int)L.N;
        d.ch = ch[li];
        d.TW = L.TW;
        const uint32_t vb = (uint32_t)ch[li] * 4;
        d.off_x = off;
        d.off_r = off + vb;
        d.off_t = off + 2 * vb;
        d.off_e = off + 3 * vb;
        d.off_s = off + 4 * vb;
        d.off_d = off + 5 * vb;
        off += 6 * vb;
        if (li >= 1) mb = std::max(mb, (int)L.max_block);
    }
    hdr.max_block = mb;
    hdr.vec_bytes = off;
    // per block: sizes, then contents
    std::vector<std::vector<unsigned char>> img(cs);
    std::vector<imgm::DsImage> hd(cs, hdr);
    size_t max_img = 0;
    for (int k = 0; k < cs; ++k) {
        std::vector<unsigned char>& B = img[k];
        size_t pos = al16(sizeof(imgm::DsImage));
        B.assign(pos, 0);
        auto put = [&](const void* src, size_t bytes) -> uint32_t {
            const size_t at = pos;
            B.resize(al16(at + bytes), 0);
            if (bytes) std::memcpy(B.data() + at, src, bytes);
            pos = B.size();
            return (uint32_t)(hdr.vec_bytes + at);
        };
        for (int li = 0; li <= top; ++li) {
            const imgm::LevelData& L = H.lv[li];
            DsLevel& d = hd[k].lv[li];
            const int64_t lo = (int64_t)k * ch[li], hi = std::min<int64_t>(L.N, lo + ch[li]);
            std::vector<int32_t> ri(ch[li], -2);
            std::vector<float> coef, dinv(ch[li], 0.0f);
            const int64_t nb = (int64_t)L.band_rows.size();
            int nst = 0;
            for (int64_t j = lo; j < hi; ++j) {
                const int32_t r = L.rowinfo[j];
                if (r >= 0) {
                    ri[j - lo] = nst++;
                    for (int c = 0; c < NC; ++c) coef.push_back(L.f_band_coef[(size_t)c * nb + r]);
                } else {
                    ri[j - lo] = r;
                }
                if (!L.f_dinv.empty()) dinv[j - lo] = L.f_dinv[j];
            }
            d.nst = nst;
            d.off_ri = put(ri.data(), ri.size() * 4);
            d.off_coef = put(coef.data(), coef.size() * 4);
            d.off_dinv = put(dinv.data(), dinv.size() * 4);
            d.off_K1 = put(L.f_K1.data(), L.f_K1.size() * 4);
            d.off_M1 = put(L.f_M1.data(), L.f_M1.size() * 4);
            // Schwarz blocks whose first member this block owns
            std::vector<int32_t> bptr(1, 0), bvptr(1, 0), bidx;
            std::vector<float> bval;
            const int64_t nblk = L.blk_ptr.empty() ? 0 : (int64_t)L.blk_ptr.size() - 1;
            for (int64_t b = 0; b < nblk; ++b) {
                const int64_t s0 = L.blk_ptr[b], nj = L.blk_ptr[b + 1] - s0;
                if (L.blk_idx[s0] / ch[li] != k) continue;
                for (int64_t a = 0; a < nj; ++a) bidx.push_back(L.blk_idx[s0 + a]);
                for (int64_t v = 0; v < nj * nj; ++v) bval.push_back(L.f_blk_val[L.blk_vptr[b] + v]);
                bptr.push_back((int32_t)bidx.size());
                bvptr.push_back((int32_t)bval.size());
            }
            d.nblk = (int)bptr.size() - 1;
            d.off_bptr = put(bptr.data(), bptr.size() * 4);
            d.off_bvptr = put(bvptr.data(), bvptr.size() * 4);
            d.off_bidx = put(bidx.data(), bidx.size() * 4);
            d.off_bval = put(bval.data(), bval.size() * 4);
            if (li >= 1) {
                d.off_rfirst = put(L.r_first.data(), L.r_first.size() * 4);
                d.off_rw = put(L.f_r_w.data(), L.f_r_w.size() * 4);
                d.off_tfirst = put(L.t_first.data(), L.t_first.size() * 4);
                d.off_tw = put(L.f_t_w.data(), L.f_t_w.size() * 4);
            }
            (void)W;
        }
        max_img = std::max(max_img, B.size());
    }
    const uint32_t image_bytes = (uint32_t)al16(max_img);
    const size_t smem = (size_t)hdr.vec_bytes + image_bytes + (size_t)(imgm::DS_TPB / 32) * mb * 4;
    if (smem > imgm::DS_SMEM_MAX) return false;
    images.assign((size_t)cs * image_bytes, 0);
    for (int k = 0; k < cs; ++k) {
        hd[k].image_bytes = image_bytes;
        hd[k].scratch_off = hdr.vec_bytes + image_bytes;
        std::memcpy(img[k].data(), &hd[k], sizeof(imgm::DsImage));
        std::memcpy(images.data() + (size_t)k * image_bytes, img[k].data(), img[k].size());
    }
    hdr0 = hd[0];
    return true;
}

// Launch parameters of the cluster V-cycle over levels 0..top for this context.
imgm::DsVcycle ds_params(const imgm_handle* h, int top, const unsigned char* images, const imgm::DsImage& hdr, int cs) {
    imgm::DsVcycle V{};
    V.images = images;
    for (int li = 0; li <= top; ++li) {
        V.s_glob[li] = h->lv[li].fd.s;
        V.d_glob[li] = h->lv[li].fd.d;
    }
    V.x_top = h->lv[top].fx;
    V.r_top = h->lv[top].fr;
    V.c_rows = h->c_rows;
    V.c_inv = h->f_c_inv;
    V.nc = h->nc;
    V.top = top;
    V.cs = cs;
    V.vec_bytes = hdr.vec_bytes;
    V.image_bytes = hdr.image_bytes;
    V.smem_bytes = hdr.scratch_off + (uint32_t)((imgm::DS_TPB / 32) * hdr.max_block * 4);
    return V;
}

// Picks the task shape of the 3-D z-marching operator apply on every level that uses it:
// rows per lane (1 or 2), planes per z chunk and, in FP32, whether the input planes are
// staged in shared memory by cp.async or loaded to registers, by timing the level's residual-mode apply
// (the V-cycle's) for each candidate on this device and keeping the fastest.  Longer
// chunks redo fewer halo planes, shorter ones give the warps more tasks and shorter
// sequential walks (small levels are latency-bound); which wins
// depends on the level's size and on how many SMs the device has.  The same shape then
// serves the level's other modes (and the CG's apply with p^T A p on the finest level).
// Levels of both arithmetic types are tuned when the FP32 V-cycle is in use.
// IMGM_ZM_YT / IMGM_ZM_ZC in the environment bypass it.
template <typename T>
cudaError_t tune_zm_level(imgm::DevLevelT<T>& d, const T* x, T* y, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
                          bool verbose, int li) {
    static const int zcs3[] = {1, 2, 3, 4, 6, 8, 11, 16, 22, 32};
    static const int zcs2[] = {2, 4, 8, 12, 16, 24, 32, 48, 64};   // 2-D: rows per chunk
    const bool two = d.dim == 2;
    const int* zcs = two ? zcs2 : zcs3;
    const int nzc = two ? 9 : 10;
    float best = 0.0f;
    int best_yt = 0, best_zc = 0, best_stage = 0;
    // FP32: registers (0), per-warp cp.async staging (1) or the CTA form (2), or only the form
    // IMGM_ZM_FORM names (tests); FP64 registers
    int s_lo = 0, s_hi = (sizeof(T) == 4 && !two) ? 2 : 0;
    if (const char* f = std::getenv("IMGM_ZM_FORM"))
        if (sizeof(T) == 4) s_lo = s_hi = std::min(2, std::max(0, std::atoi(f)));
    for (int stage = s_lo; stage <= s_hi; ++stage)
    for (int yt = 1; yt <= (two ? 1 : 2); ++yt)
        for (int zi = 0; zi < nzc; ++zi) {
            const int zc = zcs[zi];
            if (zc > d.m) continue;
            imgm::DevLevelT<T> c = d;
            c.zm_yt = yt;
            c.zm_zc = zc;
            c.zm_stage = stage;
            cudaError_t e = cudaSuccess;
            for (int k = 0; k < 2 && e == cudaSuccess; ++k)
                e = imgm::launch_apply<T>(c, imgm::RESID, x, y, y, nullptr, 0.0, nullptr, s);
            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
            for (int k = 0; k < 5 && e == cudaSuccess; ++k)
                e = imgm::launch_apply<T>(c, imgm::RESID, x, y, y, nullptr, 0.0, nullptr, s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) return e;
            if (verbose)
                std::fprintf(stderr, "imgm: level %d (%s) apply, %d rows per lane, %d planes per chunk%s: %.2f us\n",
                             li + 1, sizeof(T) == 8 ? "FP64" : "FP32", yt, zc,
                             sizeof(T) == 4 ? (stage == 2 ? ", CTA-staged" : stage ? ", staged" : ", registers") : "",
                             ms * 200.0f);
            if (best_yt == 0 || ms < best) {
                best = ms;
                best_yt = yt;
                best_zc = zc;
                best_stage = stage;
            }
        }
    d.zm_yt = best_yt;
    d.zm_zc = best_zc;
    d.zm_stage = best_stage;
    return cudaSuccess;
}

cudaError_t autotune_zm(imgm_handle* h) {
    if (std::getenv("IMGM_ZM_YT") || std::getenv("IMGM_ZM_ZC")) return cudaSuccess;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool verbose = std::getenv("IMGM_VERBOSE") != nullptr;
    for (int li = 0; li < h->L && e == cudaSuccess; ++li) {
        LevelDev& L = h->lv[li];
        if (!(h->dim == 3 ? imgm::zm_applies(L.d.m) : imgm::ym_applies(L.d.m))) continue;
        e = tune_zm_level<double>(L.d, L.t, L.e, s, e0, e1, verbose, li);
        if (e == cudaSuccess && h->precision >= 1 && L.ft)
            e = tune_zm_level<float>(L.fd, L.ft, L.fe, s, e0, e1, verbose, li);
        // the tuning wrote the level's scratch vectors: clear them again
        if (e == cudaSuccess) e = cudaMemsetAsync(L.t, 0, L.d.N * sizeof(double), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(L.e, 0, L.d.N * sizeof(double), s);
        if (e == cudaSuccess && L.fe) e = cudaMemsetAsync(L.fe, 0, L.d.N * sizeof(float), s);
        if (e == cudaSuccess && L.ft) e = cudaMemsetAsync(L.ft, 0, L.d.N * sizeof(float), s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    return e;
}

// Chooses how many coarse levels of the FP32 V-cycle run in the cluster kernel (none,
// or levels 1..top for some top) by timing whole V-cycles of each choice on this device.
cudaError_t autotune_cluster(imgm_handle* h) {
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto time_vcycles = [&](float* ms) -> cudaError_t {
        cudaError_t err = cudaSuccess;
        for (int k = 0; k < 5 && err == cudaSuccess; ++k) err = enqueue_vcycle<float>(h, h->rf, h->zf, nullptr, s);
        if (err == cudaSuccess) err = cudaEventRecord(e0, s);
        for (int k = 0; k < 20 && err == cudaSuccess; ++k) err = enqueue_vcycle<float>(h, h->rf, h->zf, nullptr, s);
        if (err == cudaSuccess) err = cudaEventRecord(e1, s);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) err = cudaEventElapsedTime(ms, e0, e1);
        return err;
    };
    auto install = [&](int top) {
        h->ds_top = top;
        if (top >= 0) h->dsv = h->ds_cand[top];
    };
    const bool verbose = std::getenv("IMGM_VERBOSE") != nullptr;
    int best_top = -1;
    float best = 0.0f;
    install(-1);
    e = time_vcycles(&best);
    if (verbose && e == cudaSuccess)
        std::fprintf(stderr, "imgm: V-cycle, all levels as separate launches: %.2f us\n", best * 50.0f);
    for (int top = (int)h->ds_cand.size() - 1; top >= 0 && e == cudaSuccess; --top) {
        if (!h->ds_images[top]) continue;
        install(top);
        float t = 0.0f;
        e = time_vcycles(&t);
        if (verbose && e == cudaSuccess)
            std::fprintf(stderr, "imgm: V-cycle, levels 1..%d resident on one cluster: %.2f us\n", top + 1, t * 50.0f);
        if (e == cudaSuccess && t < best) {
            best = t;
            best_top = top;
        }
    }
    install(e == cudaSuccess ? best_top : -1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    return e;
}

// Builds and uploads the cluster images of every top that fits, and this context's launch
// parameters for each.
int prepare_ds(imgm_handle* h) {
    const int cs = imgm::ds_cluster_size();
    const int maxtop = std::min(h->L - 2, imgm::DS_MAX_LEVELS - 1);
    h->ds_images.assign(std::max(maxtop + 1, 0), nullptr);
    h->ds_cand.assign(std::max(maxtop + 1, 0), imgm::DsVcycle{});
    if (cs <= 0) return IMGM_OK;
    for (int top = 0; top <= maxtop; ++top) {
        std::vector<unsigned char> images;
        imgm::DsImage hdr{};
        if (!build_ds_images(h, top, cs, images, hdr)) break;     // larger tops do not fit either
        unsigned char* dev = nullptr;
        CK(h->upload(&dev, images), "upload cluster images");
        h->ds_images[top] = dev;
        h->ds_cand[top] = ds_params(h, top, dev, hdr, cs);
    }
    return IMGM_OK;
}

// one level's vectors and tile counter: per solve context
int alloc_level_vectors(imgm_handle* h, LevelDev& dst) {
    const int64_t N = dst.d.N;
    unsigned int* ctr = nullptr;
    CK(h->alloc(&ctr, 2), "alloc tile counter");
    CK(cudaMemset(ctr, 0, 2 * sizeof(unsigned int)), "memset tile counter");
    dst.d.tile_ctr = ctr;
    dst.fd.tile_ctr = ctr;
    // scratch of the sum-factorised transfers to the next coarser level (3-D levels whose
    // transfers take the passes; the row kernels serve the small ones)
    if (dst.d.dim == 3 && dst.d.m >= 34) {
        const int64_t mf = dst.d.m, mc = (dst.d.m - dst.d.p) / 2 + dst.d.p;
        CK(h->alloc(&dst.d.xs1, mf * mf * mc), "alloc transfer scratch");
        CK(h->alloc(&dst.d.xs2, mf * mc * mc), "alloc transfer scratch");
        dst.fd.xs1 = dst.d.xs1;
        dst.fd.xs2 = dst.d.xs2;
    }
    CK(h->alloc(&dst.x, N), "alloc x");
    CK(h->alloc(&dst.r, N), "alloc r");
    CK(h->alloc(&dst.t, N), "alloc t");
    CK(h->alloc(&dst.e, N), "alloc e");
    CK(cudaMemset(dst.x, 0, N * sizeof(double)), "memset");
    CK(cudaMemset(dst.r, 0, N * sizeof(double)), "memset");
    CK(cudaMemset(dst.t, 0, N * sizeof(double)), "memset");
    CK(cudaMemset(dst.e, 0, N * sizeof(double)), "memset");
    if (h->precision >= 1) {
        CK(h->alloc(&dst.fx, N), "alloc x32");
        CK(h->alloc(&dst.fr, N), "alloc r32");
        CK(h->alloc(&dst.ft, N), "alloc t32");
        CK(h->alloc(&dst.fe, N), "alloc e32");
        CK(cudaMemset(dst.fx, 0, N * sizeof(float)), "memset");
        CK(cudaMemset(dst.fr, 0, N * sizeof(float)), "memset");
        CK(cudaMemset(dst.ft, 0, N * sizeof(float)), "memset");
        CK(cudaMemset(dst.fe, 0, N * sizeof(float)), "memset");
    }
    return IMGM_OK;
}

// Everything a solve context owns besides the level vectors: FP32 finest vectors, CG
// vectors, reduction scratch, state and history.
int alloc_context(imgm_handle* h) {
    const int64_t N = h->lv[h->L - 1].d.N;
    if (h->precision == 1) {
        CK(h->alloc(&h->zf, N), "alloc");
        CK(h->alloc(&h->rf, N), "alloc");
        CK(h->alloc(&h->zpf, N), "alloc");
        CK(cudaMemset(h->zf, 0, N * sizeof(float)), "memset");
        CK(cudaMemset(h->rf, 0, N * sizeof(float)), "memset");
        CK(cudaMemset(h->zpf, 0, N * sizeof(float)), "memset");
    }
    CK(h->alloc(&h->cx, N), "alloc");
    CK(h->alloc(&h->cr, N), "alloc");
    CK(h->alloc(&h->cp, N), "alloc");
    CK(h->alloc(&h->cq, N), "alloc");
    CK(h->alloc(&h->cz, N), "alloc");
    CK(h->alloc(&h->cb, N), "alloc");
    if (h->precision == 2) {
        CK(h->alloc(&h->czp, N), "alloc");
        CK(cudaMemset(h->czp, 0, N * sizeof(double)), "memset");
    }
    CK(h->alloc(&h->partial, (size_t)imgm::FCG_MAX * imgm::reduction_blocks()), "alloc");
    CK(h->alloc(&h->st, 1), "alloc");
    CK(cudaMemset(h->st, 0, sizeof(PcgState)), "memset");
    CK(h->alloc(&h->partial_aux, 2 * (size_t)imgm::reduction_blocks()), "alloc");
    CK(h->alloc(&h->st_aux, 1), "alloc");
    CK(cudaMemset(h->st_aux, 0, sizeof(PcgState)), "memset");
    CK(cudaMemset(h->cz, 0, N * sizeof(double)), "memset");
    h->hist_cap = 100001;
    CK(h->alloc(&h->hist, (size_t)h->hist_cap), "alloc");
    return IMGM_OK;
}

int upload_level(imgm_handle* h, const imgm::LevelData& src, LevelDev& dst, int level_index) {
    const imgm::Hierarchy& H = h->H;
    DevLevel& d = dst.d;
    d.dim = H.dim;
    d.p = H.p;
    d.m = src.m;
    d.ncoef = H.ncoef;
    d.N = src.N;
    d.nb = (int32_t)src.band_rows.size();
    d.nblk = (int32_t)(src.blk_ptr.empty() ? 0 : src.blk_ptr.size() - 1);
    d.max_block = (int32_t)src.max_block;
    d.TW = src.TW;
    int32_t* ri;
    double *bc, *k1, *m1, *dv, *bv, *rw, *tw;
    int64_t *bp, *bvp;
    int32_t *bi, *rf, *tf;
    CK(h->upload(&ri, src.rowinfo), "upload rowinfo");
    CK(h->upload(&bc, src.band_coef), "upload stored rows");
    int32_t* brow;
    CK(h->upload(&brow, src.band_rows), "upload stored row ids");
    d.band_row = brow;
    CK(h->upload(&k1, src.K1), "upload K1");
    CK(h->upload(&m1, src.M1), "upload M1");
    CK(h->upload(&dv, src.dinv.empty() ? std::vector<double>(src.N, 0.0) : src.dinv), "upload dinv");
    CK(h->upload(&bp, src.blk_ptr.empty() ? std::vector<int64_t>(1, 0) : src.blk_ptr), "upload block ptr");
    CK(h->upload(&bi, src.blk_idx), "upload block idx");
    CK(h->upload(&bvp, src.blk_vptr.empty() ? std::vector<int64_t>(1, 0) : src.blk_vptr), "upload block vptr");
    CK(h->upload(&bv, src.blk_val), "upload block values");
    int32_t* bof;
    {
        // the block of every (block, function) pair: one thread per pair applies A_j^{-1}
        std::vector<int32_t> of(src.blk_idx.size());
        for (size_t b = 0; b + 1 < src.blk_ptr.size(); ++b)
            for (int64_t q = src.blk_ptr[b]; q < src.blk_ptr[b + 1]; ++q) of[(size_t)q] = (int32_t)b;
        CK(h->upload(&bof, of), "upload block of pair");
    }
    d.blk_of = bof;
    d.npair = (int64_t)src.blk_idx.size();
    CK(h->upload(&rf, src.r_first), "upload restriction");
    CK(h->upload(&rw, src.r_w), "upload restriction");
    CK(h->upload(&tf, src.t_first), "upload prolongation");
    CK(h->upload(&tw, src.t_w), "upload prolongation");
    d.rowinfo = ri;
    d.band_coef = bc;
    d.K1 = k1;
    d.M1 = m1;
    d.dinv = dv;
    d.blk_ptr = bp;
    d.blk_idx = bi;
    d.blk_vptr = bvp;
    d.blk_val = bv;
    d.r_first = rf;
    d.r_w = rw;
    d.t_first = tf;
    d.t_w = tw;
    if (h->precision >= 1) {
        imgm::DevLevelT<float>& f = dst.fd;
        f.dim = d.dim;
        f.p = d.p;
        f.m = d.m;
        f.ncoef = d.ncoef;
        f.N = d.N;
        f.nb = d.nb;
        f.nblk = d.nblk;
        f.max_block = d.max_block;
        f.TW = d.TW;
        f.rowinfo = d.rowinfo;
        f.band_row = d.band_row;
        f.blk_ptr = d.blk_ptr;
        f.blk_idx = d.blk_idx;
        f.blk_vptr = d.blk_vptr;
        f.blk_of = d.blk_of;
        f.npair = d.npair;
        f.r_first = d.r_first;
        f.t_first = d.t_first;
        float *bcf, *k1f, *m1f, *dvf, *bvf, *rwf, *twf, *sf, *df;
        CK(h->upload(&bcf, src.f_band_coef), "upload fp32 rows");
        CK(h->upload(&k1f, src.f_K1), "upload fp32 K1");
        CK(h->upload(&m1f, src.f_M1), "upload fp32 M1");
        CK(h->upload(&dvf, src.f_dinv), "upload fp32 dinv");
        CK(h->upload(&bvf, src.f_blk_val), "upload fp32 blocks");
        CK(h->upload(&rwf, src.f_r_w), "upload fp32 restriction");
        CK(h->upload(&twf, src.f_t_w), "upload fp32 prolongation");
        CK(h->upload(&sf, src.f_s), "upload fp32 scale");
        CK(h->upload(&df, src.f_d), "upload fp32 scale");
        f.band_coef = bcf;
        f.K1 = k1f;
        f.M1 = m1f;
        f.dinv = dvf;
        f.blk_val = bvf;
        f.r_w = rwf;
        f.t_w = twf;
        f.s = sf;
        f.d = df;
    }
    dst.ncolour = src.ncolour;
    dst.blk_cptr = src.blk_cptr;
    dst.sg_cptr = src.sg_cptr;
    if (src.ncolour > 0) {
        CK(h->upload(&dst.sg_row, src.sg_row), "upload one-function blocks");
        CK(h->upload(&dst.sg_inv, src.sg_inv), "upload one-function blocks");
        if (h->precision >= 1) CK(h->upload(&dst.f_sg_inv, src.f_sg_inv), "upload fp32 one-function blocks");
    }
    imgm_level_info& in = dst.info;
    in.n_grid = src.N;
    in.n_active = src.n_active;
    in.m = src.m;
    in.n_band = (int64_t)src.band_rows.size();
    in.n_blocks = d.nblk;
    int64_t ent = 0;
    for (int b = 0; b < d.nblk; ++b) ent += src.blk_vptr[b + 1] - src.blk_vptr[b];
    in.block_entries = ent;
    in.max_block = src.max_block;
    in.pruned = (level_index == 0) ? H.coarse_pruned : src.pruned;
    return IMGM_OK;
}

imgm::Problem make_problem(const imgm_geometry* geom, const imgm_config* cfg) {
    imgm::Problem pb;
    pb.dim = geom->dim;
    pb.lo = geom->lo;
    pb.hi = geom->hi;
    for (int i = 0; i < geom->n_holes; ++i) {
        imgm::Ball b{};
        for (int k = 0; k < geom->dim; ++k) b.c[k] = geom->centers[i * geom->dim + k];
        b.r = geom->radii[i];
        pb.holes.push_back(b);
    }
    pb.n = cfg->n;
    pb.basis = cfg->basis;
    pb.p = cfg->degree;
    pb.levels = cfg->levels;
    pb.depth = cfg->depth;
    pb.bc = cfg->bc;
    pb.gamma = cfg->gamma;
    pb.precision = cfg->precision;
    pb.smoother = cfg->smoother;
    return pb;
}

int validate_inputs(const imgm_geometry* geom, const imgm_config* cfg) {
    if (!geom || !cfg) return fail(nullptr, IMGM_ERR_INVALID, "null geometry or config");
    if (geom->dim != 2 && geom->dim != 3) return fail(nullptr, IMGM_ERR_INVALID, "dim must be 2 or 3");
    if (geom->n_holes < 0 || (geom->n_holes > 0 && (!geom->centers || !geom->radii)))
        return fail(nullptr, IMGM_ERR_INVALID, "bad hole arrays");
    for (int i = 0; i < geom->n_holes; ++i)
        if (!(geom->radii[i] > 0.0)) return fail(nullptr, IMGM_ERR_INVALID, "hole radii must be positive");
    return IMGM_OK;
}

}  // namespace

extern "C" {

const char* imgm_last_error(const imgm_handle* h) { return h ? h->err.c_str() : g_setup_error.c_str(); }

int imgm_setup(const imgm_geometry* geom, const imgm_config* cfg, imgm_handle** out) {
    if (!out) return fail(nullptr, IMGM_ERR_INVALID, "null output handle");
    *out = nullptr;
    int v = validate_inputs(geom, cfg);
    if (v != IMGM_OK) return v;
    std::unique_ptr<imgm_handle> h(new (std::nothrow) imgm_handle(std::make_shared<SharedData>()));
    if (!h) return fail(nullptr, IMGM_ERR_INVALID, "out of host memory");
    imgm::Problem pb = make_problem(geom, cfg);
    std::string err;
    if (!imgm::build_hierarchy(pb, h->H, err)) {
        int code = (err.find("positive definite") != std::string::npos) ? IMGM_ERR_NOT_SPD : IMGM_ERR_UNSUPPORTED;
        if (err.find("must") != std::string::npos || err.find("too") != std::string::npos) code = IMGM_ERR_INVALID;
        if (err.find("coarsest level has") != std::string::npos) code = IMGM_ERR_UNSUPPORTED;
        return fail(nullptr, code, err);
    }
    imgm_handle* hp = h.get();
    hp->dim = h->H.dim;
    hp->p = h->H.p;
    hp->L = h->H.L;
    hp->gamma = h->H.gamma;
    hp->precision = cfg->precision;
    hp->smoother = cfg->smoother;
    hp->gamma_diag = cfg->smoother == 1 ? 0.0 : hp->gamma;
    hp->lv.resize(hp->L);
    for (int li = 0; li < hp->L; ++li) {
        int rc = upload_level(hp, hp->H.lv[li], hp->lv[li], li);
        if (rc == IMGM_OK) rc = alloc_level_vectors(hp, hp->lv[li]);
        if (rc != IMGM_OK) {
            g_setup_error = hp->err;
            return rc;
        }
    }
    {
        imgm_handle* h = hp;   // for CK
        CK(h->upload(&h->c_rows, h->H.c_rows), "upload coarse rows");
        CK(h->upload(&h->c_inv, h->H.c_inv), "upload coarse inverse");
        h->nc = (int)h->H.c_rows.size();
        if (h->precision >= 1) CK(h->upload(&h->f_c_inv, h->H.f_c_inv), "upload fp32 coarse inverse");
        CK(h->upload(&h->b, h->H.b), "upload rhs");
        int rc = alloc_context(h);
        if (rc != IMGM_OK) {
            g_setup_error = h->err;
            return rc;
        }
        CK(autotune_zm(h), "apply autotune");
        // the coarse levels of the FP32 V-cycle resident on one cluster, when the device has
        // clusters, the levels fit and the autotuner finds it faster
        if (h->precision == 1 && h->smoother == 0 && h->L >= 2) {
            rc = prepare_ds(h);
            if (rc != IMGM_OK) {
                g_setup_error = h->err;
                return rc;
            }
            CK(autotune_cluster(h), "cluster autotune");
            // IMGM_CLUSTER_TOP=k forces levels 1..k+1 onto the cluster (when they fit), -1 none
            if (const char* v = std::getenv("IMGM_CLUSTER_TOP")) {
                const int t = std::atoi(v);
                if (t < 0) {
                    h->ds_top = -1;
                } else {
                    int best = -1;
                    for (int q = 0; q <= t && q < (int)h->ds_images.size(); ++q)
                        if (h->ds_images[q]) best = q;
                    h->ds_top = best;
                    if (best >= 0) h->dsv = h->ds_cand[best];
                }
            }
        }
        CK(cudaDeviceSynchronize(), "setup sync");
    }
    hp->on_device = true;
    *out = h.release();
    return IMGM_OK;
}

void imgm_destroy(imgm_handle* h) {
    if (!h) return;
    cudaDeviceSynchronize();
    delete h;
}

int imgm_levels(const imgm_handle* h) { return h ? h->L : IMGM_ERR_INVALID; }

int imgm_get_level_info(const imgm_handle* h, int level, imgm_level_info* info) {
    if (!h || !info || level < 1 || level > h->L) return IMGM_ERR_INVALID;
    *info = h->lv[level - 1].info;
    return IMGM_OK;
}

int imgm_active_mask(const imgm_handle* h, int level, uint8_t* host_mask) {
    if (!h || !host_mask || level < 1 || level > h->L) return IMGM_ERR_INVALID;
    const std::vector<uint8_t>& a = h->H.lv[level - 1].active;
    std::memcpy(host_mask, a.data(), a.size());
    return IMGM_OK;
}

int imgm_rhs(imgm_handle* h, double* dev_b, void* stream) {
    int c = check_level(h, h ? h->L : 0, 1);
    if (c) return c;
    if (!dev_b) return fail(h, IMGM_ERR_INVALID, "null pointer");
    CK(cudaMemcpyAsync(dev_b, h->b, h->lv[h->L - 1].d.N * sizeof(double), cudaMemcpyDeviceToDevice, (cudaStream_t)stream),
       "rhs copy");
    return IMGM_OK;
}

int imgm_apply_operator(imgm_handle* h, int level, const double* dev_x, double* dev_y, void* stream) {
    int c = check_level(h, level, 1);
    if (c) return c;
    if (!dev_x || !dev_y || dev_x == dev_y) return fail(h, IMGM_ERR_INVALID, "bad vector pointers");
    const LevelDev& L = h->lv[level - 1];
    CK(imgm::launch_apply<double>(L.d, imgm::APPLY, dev_x, nullptr, dev_y, nullptr, 0.0, nullptr, (cudaStream_t)stream),
       "apply");
    return IMGM_OK;
}

int imgm_smooth(imgm_handle* h, int level, const double* dev_r, double* dev_z, void* stream) {
    int c = check_level(h, level, 2);
    if (c) return c;
    if (!dev_r || !dev_z || dev_r == dev_z) return fail(h, IMGM_ERR_INVALID, "bad vector pointers");
    LevelDev& L = h->lv[level - 1];
    cudaStream_t s = (cudaStream_t)stream;
    if (h->smoother == 1) {
        // forward coloured sweep from 0, residual (in the level's t) updated after each colour
        CK(imgm::launch_scale_diag<double>(L.d, dev_r, dev_z, 0.0, nullptr, s), "smooth zero");
        for (int k = 0; k < L.ncolour; ++k) {
            CK(colour_step<double>(L, k, k == 0 ? dev_r : L.t, dev_z, nullptr, s), "smooth colour");
            if (k + 1 < L.ncolour)
                CK(imgm::launch_apply<double>(L.d, imgm::RESID, dev_z, dev_r, L.t, nullptr, 0.0, nullptr, s), "smooth residual");
        }
        return IMGM_OK;
    }
    CK(imgm::launch_scale_diag<double>(L.d, dev_r, dev_z, h->gamma, nullptr, s), "smooth diag");
    CK(imgm::launch_blocks<double>(L.d, dev_r, dev_z, h->gamma, nullptr, s), "smooth blocks");
    return IMGM_OK;
}

int imgm_restrict(imgm_handle* h, int level, const double* dev_r, double* dev_rc, void* stream) {
    int c = check_level(h, level, 2);
    if (c) return c;
    if (!dev_r || !dev_rc) return fail(h, IMGM_ERR_INVALID, "bad vector pointers");
    CK(imgm::launch_restrict<double>(h->lv[level - 1].d, h->lv[level - 2].d, dev_r, dev_rc, nullptr, 0.0, nullptr,
                             (cudaStream_t)stream),
       "restrict");
    return IMGM_OK;
}

int imgm_prolong(imgm_handle* h, int level, const double* dev_xc, double* dev_e, void* stream) {
    int c = check_level(h, level, 2);
    if (c) return c;
    if (!dev_xc || !dev_e) return fail(h, IMGM_ERR_INVALID, "bad vector pointers");
    CK(imgm::launch_prolong<double>(h->lv[level - 1].d, h->lv[level - 2].d, dev_xc, dev_e, nullptr, nullptr,
                            (cudaStream_t)stream),
       "prolong");
    return IMGM_OK;
}

int imgm_coarse_solve(imgm_handle* h, const double* dev_r, double* dev_x, void* stream) {
    int c = check_level(h, 1, 1);
    if (c) return c;
    if (!dev_r || !dev_x || dev_r == dev_x) return fail(h, IMGM_ERR_INVALID, "bad vector pointers");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemsetAsync(dev_x, 0, h->lv[0].d.N * sizeof(double), s), "coarse memset");
    CK(imgm::launch_coarse<double>(h->c_rows, h->c_inv, h->nc, dev_r, dev_x, nullptr, s), "coarse solve");
    return IMGM_OK;
}

// z = B r, one V-cycle (FP64, or FP32 on Jacobi-scaled data for precision 1)
cudaError_t enqueue_precondition(imgm_handle* h, const double* r, double* z, cudaStream_t s) {
    LevelDev& F = h->lv[h->L - 1];
    cudaError_t e;
    if (h->precision == 1) {
        if ((e = imgm::launch_vcycle_in<float>(F.d.N, r, F.fd.s, F.fd.dinv, h->gamma_diag, h->rf, h->zf, nullptr, s)) !=
            cudaSuccess)
            return e;
        if ((e = enqueue_vcycle<float>(h, h->rf, h->zf, nullptr, s)) != cudaSuccess) return e;
        return imgm::launch_vcycle_out<float>(F.d.N, h->zf, F.fd.s, z, s);
    }
    if ((e = imgm::launch_scale_diag<double>(F.d, r, z, h->gamma_diag, nullptr, s)) != cudaSuccess) return e;
    return enqueue_vcycle<double>(h, r, z, nullptr, s);
}

int imgm_apply_preconditioner(imgm_handle* h, const double* dev_r, double* dev_z, void* stream) {
    int c = check_level(h, h ? h->L : 0, 1);
    if (c) return c;
    if (!dev_r || !dev_z || dev_r == dev_z) return fail(h, IMGM_ERR_INVALID, "bad vector pointers");
    CK(enqueue_precondition(h, dev_r, dev_z, (cudaStream_t)stream), "vcycle");
    return IMGM_OK;
}

int imgm_pcg_solve(imgm_handle* h, const double* dev_b, double* dev_x, double rtol, int maxit, imgm_result* out,
                   double* dev_hist, void* stream) {
    int c = check_level(h, h ? h->L : 0, 1);
    if (c) return c;
    if (!dev_b || !dev_x || !out) return fail(h, IMGM_ERR_INVALID, "null pointer");
    if (maxit < 0 || maxit >= h->hist_cap || !(rtol >= 0.0)) return fail(h, IMGM_ERR_INVALID, "bad rtol or maxit");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = h->lv[h->L - 1].d.N;
    PcgState init;
    std::memset(&init, 0, sizeof(init));
    init.tol2 = rtol * rtol;
    init.maxit = maxit;
    CK(cudaMemcpyAsync(h->st, &init, sizeof(init), cudaMemcpyHostToDevice, s), "state");
    CK(cudaMemcpyAsync(h->cb, dev_b, N * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy b");
    CK(cudaMemcpyAsync(h->cx, dev_x, N * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy x0");
    // IMGM_SOLVE_GRAPH=0: the same kernels from a host loop instead of the conditional graph
    // (profilers cannot look inside graphs that hold conditional nodes)
    static const bool no_graph = [] {
        const char* v = std::getenv("IMGM_SOLVE_GRAPH");
        return v && v[0] == '0';
    }();
    if (no_graph) h->graph_failed = true;
    if (!h->exec && !h->graph_failed) {
        cudaError_t ge = build_solve_graph(h);
        if (ge != cudaSuccess) {
            // capture without programmatic edges
            cudaGetLastError();
            if (std::getenv("IMGM_VERBOSE"))
                std::fprintf(stderr, "imgm: solve graph with programmatic launches not built (%s)\n",
                             cudaGetErrorString(ge));
            imgm::set_programmatic_launch(false);
            ge = build_solve_graph(h);
            imgm::set_programmatic_launch(true);
        }
        if (ge == cudaSuccess && std::getenv("IMGM_VERBOSE")) std::fprintf(stderr, "imgm: solve graph built\n");
        if (ge != cudaSuccess) {
            h->graph_failed = true;
            cudaGetLastError();
            if (std::getenv("IMGM_VERBOSE"))
                std::fprintf(stderr, "imgm: conditional solve graph not built (%s), host loop\n", cudaGetErrorString(ge));
        }
    }
    const int64_t launches0 = imgm::launch_count();
    if (h->exec) {
        CK(cudaGraphLaunch(h->exec, s), "graph launch");
    } else {
        // fallback without conditional graph nodes: host loop, convergence read back every 8 steps
        CK(enqueue_solve_start(h, s), "start");
        int done = 0;
        int it = 0;
        while (!done && it < maxit) {
            for (int k = 0; k < 8; ++k, ++it) CK(enqueue_iteration(h, s), "iteration");
            CK(cudaMemcpyAsync(&done, &h->st->done, sizeof(int), cudaMemcpyDeviceToHost, s), "done flag");
            CK(cudaStreamSynchronize(s), "sync");
        }
        CK(enqueue_solve_finish(h, s), "finish");
    }
    CK(cudaMemcpyAsync(dev_x, h->cx, N * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy x");
    PcgState fin;
    CK(cudaMemcpyAsync(&fin, h->st, sizeof(fin), cudaMemcpyDeviceToHost, s), "state");
    if (dev_hist)
        CK(cudaMemcpyAsync(dev_hist, h->hist, (size_t)(maxit + 1) * sizeof(double), cudaMemcpyDeviceToDevice, s),
           "hist");
    CK(cudaStreamSynchronize(s), "solve sync");
    out->iterations = fin.iter;
    out->status = fin.status;
    // graph: the start part, one loop body per iteration, the finish part
    out->kernel_launches = h->exec ? h->graph_kernels[0] + (int64_t)fin.iter * h->graph_kernels[1] + h->graph_kernels[2]
                                   : imgm::launch_count() - launches0;
    out->rel_residual = fin.bb > 0 ? std::sqrt(fin.rr / fin.bb) : 0.0;
    out->true_rel_residual = fin.bb > 0 ? std::sqrt(fin.true_rr / fin.bb) : 0.0;
    if (h->net) {
        int c2 = net_wait_status(h, h->lws);
        if (c2) return c2;
    }
    return fin.status == -5 ? IMGM_ERR_BREAKDOWN : (fin.status == 1 ? IMGM_MAX_ITER : IMGM_OK);
}

int imgm_residual_norm2(imgm_handle* h, const double* dev_b, const double* dev_x, double* dev_out, void* stream) {
    int c = check_level(h, h ? h->L : 0, 1);
    if (c) return c;
    if (!dev_b || !dev_x || !dev_out) return fail(h, IMGM_ERR_INVALID, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    LevelDev& F = h->lv[h->L - 1];
    CK(imgm::launch_apply<double>(F.d, imgm::RESID, dev_x, dev_b, F.t, nullptr, h->gamma, nullptr, s), "residual");
    CK(imgm::launch_true_residual_norm(F.d.N, F.t, h->partial_aux, h->st_aux, s), "residual norm");
    CK(cudaMemcpyAsync(dev_out, &h->st_aux->true_rr, sizeof(double), cudaMemcpyDeviceToDevice, s), "norm copy");
    return IMGM_OK;
}

int imgm_residual_norm2_noalloc(imgm_handle* h, const double* dev_b, const double* dev_x, double* dev_out,
                                void* stream) {
    int c = check_level(h, h ? h->L : 0, 1);
    if (c) return c;
    if (!dev_b || !dev_x || !dev_out) return fail(h, IMGM_ERR_INVALID, "null pointer");
    LevelDev& F = h->lv[h->L - 1];
    if (F.d.N > NOALLOC_MAX_ROWS)
        return fail(h, IMGM_ERR_UNSUPPORTED,
                    "imgm_residual_norm2_noalloc: the finest level has " + std::to_string(F.d.N) +
                        " rows, more than the static scratch holds (" + std::to_string(NOALLOC_MAX_ROWS) + ")");
    if (imgm::reduction_blocks() > NOALLOC_MAX_PARTIALS)
        return fail(h, IMGM_ERR_UNSUPPORTED, "imgm_residual_norm2_noalloc: too many reduction blocks for the scratch");
    int dev = 0;
    CK(cudaGetDevice(&dev), "noalloc: cudaGetDevice");
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(h, IMGM_ERR_UNSUPPORTED, "noalloc: device ordinal too large");
    double* base = nullptr;
    {
        // first call on this device: look up the device address of the scratch array
        // (its name in host code is only a host-side stand-in)
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(h, e, "noalloc: cudaGetSymbolAddress");
            g_noalloc_ptr[dev] = (double*)p;
        }
        base = g_noalloc_ptr[dev];
    }
    PcgState* st = reinterpret_cast<PcgState*>(base);
    double* partial = base + NOALLOC_STATE_DOUBLES;
    double* t = partial + NOALLOC_MAX_PARTIALS;
    cudaStream_t s = (cudaStream_t)stream;
    // the reduction ticket must start at zero; the array keeps the previous call's contents
    CK(cudaMemsetAsync(st, 0, sizeof(PcgState), s), "noalloc: clear state");
    CK(imgm::launch_apply<double>(F.d, imgm::RESID, dev_x, dev_b, t, nullptr, h->gamma, nullptr, s), "noalloc: residual");
    CK(imgm::launch_true_residual_norm(F.d.N, t, partial, st, s), "noalloc: residual norm");
    CK(cudaMemcpyAsync(dev_out, &st->true_rr, sizeof(double), cudaMemcpyDeviceToDevice, s), "noalloc: norm copy");
    return IMGM_OK;
}

int imgm_pcg_solve_host(imgm_handle* h, const double* host_b, double* host_x, double rtol, int maxit,
                        imgm_result* out, void* stream) {
    int c = check_level(h, h ? h->L : 0, 1);
    if (c) return c;
    if (!host_b || !host_x || !out) return fail(h, IMGM_ERR_INVALID, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = h->lv[h->L - 1].d.N;
    // stage through the handle's own CG vectors: b -> cq, x0 = 0 -> cp (both are
    // overwritten by the solve before they are read)
    CK(cudaMemcpyAsync(h->cq, host_b, N * sizeof(double), cudaMemcpyHostToDevice, s), "h2d b");
    CK(cudaMemsetAsync(h->cp, 0, N * sizeof(double), s), "x0");
    int rc = imgm_pcg_solve(h, h->cq, h->cp, rtol, maxit, out, nullptr, stream);
    if (rc < 0) return rc;
    CK(cudaMemcpyAsync(host_x, h->cx, N * sizeof(double), cudaMemcpyDeviceToHost, s), "d2h x");
    CK(cudaStreamSynchronize(s), "sync");
    return rc;
}

int imgm_setup_host(const imgm_geometry* geom, const imgm_config* cfg, imgm_handle** out) {
    if (!out) return fail(nullptr, IMGM_ERR_INVALID, "null output handle");
    *out = nullptr;
    int v = validate_inputs(geom, cfg);
    if (v != IMGM_OK) return v;
    std::unique_ptr<imgm_handle> h(new (std::nothrow) imgm_handle(std::make_shared<SharedData>()));
    if (!h) return fail(nullptr, IMGM_ERR_INVALID, "out of host memory");
    imgm::Problem pb = make_problem(geom, cfg);
    std::string err;
    if (!imgm::build_hierarchy(pb, h->H, err)) {
        int code = (err.find("positive definite") != std::string::npos) ? IMGM_ERR_NOT_SPD : IMGM_ERR_UNSUPPORTED;
        if (err.find("must") != std::string::npos || err.find("too") != std::string::npos) code = IMGM_ERR_INVALID;
        return fail(nullptr, code, err);
    }
    h->dim = h->H.dim;
    h->p = h->H.p;
    h->L = h->H.L;
    h->gamma = h->H.gamma;
    h->smoother = h->H.smoother;
    h->gamma_diag = h->smoother == 1 ? 0.0 : h->gamma;
    h->lv.resize(h->L);
    for (int li = 0; li < h->L; ++li) {
        const imgm::LevelData& s = h->H.lv[li];
        imgm_level_info& in = h->lv[li].info;
        in.n_grid = s.N;
        in.n_active = s.n_active;
        in.m = s.m;
        in.n_band = (int64_t)s.band_rows.size();
        in.n_blocks = s.blk_ptr.empty() ? 0 : (int64_t)s.blk_ptr.size() - 1;
        in.block_entries = (int64_t)s.blk_val.size();
        in.max_block = s.max_block;
        in.pruned = (li == 0) ? h->H.coarse_pruned : s.pruned;
    }
    *out = h.release();
    return IMGM_OK;
}

int imgm_host_operator_rows(const imgm_handle* h, int level, int64_t nrows, const int64_t* rows, double* out) {
    if (!h || level < 1 || level > h->L || nrows < 0 || (nrows > 0 && (!rows || !out))) return IMGM_ERR_INVALID;
    const imgm::Hierarchy& H = h->H;
    const imgm::LevelData& lv = H.lv[level - 1];
    const int p = H.p, W = 2 * p + 1, dim = H.dim, nc = H.ncoef;
    const int64_t m = lv.m, nb = (int64_t)lv.band_rows.size();
    for (int64_t k = 0; k < nrows; ++k) {
        const int64_t r = rows[k];
        double* o = out + k * nc;
        std::fill(o, o + nc, 0.0);
        if (r < 0 || r >= lv.N) return IMGM_ERR_INVALID;
        const int ri = lv.rowinfo[r];
        if (ri == -2) continue;
        if (ri >= 0) {
            for (int c = 0; c < nc; ++c) o[c] = lv.band_coef[(size_t)c * nb + ri];
            continue;
        }
        int i[3] = {(int)(r % m), (int)((r / m) % m), dim == 3 ? (int)(r / (m * m)) : 0};
        for (int c = 0; c < nc; ++c) {
            int off[3] = {c % W - p, (c / W) % W - p, dim == 3 ? c / (W * W) - p : 0};
            int j[3] = {i[0] + off[0], i[1] + off[1], i[2] + off[2]};
            bool ok = true;
            for (int d = 0; d < dim; ++d) ok = ok && j[d] >= 0 && j[d] < m;
            if (!ok) continue;
            int64_t jf = j[0] + m * (j[1] + (dim == 3 ? m * j[2] : 0));
            if (!lv.active[jf]) continue;
            auto K = [&](int d) { return lv.K1[(size_t)i[d] * W + off[d] + p]; };
            auto M = [&](int d) { return lv.M1[(size_t)i[d] * W + off[d] + p]; };
            o[c] = (dim == 2) ? K(0) * M(1) + M(0) * K(1)
                              : K(0) * M(1) * M(2) + M(0) * K(1) * M(2) + M(0) * M(1) * K(2);
        }
    }
    return IMGM_OK;
}

int imgm_host_rhs(const imgm_handle* h, double* out) {
    if (!h || !out) return IMGM_ERR_INVALID;
    std::memcpy(out, h->H.b.data(), h->H.b.size() * sizeof(double));
    return IMGM_OK;
}

int imgm_host_block_sizes(const imgm_handle* h, int level, int64_t* nblk, int64_t* nidx, int64_t* nval) {
    if (!h || level < 2 || level > h->L || !nblk || !nidx || !nval) return IMGM_ERR_INVALID;
    const imgm::LevelData& lv = h->H.lv[level - 1];
    *nblk = lv.blk_ptr.empty() ? 0 : (int64_t)lv.blk_ptr.size() - 1;
    *nidx = (int64_t)lv.blk_idx.size();
    *nval = (int64_t)lv.blk_val.size();
    return IMGM_OK;
}

int imgm_host_blocks(const imgm_handle* h, int level, int64_t* ptr, int32_t* idx, int64_t* vptr, double* val,
                     double* dinv) {
    if (!h || level < 2 || level > h->L) return IMGM_ERR_INVALID;
    const imgm::LevelData& lv = h->H.lv[level - 1];
    if (ptr) std::memcpy(ptr, lv.blk_ptr.data(), lv.blk_ptr.size() * sizeof(int64_t));
    if (idx) std::memcpy(idx, lv.blk_idx.data(), lv.blk_idx.size() * sizeof(int32_t));
    if (vptr) std::memcpy(vptr, lv.blk_vptr.data(), lv.blk_vptr.size() * sizeof(int64_t));
    if (val) std::memcpy(val, lv.blk_val.data(), lv.blk_val.size() * sizeof(double));
    if (dinv) std::memcpy(dinv, lv.dinv.data(), lv.dinv.size() * sizeof(double));
    return IMGM_OK;
}

int imgm_host_restriction(const imgm_handle* h, int level, int32_t* first, double* w) {
    if (!h || level < 2 || level > h->L || !first || !w) return IMGM_ERR_INVALID;
    const imgm::LevelData& lv = h->H.lv[level - 1];
    std::memcpy(first, lv.r_first.data(), lv.r_first.size() * sizeof(int32_t));
    std::memcpy(w, lv.r_w.data(), lv.r_w.size() * sizeof(double));
    return IMGM_OK;
}

int imgm_host_coarse_size(const imgm_handle* h, int64_t* nc) {
    if (!h || !nc) return IMGM_ERR_INVALID;
    *nc = (int64_t)h->H.c_rows.size();
    return IMGM_OK;
}

int imgm_host_coarse(const imgm_handle* h, int32_t* rows, double* inv) {
    if (!h || !rows || !inv) return IMGM_ERR_INVALID;
    std::memcpy(rows, h->H.c_rows.data(), h->H.c_rows.size() * sizeof(int32_t));
    std::memcpy(inv, h->H.c_inv.data(), h->H.c_inv.size() * sizeof(double));
    return IMGM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Solve contexts and batches

int imgm_clone(const imgm_handle* src, imgm_handle** out) {
    if (!out) return fail(nullptr, IMGM_ERR_INVALID, "null output handle");
    *out = nullptr;
    if (!src || !src->on_device) return fail(nullptr, IMGM_ERR_INVALID, "handle has no device data");
    std::unique_ptr<imgm_handle> h(new (std::nothrow) imgm_handle(src->sh));
    if (!h) return fail(nullptr, IMGM_ERR_INVALID, "out of host memory");
    imgm_handle* hp = h.get();
    hp->dim = src->dim;
    hp->p = src->p;
    hp->L = src->L;
    hp->gamma = src->gamma;
    hp->smoother = src->smoother;
    hp->gamma_diag = src->gamma_diag;
    hp->precision = src->precision;
    hp->c_rows = src->c_rows;
    hp->c_inv = src->c_inv;
    hp->f_c_inv = src->f_c_inv;
    hp->nc = src->nc;
    hp->b = src->b;
    hp->lv = src->lv;          // level tables shared; vectors replaced below
    for (LevelDev& L : hp->lv) {
        int rc = alloc_level_vectors(hp, L);
        if (rc != IMGM_OK) {
            g_setup_error = hp->err;
            return rc;
        }
    }
    int rc = alloc_context(hp);
    if (rc != IMGM_OK) {
        g_setup_error = hp->err;
        return rc;
    }
    // the cluster images are shared; the launch parameters point at this context's vectors
    hp->ds_images = src->ds_images;
    hp->ds_cand.assign(src->ds_cand.size(), imgm::DsVcycle{});
    for (size_t t = 0; t < src->ds_cand.size(); ++t)
        if (src->ds_images[t]) {
            hp->ds_cand[t] = src->ds_cand[t];
            hp->ds_cand[t].x_top = hp->lv[t].fx;
            hp->ds_cand[t].r_top = hp->lv[t].fr;
        }
    hp->ds_top = src->ds_top;
    if (hp->ds_top >= 0) hp->dsv = hp->ds_cand[hp->ds_top];
    {
        imgm_handle* h = hp;
        CK(cudaDeviceSynchronize(), "clone sync");
    }
    hp->on_device = true;
    *out = h.release();
    return IMGM_OK;
}

struct imgm_batch {
    std::vector<imgm_handle*> hs;
    std::vector<cudaStream_t> streams;   // one capture stream per solve (the branches)
    std::vector<cudaEvent_t> events;
    cudaStream_t root = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> kernels;        // per solve: start, body, finish kernel counts
    std::vector<imgm_net*> nets;         // networks the recorded solves run (one count each)
    std::string err;
    ~imgm_batch() {
        for (imgm_net* n : nets) n->attached -= 1;
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        for (cudaStream_t s : streams) cudaStreamDestroy(s);
        if (fork) cudaEventDestroy(fork);
        if (root) cudaStreamDestroy(root);
    }
};

namespace {
int batch_fail(imgm_batch* b, int code, const std::string& msg) {
    if (b) b->err = msg;
    g_setup_error = msg;
    return code;
}
}  // namespace

int imgm_batch_create(imgm_handle* const* hs, int n, imgm_batch** out) {
    if (!out) return batch_fail(nullptr, IMGM_ERR_INVALID, "null output batch");
    *out = nullptr;
    if (!hs || n <= 0) return batch_fail(nullptr, IMGM_ERR_INVALID, "empty batch");
    for (int k = 0; k < n; ++k) {
        if (!hs[k] || !hs[k]->on_device) return batch_fail(nullptr, IMGM_ERR_INVALID, "handle has no device data");
        for (int j = 0; j < k; ++j)
            if (hs[j] == hs[k])
                return batch_fail(nullptr, IMGM_ERR_INVALID, "a context appears twice (use imgm_clone for more right-hand sides)");
    }
    std::unique_ptr<imgm_batch> b(new (std::nothrow) imgm_batch());
    if (!b) return batch_fail(nullptr, IMGM_ERR_INVALID, "out of host memory");
    b->hs.assign(hs, hs + n);
    b->streams.assign(n, nullptr);
    b->events.assign(n, nullptr);
    b->kernels.assign(3 * (size_t)n, 0);
    cudaError_t e = cudaStreamCreateWithFlags(&b->root, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&b->streams[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->events[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return batch_fail(nullptr, IMGM_ERR_CUDA, std::string("batch streams: ") + cudaGetErrorString(e));
    // one graph: fork from the root stream, every solve on its own branch (each with its own
    // device-side convergence loop), join back on the root
    cudaGraph_t g = nullptr;
    do {
        if ((e = cudaStreamBeginCapture(b->root, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) break;
        cudaError_t ce = cudaEventRecord(b->fork, b->root);
        for (int k = 0; k < n && ce == cudaSuccess; ++k) {
            ce = cudaStreamWaitEvent(b->streams[k], b->fork, 0);
            if (ce == cudaSuccess) ce = capture_solve(hs[k], b->streams[k]);
            for (int q = 0; q < 3; ++q) b->kernels[3 * (size_t)k + q] = hs[k]->graph_kernels[q];
            if (ce == cudaSuccess) ce = cudaEventRecord(b->events[k], b->streams[k]);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->root, b->events[k], 0);
        }
        e = cudaStreamEndCapture(b->root, &g);
        if (ce != cudaSuccess) e = ce;
        if (e != cudaSuccess) break;
        e = cudaGraphInstantiate(&b->exec, g, 0);
    } while (0);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return batch_fail(nullptr, IMGM_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    }
    b->graph = g;
    // the recorded solves read the attached networks' weights: each counts as an attachment
    // until the batch is destroyed, so such a network cannot be freed under the graph
    for (int k = 0; k < n; ++k)
        if (hs[k]->net) {
            hs[k]->net->attached += 1;
            b->nets.push_back(hs[k]->net);
        }
    *out = b.release();
    return IMGM_OK;
}

int imgm_batch_solve(imgm_batch* b, const double* const* dev_b, double* const* dev_x, double rtol, int maxit,
                     imgm_result* out, void* stream) {
    if (!b || !b->exec) return batch_fail(b, IMGM_ERR_INVALID, "no batch");
    if (!dev_b || !dev_x || !out) return batch_fail(b, IMGM_ERR_INVALID, "null pointer");
    const int n = (int)b->hs.size();
    cudaStream_t s = (cudaStream_t)stream;
    PcgState init;
    std::memset(&init, 0, sizeof(init));
    init.tol2 = rtol * rtol;
    init.maxit = maxit;
    for (int k = 0; k < n; ++k) {
        imgm_handle* h = b->hs[k];
        if (!dev_b[k] || !dev_x[k]) return batch_fail(b, IMGM_ERR_INVALID, "null vector");
        if (maxit < 0 || maxit >= h->hist_cap || !(rtol >= 0.0)) return batch_fail(b, IMGM_ERR_INVALID, "bad rtol or maxit");
        const int64_t N = h->lv[h->L - 1].d.N;
        cudaError_t e = cudaMemcpyAsync(h->st, &init, sizeof(init), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->cb, dev_b[k], N * sizeof(double), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->cx, dev_x[k], N * sizeof(double), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return batch_fail(b, IMGM_ERR_CUDA, cudaGetErrorString(e));
    }
    cudaError_t e = cudaGraphLaunch(b->exec, s);
    std::vector<PcgState> fin(n);
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        imgm_handle* h = b->hs[k];
        const int64_t N = h->lv[h->L - 1].d.N;
        e = cudaMemcpyAsync(dev_x[k], h->cx, N * sizeof(double), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&fin[k], h->st, sizeof(PcgState), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return batch_fail(b, IMGM_ERR_CUDA, cudaGetErrorString(e));
    int rc = IMGM_OK;
    for (int k = 0; k < n; ++k) {
        const PcgState& f = fin[k];
        out[k].iterations = f.iter;
        out[k].status = f.status;
        out[k].rel_residual = f.bb > 0 ? std::sqrt(f.rr / f.bb) : 0.0;
        out[k].true_rel_residual = f.bb > 0 ? std::sqrt(f.true_rr / f.bb) : 0.0;
        out[k].kernel_launches = b->kernels[3 * (size_t)k] + (int64_t)f.iter * b->kernels[3 * (size_t)k + 1] +
                                 b->kernels[3 * (size_t)k + 2];
        const int ck = f.status == -5 ? IMGM_ERR_BREAKDOWN : (f.status == 1 ? IMGM_MAX_ITER : IMGM_OK);
        if (rc == IMGM_OK) rc = ck;
    }
    return rc;
}

void imgm_batch_destroy(imgm_batch* b) {
    if (!b) return;
    cudaDeviceSynchronize();
    delete b;
}

// ---- learned correction stage --------------------------------------------------------

namespace {

int net_fail(int code, const std::string& msg) { return fail(nullptr, code, msg); }

#define NCK(call, where)                                                                      \
    do {                                                                                      \
        cudaError_t _e = (call);                                                              \
        if (_e != cudaSuccess) return net_fail(IMGM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(_e)); \
    } while (0)

bool net_dims_ok(int nx, int ny, int nz) {
    return nx >= 1 && ny >= 1 && nz >= 1 && (int64_t)nx * ny * nz <= (int64_t(1) << 31);
}

// the stage's vectors, mask and activations on h's finest grid (allocated once)
int ensure_learned_vectors(imgm_handle* h) {
    if (h->l_r1) return IMGM_OK;
    LevelDev& F = h->lv[h->L - 1];
    const int64_t N = F.d.N;
    CK(h->alloc(&h->l_r1, N), "alloc");
    CK(h->alloc(&h->l_c, N), "alloc");
    CK(h->alloc(&h->l_q, N), "alloc");
    CK(h->alloc(&h->l_mask, N), "alloc");
    const std::vector<uint8_t>& a = h->H.lv[h->L - 1].active;
    CK(cudaMemcpy(h->l_mask, a.data(), (size_t)N, cudaMemcpyHostToDevice), "mask upload");
    CK(cudaMemset(h->l_r1, 0, N * sizeof(double)), "memset");
    CK(cudaMemset(h->l_c, 0, N * sizeof(double)), "memset");
    CK(cudaMemset(h->l_q, 0, N * sizeof(double)), "memset");
    CK(h->lws.ensure(F.d.m, F.d.m, F.d.m, false), "activations");
    return IMGM_OK;
}

}  // namespace

int imgm_net_create(const float* host_weights, imgm_net** out) {
    if (!out) return net_fail(IMGM_ERR_INVALID, "null output network");
    *out = nullptr;
    if (!host_weights) return net_fail(IMGM_ERR_INVALID, "null weights");
    std::unique_ptr<imgm_net> n(new (std::nothrow) imgm_net());
    if (!n) return net_fail(IMGM_ERR_INVALID, "out of host memory");
    const size_t nw = imgm::NET_NW;
    NCK(cudaMalloc(&n->w, nw * sizeof(float)), "alloc");
    NCK(cudaMalloc(&n->g, nw * sizeof(float)), "alloc");
    NCK(cudaMalloc(&n->m, nw * sizeof(float)), "alloc");
    NCK(cudaMalloc(&n->v, nw * sizeof(float)), "alloc");
    NCK(cudaMalloc(&n->wb, nw * sizeof(uint16_t)), "alloc");
    NCK(cudaMalloc(&n->wbt, nw * sizeof(uint16_t)), "alloc");
    NCK(cudaMemcpy(n->w, host_weights, nw * sizeof(float), cudaMemcpyHostToDevice), "weights upload");
    NCK(cudaMemset(n->g, 0, nw * sizeof(float)), "memset");
    NCK(cudaMemset(n->m, 0, nw * sizeof(float)), "memset");
    NCK(cudaMemset(n->v, 0, nw * sizeof(float)), "memset");
    NCK(imgm::net_convert(n->w, n->wb, n->wbt, nullptr), "convert");
    NCK(cudaDeviceSynchronize(), "sync");
    *out = n.release();
    return IMGM_OK;
}

int imgm_net_destroy(imgm_net* net) {
    if (!net) return IMGM_OK;
    if (net->attached > 0)
        return net_fail(IMGM_ERR_INVALID, "the network is still attached to a handle or recorded in a batch");
    cudaDeviceSynchronize();
    delete net;
    return IMGM_OK;
}

int imgm_net_get_weights(const imgm_net* net, float* host_weights) {
    if (!net || !host_weights) return net_fail(IMGM_ERR_INVALID, "null pointer");
    NCK(cudaDeviceSynchronize(), "sync");
    if (int c = net_wait_status(nullptr, net->ws)) return c;
    NCK(cudaMemcpy(host_weights, net->w, imgm::NET_NW * sizeof(float), cudaMemcpyDeviceToHost), "weights");
    return IMGM_OK;
}

int imgm_net_get_grads(const imgm_net* net, float* host_grads) {
    if (!net || !host_grads) return net_fail(IMGM_ERR_INVALID, "null pointer");
    NCK(cudaDeviceSynchronize(), "sync");
    if (int c = net_wait_status(nullptr, net->ws)) return c;
    NCK(cudaMemcpy(host_grads, net->g, imgm::NET_NW * sizeof(float), cudaMemcpyDeviceToHost), "gradients");
    return IMGM_OK;
}

int imgm_net_forward(imgm_net* net, int nx, int ny, int nz, const double* dev_in, const uint8_t* dev_mask,
                     double* dev_out, void* stream) {
    if (!net || !dev_in || !dev_out || dev_in == dev_out) return net_fail(IMGM_ERR_INVALID, "bad pointers");
    if (!net_dims_ok(nx, ny, nz)) return net_fail(IMGM_ERR_INVALID, "bad grid size");
    cudaStream_t s = (cudaStream_t)stream;
    if ((int64_t)nx * ny * nz > net->ws.cap) NCK(cudaStreamSynchronize(s), "sync");
    NCK(net->ws.ensure(nx, ny, nz, net->ws.train), "activations");
    NCK(imgm::net_forward(net->wb, net->ws, dev_in, dev_mask, 1.0, dev_out, nullptr, s), "forward");
    return IMGM_OK;
}

int imgm_net_zero_grad(imgm_net* net, void* stream) {
    if (!net) return net_fail(IMGM_ERR_INVALID, "null network");
    NCK(cudaMemsetAsync(net->g, 0, imgm::NET_NW * sizeof(float), (cudaStream_t)stream), "memset");
    return IMGM_OK;
}

int imgm_net_accumulate(imgm_net* net, int nx, int ny, int nz, const double* dev_in, const double* dev_target,
                        const uint8_t* dev_mask, double in_scale, double scale, double* dev_loss, void* stream) {
    if (!net || !dev_in || !dev_target || !dev_loss) return net_fail(IMGM_ERR_INVALID, "null pointer");
    if (!net_dims_ok(nx, ny, nz)) return net_fail(IMGM_ERR_INVALID, "bad grid size");
    if (!(scale >= 0.0) || !std::isfinite(scale)) return net_fail(IMGM_ERR_INVALID, "bad loss scale");
    if (!(in_scale > 0.0) || !std::isfinite(in_scale)) return net_fail(IMGM_ERR_INVALID, "bad input scale");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nvox = (int64_t)nx * ny * nz;
    if (nvox > net->ws.cap || !net->ws.train) NCK(cudaStreamSynchronize(s), "sync");
    NCK(net->ws.ensure(nx, ny, nz, true), "activations");
    NCK(imgm::net_forward(net->wb, net->ws, dev_in, dev_mask, in_scale, nullptr, net->ws.o, s), "forward");
    NCK(imgm::net_backward(net->wbt, net->ws, dev_target, dev_mask, scale, net->g, dev_loss, s), "backward");
    return IMGM_OK;
}

int imgm_net_adam_step(imgm_net* net, float lr, float beta1, float beta2, float eps, void* stream) {
    if (!net) return net_fail(IMGM_ERR_INVALID, "null network");
    if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return net_fail(IMGM_ERR_INVALID, "bad Adam parameters");
    net->t += 1;
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, (double)net->t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, (double)net->t)));
    NCK(imgm::net_adam(net->w, net->g, net->m, net->v, net->wb, net->wbt, lr, beta1, beta2, eps, c1, c2,
                       (cudaStream_t)stream),
        "adam");
    return IMGM_OK;
}

int imgm_set_net(imgm_handle* h, imgm_net* net) {
    int c = check_level(h, h ? h->L : 0, 1);
    if (c) return c;
    if (net && h->dim != 3) return fail(h, IMGM_ERR_UNSUPPORTED, "the learned stage is three-dimensional");
    if (net && h->precision == 1)
        return fail(h, IMGM_ERR_UNSUPPORTED, "the learned stage follows an FP64 V-cycle output (precision 0 or 2)");
    if (net && (c = ensure_learned_vectors(h)) != IMGM_OK) return c;
    CK(cudaDeviceSynchronize(), "sync");
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->exec = nullptr;
    h->graph = nullptr;
    h->graph_failed = false;
    if (h->net) h->net->attached -= 1;
    if (net) net->attached += 1;
    h->net = net;
    return IMGM_OK;
}

int imgm_set_fcg(imgm_handle* h, int m) {
    int c = check_level(h, h ? h->L : 0, 1);
    if (c) return c;
    if (m < 0 || m > imgm::FCG_MAX) return fail(h, IMGM_ERR_INVALID, "FCG(m) needs 0 <= m <= 8");
    if (m > 0 && h->precision == 1)
        return fail(h, IMGM_ERR_UNSUPPORTED, "FCG(m) takes the FP64 V-cycle output (precision 0 or 2)");
    CK(cudaDeviceSynchronize(), "sync");
    if (m > h->fcg_cap) {
        const int64_t N = h->lv[h->L - 1].d.N;
        CK(h->alloc(&h->fcg_P, (size_t)m * N), "alloc FCG directions");
        CK(h->alloc(&h->fcg_Q, (size_t)m * N), "alloc FCG directions");
        h->fcg_cap = m;
    }
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->exec = nullptr;
    h->graph = nullptr;
    h->graph_failed = false;
    h->fcg_m = m;
    return IMGM_OK;
}

int imgm_learned_stage(imgm_handle* h, const double* dev_r, double* dev_z, double* dev_omega, void* stream) {
    int c = check_level(h, h ? h->L : 0, 1);
    if (c) return c;
    if (!h->net) return fail(h, IMGM_ERR_INVALID, "no network attached");
    if (!dev_r || !dev_z || dev_r == dev_z) return fail(h, IMGM_ERR_INVALID, "bad vector pointers");
    CK(enqueue_learned(h, dev_r, dev_z, dev_omega, (cudaStream_t)stream), "learned stage");
    return IMGM_OK;
}

int imgm_learned_pair(imgm_handle* h, const double* dev_e0, double* dev_r1, double* dev_e1, double* dev_r_rms,
                      void* stream) {
    int c = check_level(h, h ? h->L : 0, 1);
    if (c) return c;
    if (!dev_e0 || !dev_r1 || !dev_e1 || dev_e0 == dev_r1 || dev_e0 == dev_e1 || dev_r1 == dev_e1)
        return fail(h, IMGM_ERR_INVALID, "bad vector pointers");
    if ((c = ensure_learned_vectors(h)) != IMGM_OK) return c;
    cudaStream_t s = (cudaStream_t)stream;
    LevelDev& F = h->lv[h->L - 1];
    const int64_t N = F.d.N;
    CK(imgm::launch_apply<double>(F.d, imgm::APPLY, dev_e0, nullptr, h->l_r1, nullptr, 0.0, nullptr, s), "A e0");
    CK(enqueue_precondition(h, h->l_r1, h->l_c, s), "vcycle");
    CK(imgm::pair_error(N, dev_e0, h->l_c, dev_e1, s), "e1");
    CK(imgm::launch_apply<double>(F.d, imgm::APPLY, dev_e1, nullptr, dev_r1, nullptr, 0.0, nullptr, s), "A e1");
    CK(imgm::pair_normalise(N, dev_r1, dev_e1, (double)F.info.n_active, h->lws.partial, dev_r_rms, s), "normalise");
    return IMGM_OK;
}
