/*
 * imgm -- multigrid-preconditioned conjugate gradients for immersed (cut-cell)
 * B-spline / Lagrange discretisations of the Poisson problem, on one GB300 GPU.
 *
 * Method: de Prenter, Verhoosel, van Brummelen, Evans, Messe, Benzaken, Maute,
 * "Scalable multigrid methods for immersed finite element methods and immersed
 * isogeometric analysis" (arXiv 1903.10977).
 *
 * Conventions used by every entry point
 * -------------------------------------
 * - A level l runs from 1 (coarsest) to L (finest).  Level l has n_l = n / 2^(L-l)
 *   elements per direction and m_l degrees of freedom per direction (open uniform
 *   B-splines: m_l = n_l + p).  A level vector has m_l^d FP64 entries in x-fastest
 *   order (index = ix + m*(iy + m*iz)); entries of inactive functions (no support in
 *   the physical domain, or removed by the u = 0 condition on the box faces) are 0 on
 *   input and are written as 0 on output.
 * - "dev_" pointers are CUDA device pointers owned by the caller; "host_" pointers are
 *   host memory owned by the caller.  The library owns the handle and everything it
 *   allocates in imgm_setup; imgm_destroy frees it.
 * - Every GPU call is ordered on the CUDA stream passed as `stream` (a cudaStream_t;
 *   NULL = the legacy default stream) and returns without waiting for the GPU, unless
 *   its comment says otherwise.  Calls on one handle use the handle's scratch
 *   vectors and must not run concurrently on different streams.
 * - Return value: IMGM_OK (0) or a negative IMGM_ERR_* code; imgm_last_error(h) gives
 *   a message.  No call aborts the process or traps on the GPU.
 *
 * Deliberately narrower than a general interface: imgm_setup is host-synchronous and
 * takes no stream (setup is not on the timed path); Lagrange bases are supported for
 * degree 1 only (the same space as linear B-splines); there is no timeout status (no
 * kernel waits on anything but its own grid; should a tensor-core convolution's bounded
 * wait on its own matrix multiplies give up, it leaves the GPU usable and the next
 * imgm_pcg_solve of a handle with that network, or imgm_net_get_weights / _get_grads,
 * returns IMGM_ERR_CUDA); sizes come from imgm_get_level_info.
 */
#ifndef IMGM_H
#define IMGM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IMGM_OK 0
#define IMGM_ERR_INVALID (-1)      /* bad argument */
#define IMGM_ERR_UNSUPPORTED (-2)  /* configuration outside what is implemented */
#define IMGM_ERR_CUDA (-3)         /* a CUDA runtime call failed */
#define IMGM_ERR_NOT_SPD (-4)      /* a factorisation met a non-positive pivot */
#define IMGM_ERR_BREAKDOWN (-5)    /* CG: p^T A p <= 0 or not finite */
#define IMGM_MAX_ITER 1            /* CG stopped at maxit before reaching rtol (warning) */
/* There is no timeout code: no kernel of this library waits on another grid, a flag set
 * by the host or another device, so every launch ends by itself; a solve that does not
 * converge ends at maxit with IMGM_MAX_ITER. */

typedef struct imgm_handle imgm_handle;

/* Physical domain: the box [lo, hi]^dim minus n_holes disjoint closed balls
 * (level set psi(x) = min_i |x - c_i| - r_i, Omega = {psi > 0}; Sec. 2, Fig. 1).
 * centers: n_holes*dim doubles, row-major; radii: n_holes doubles (host memory,
 * read during imgm_setup only). */
typedef struct {
    int dim;                 /* 2 or 3 */
    int n_holes;
    const double* centers;
    const double* radii;
    double lo, hi;
} imgm_geometry;

/* Discretisation and solver parameters (Sec. 2 and Sec. 3). */
typedef struct {
    int n;                   /* elements per direction on the finest grid; n % 2^(levels-1) == 0 */
    int basis;               /* 0 = uniform open B-splines, 1 = Lagrange (degree 1 only: the same space) */
    int degree;              /* 1, 2 or 3 */
    int levels;              /* L >= 2 multigrid levels (Algorithm 1) */
    int depth;               /* cut-cell bisection depth (Sec. 2, Fig. 1) */
    int bc;                  /* 0 = penalty beta = 2/h (the paper's), 1 = symmetric Nitsche */
    double gamma;            /* additive Schwarz relaxation; <= 0 selects 1/(p+1)^d (Eq. applyCS) */
    int precision;           /* V-cycle arithmetic: 0 = FP64; 1 = FP32 on Jacobi-scaled data inside the
                                FP64 CG, which then uses the flexible (Polak-Ribiere) beta; 2 = the
                                finest level in FP64 and the levels below it in FP32 (flexible CG;
                                additive smoother only) */
    int smoother;            /* 0 = additive Schwarz with relaxation gamma (Sec. 3.4, Eq. applyCS);
                                1 = coloured multiplicative Schwarz (Sec. 3.4): (p+1)^d colours by the
                                owner's index mod p+1, residual updated after each colour, colours
                                reversed in the post-smoothing sweep, no relaxation (gamma unused) */
} imgm_config;

typedef struct {
    int iterations;          /* CG iterations performed */
    int status;              /* IMGM_OK, IMGM_MAX_ITER or IMGM_ERR_BREAKDOWN */
    double rel_residual;     /* ||r_k|| / ||b|| of the recursively updated residual */
    double true_rel_residual;/* ||b - A x|| / ||b||, recomputed at exit */
    int64_t kernel_launches; /* kernels of this library the solve ran on the device (measurement aid;
                                the paper has no counterpart) */
} imgm_result;

typedef struct {
    int64_t n_grid;          /* m^d */
    int64_t n_active;        /* active functions */
    int64_t m;               /* functions per direction */
    int64_t n_band;          /* rows stored explicitly (support touches a non-full element) */
    int64_t n_blocks;        /* Schwarz blocks with more than one function after pruning */
    int64_t block_entries;   /* sum of n_j^2 over those blocks */
    int64_t max_block;       /* largest block */
    int64_t pruned;          /* functions removed from blocks by the tiny-eigenvalue rule */
} imgm_level_info;

/* Builds the immersed discretisation and the whole multigrid hierarchy on the host
 * (cut-cell quadrature, assembly of the stored rows, two-scale restriction, Galerkin
 * coarse rows R A R^T, Schwarz blocks with encapsulating supports and the Remark 3.3
 * rule, coarsest-level inverse) and uploads it to the current CUDA device.
 * Sec. 2 (discretisation), Sec. 3.3 (Eq. coarsening, Remark 3.1), Sec. 3.4 (blocks,
 * Remark 3.3).  Synchronous: it takes no stream, builds everything on the host (OpenMP),
 * uploads it and times the setup-time autotuner's candidates on a stream of its own, and
 * returns after the device has finished; the handle's tables are then read-only.  On
 * success *out receives a new handle. */
int imgm_setup(const imgm_geometry* geom, const imgm_config* cfg, imgm_handle** out);

/* Frees everything the handle owns (device and host).  Waits for the device. */
void imgm_destroy(imgm_handle* h);

/* Message for the last failed call on h (or on a failed imgm_setup when h == NULL). */
const char* imgm_last_error(const imgm_handle* h);

/* Number of levels L. */
int imgm_levels(const imgm_handle* h);

/* Sizes and setup statistics of one level (1 <= level <= L). */
int imgm_get_level_info(const imgm_handle* h, int level, imgm_level_info* info);

/* Active-function mask of a level into host_mask (n_grid bytes, 1 = active). */
int imgm_active_mask(const imgm_handle* h, int level, uint8_t* host_mask);

/* Right-hand side b of the built-in manufactured problem u = prod sin(pi x_k)
 * (finest level, Eq. operatorsMulti) into dev_b (n_grid doubles). */
int imgm_rhs(imgm_handle* h, double* dev_b, void* stream);

/* dev_y = A_l dev_x on level l (Eq. systemMulti on the finest level; the Galerkin
 * operator R A R^T of Remark 3.1 on coarser levels).  dev_x and dev_y must not overlap. */
int imgm_apply_operator(imgm_handle* h, int level, const double* dev_x, double* dev_y, void* stream);

/* dev_z = gamma M_l^{-1} dev_r with the additive Schwarz operator
 * M^{-1} = sum_j P_j A_j^{-1} P_j^T (Sec. 3.4), level l >= 2. */
int imgm_smooth(imgm_handle* h, int level, const double* dev_r, double* dev_z, void* stream);

/* dev_rc = R_l dev_r: restriction from level l >= 2 to level l-1 (Eq. coarsening). */
int imgm_restrict(imgm_handle* h, int level, const double* dev_r, double* dev_rc, void* stream);

/* dev_e = R_l^T dev_xc: prolongation from level l-1 to level l >= 2 (Sec. 3.3). */
int imgm_prolong(imgm_handle* h, int level, const double* dev_xc, double* dev_e, void* stream);

/* dev_x = A_1^{-1} dev_r on the coarsest level (Algorithm 1, direct solve). */
int imgm_coarse_solve(imgm_handle* h, const double* dev_r, double* dev_x, void* stream);

/* dev_z = B dev_r: one V-cycle of Algorithm 1 from the finest level (the CG
 * preconditioner of Sec. 3.2).  dev_r is not modified. */
int imgm_apply_preconditioner(imgm_handle* h, const double* dev_r, double* dev_z, void* stream);

/* Solves A x = b by CG preconditioned with one V-cycle per iteration (Sec. 3.2), from
 * the initial guess in dev_x, until ||r_k|| <= rtol ||b|| or maxit iterations.  dev_x
 * receives the solution.  dev_hist (nullable, maxit+1 doubles) receives ||r_k||/||b||.
 * Waits for the device before returning (it reports *out). */
int imgm_pcg_solve(imgm_handle* h, const double* dev_b, double* dev_x, double rtol, int maxit,
                   imgm_result* out, double* dev_hist, void* stream);

/* imgm_pcg_solve with host buffers: copies host_b to the device, solves from x = 0,
 * copies the solution to host_x (n_grid doubles each).  Synchronous. */
int imgm_pcg_solve_host(imgm_handle* h, const double* host_b, double* host_x, double rtol, int maxit,
                        imgm_result* out, void* stream);

/* dev_out[0] = ||dev_b - A dev_x||_2^2 on the finest level (the residual of Eq.
 * residualMulti, whose norm is the stopping quantity of the CG solve of Sec. 3.2).
 * dev_b and dev_x: n_grid doubles; dev_out: one double.  Uses the handle's scratch
 * vectors, so it must not overlap other calls on the same handle. */
int imgm_residual_norm2(imgm_handle* h, const double* dev_b, const double* dev_x, double* dev_out, void* stream);

/* imgm_residual_norm2 for callers that cannot allocate device memory while they run
 * (a process whose memory a caching allocator has reserved up front, or a latency-
 * critical loop that cannot afford cudaMalloc's device-wide synchronisation).  The paper
 * has no counterpart: this is an interface variant, not a step of the method.
 * Same arguments and result as imgm_residual_norm2; it calls no cudaMalloc, cudaFree or
 * allocating library routine.  Its scratch is a static device array of 4 MiB that
 * every GPU loading the library holds until the process exits; it serves finest levels
 * of at most 2^19 rows and returns IMGM_ERR_UNSUPPORTED, with a message naming the
 * limit, for larger ones.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) and should come before any stream capture on that
 * device.  All calls share the one array, so calls that overlap on the GPU (different
 * streams, handles or threads) race and give wrong results; serialise them. */
int imgm_residual_norm2_noalloc(imgm_handle* h, const double* dev_b, const double* dev_x, double* dev_out,
                                void* stream);

/* ---- Solve contexts and batches -------------------------------------------------
 * Several solves at once: the per-solve work of Sec. 3.2 (CG with the V-cycle of
 * Algorithm 1) is unchanged; what is new is only how many run together.  The paper has
 * no counterpart. */

/* A second solve context for the problem of h: it shares h's host hierarchy and device
 * tables (read-only; freed when the last of h and its clones is destroyed) and owns its
 * own vectors, reduction scratch and solve graph, so that it can solve at the same time as
 * h (another right-hand side of the same geometry).  Returns IMGM_ERR_INVALID for a
 * host-only handle, IMGM_ERR_CUDA if device memory runs out. */
int imgm_clone(const imgm_handle* h, imgm_handle** out);

typedef struct imgm_batch imgm_batch;

/* One CUDA graph that runs the CG solves of the n contexts hs[0..n) concurrently, each on
 * its own branch with its own device-side convergence loop (conditional WHILE node), so
 * that one graph launch solves them all.  The contexts must be distinct (clone a context
 * for more right-hand sides of one problem), may belong to different problems of any
 * size, and must outlive the batch.  Errors: IMGM_ERR_INVALID (empty list, repeated or
 * host-only context), IMGM_ERR_CUDA (stream capture or instantiation failed; the message
 * is in imgm_last_error(NULL)). */
int imgm_batch_create(imgm_handle* const* hs, int n, imgm_batch** out);

/* Solves hs[k] x_k = b_k for every k with one graph launch on `stream` (cudaStream_t, NULL
 * for the default stream): dev_b[k] and dev_x[k] are device vectors of n_grid doubles of
 * context k (x_k in: initial guess, out: solution), rtol and maxit as in imgm_pcg_solve.
 * out[k] receives each solve's result.  Waits for the device.  Returns IMGM_OK when every
 * solve converged, else the status of the first solve that did not. */
int imgm_batch_solve(imgm_batch* b, const double* const* dev_b, double* const* dev_x, double rtol, int maxit,
                     imgm_result* out, void* stream);

void imgm_batch_destroy(imgm_batch* b);

/* ---- Learned correction stage ------------------------------------------------------
 * An extension beside the paper's method (which has no learned part): after the V-cycle
 * of Algorithm 1 gives z = B r, a small network proposes c = N(r - A z) and z becomes
 * z + omega c with omega = ((r - A z) . c) / (c . A c), the step that minimises the A-norm
 * of the error of A e = r along c (omega = 0 unless c . A c > 0).  CG then takes the
 * Polak-Ribiere beta z_{k+1} . (r_{k+1} - r_k) / (z_k . r_k), as the preconditioner now
 * varies from step to step.
 *
 * N: three 3-D convolutions on the grid of basis functions (1 -> 16 -> 16 -> 1 channels,
 * 3 x 3 x 3 kernels, zero padding, no biases, ReLU after the first two), weights read as
 * bfloat16, activations stored as bfloat16, sums in FP32.  The input is rounded FP64 ->
 * FP32 -> bfloat16 and zeroed off the mask; the output is zero off the mask.
 * Weights: IMGM_NET_WEIGHTS floats, layer by layer, each layer [tap][out][in] with
 * tap = 9 (dz + 1) + 3 (dy + 1) + (dx + 1); a grid vector of nx * ny * nz entries is
 * indexed x + nx (y + ny z) (a finest-level vector of a 3-D problem: nx = ny = nz = m).
 * Network calls report errors through imgm_last_error(NULL): IMGM_ERR_INVALID for a null
 * pointer, an empty grid or a bad scale or Adam parameter (checked before any CUDA call),
 * IMGM_ERR_CUDA when an allocation or launch fails.  Device vectors passed in stay owned
 * by the caller; the library keeps no pointer to them after a call returns (a network
 * owns its weights, Adam state and activation buffers; a handle owns its stage vectors). */
#define IMGM_NET_WEIGHTS 7776

typedef struct imgm_net imgm_net;

/* A network with the given FP32 weights (host array, copied) and zero Adam state. */
int imgm_net_create(const float* host_weights, imgm_net** out);
/* Frees the network (waits for the device) and returns IMGM_OK; NULL is a no-op.
 * A network counts its attachments: every handle it is attached to (imgm_set_net) and
 * every batch created while one of its handles held it (the batch's recorded solves read
 * its weights, whatever imgm_set_net does to the handle afterwards).  While that count is
 * above zero the call frees nothing and returns IMGM_ERR_INVALID (message in
 * imgm_last_error(NULL)): detach it from its handles (or destroy them) and destroy those
 * batches first. */
int imgm_net_destroy(imgm_net* net);
/* Copies the FP32 master weights / the gradient accumulator to the host (waits). */
int imgm_net_get_weights(const imgm_net* net, float* host_weights);
int imgm_net_get_grads(const imgm_net* net, float* host_grads);

/* dev_out = N(dev_in) on an nx x ny x nz grid (device doubles; dev_mask: device bytes,
 * 1 = active, or NULL for all).  Uses the network's own activation buffers (grown on
 * demand, which waits for the stream), so calls on one network must not overlap. */
int imgm_net_forward(imgm_net* net, int nx, int ny, int nz, const double* dev_in, const uint8_t* dev_mask,
                     double* dev_out, void* stream);

/* Training.  zero_grad clears the gradient accumulator; accumulate adds the gradient of
 * L = scale * sum_v m_v (N(in_scale in)_v - target_v)^2 (reverse mode through the stored
 * activations; in_scale > 0 multiplies the input before its rounding to bfloat16) and
 * adds L to dev_loss[0] (a device double the caller zeroes);
 * adam_step applies one Adam step (Kingma and Ba, 2015) with bias correction to the
 * FP32 weights and refreshes their bfloat16 copies. */
int imgm_net_zero_grad(imgm_net* net, void* stream);
int imgm_net_accumulate(imgm_net* net, int nx, int ny, int nz, const double* dev_in, const double* dev_target,
                        const uint8_t* dev_mask, double in_scale, double scale, double* dev_loss, void* stream);
int imgm_net_adam_step(imgm_net* net, float lr, float beta1, float beta2, float eps, void* stream);

/* Attaches net to h's solves (NULL detaches): imgm_pcg_solve then runs the stage after
 * every V-cycle.  The network must outlive the attachment.  IMGM_ERR_UNSUPPORTED for a
 * 2-D problem or precision 1 (the stage follows an FP64 V-cycle output).  Rebuilds the
 * solve graph on the next solve.  A batch keeps the stage as it was when the batch was
 * created: batches created before the call keep their V-cycle (with or without a
 * network), and a batch created while a network was attached runs that network until
 * it is destroyed (and holds one attachment of it; see imgm_net_destroy). */
int imgm_set_net(imgm_handle* h, imgm_net* net);

/* Truncated flexible CG for h's solves, FCG(m) (Notay, "Flexible conjugate gradients",
 * SIAM J. Sci. Comput. 22, 2000): each new direction is the preconditioned residual z
 * A-orthogonalised against the last m directions, p = z - sum_j (z^T A p_j)/(p_j^T A p_j) p_j,
 * and alpha = (r^T p)/(p^T A p).  For a fixed SPD preconditioner it is plain PCG up to
 * rounding; with the learned stage (a preconditioner that varies from step to step) the
 * m stored directions keep more of the Krylov acceleration than the one-direction
 * Polak-Ribiere form.  m = 0 returns to the default (PCG, or Polak-Ribiere with a network
 * or an FP32 V-cycle); 1 <= m <= 8.  Allocates 2 m n_grid doubles on the first call with a
 * larger m (synchronous; call it outside stream capture).  Errors: IMGM_ERR_INVALID (m out
 * of range), IMGM_ERR_UNSUPPORTED (precision 1: its V-cycle output is FP32), IMGM_ERR_CUDA.
 * The paper has no counterpart: its CG takes the fixed V-cycle of Algorithm 1. */
int imgm_set_fcg(imgm_handle* h, int m);

/* One stage with the attached network: dev_z (in: B dev_r, out: the corrected value);
 * dev_omega (device double, may be NULL) receives omega. */
int imgm_learned_stage(imgm_handle* h, const double* dev_r, double* dev_z, double* dev_omega, void* stream);

/* A training pair from the V-cycle of h: e1 = e0 - B A e0, r1 = A e1, both divided by the
 * root mean square of e1 over the active functions (dev_e0 active-supported; three
 * distinct device vectors of n_grid doubles).  dev_r_rms (device double, may be NULL)
 * receives the root mean square of the scaled r1: the mean over a training set gives the
 * set's input scale (1 / mean), one factor for every pair, since r1 shrinks with the mesh
 * size while e1 does not. */
int imgm_learned_pair(imgm_handle* h, const double* dev_e0, double* dev_r1, double* dev_e1, double* dev_r_rms,
                      void* stream);

/* ---- Setup inspection (host only; no GPU needed) --------------------------------
 * imgm_setup_host builds the same hierarchy as imgm_setup without touching the GPU;
 * such a handle serves only the imgm_host_* calls below, imgm_levels,
 * imgm_get_level_info and imgm_active_mask.  These calls copy setup data out for testing
 * and inspection; they compute none of the solve. */
int imgm_setup_host(const imgm_geometry* geom, const imgm_config* cfg, imgm_handle** out);

/* Operator rows of level l: for each of the nrows full-grid row indices in rows,
 * the (2p+1)^d coefficients A[row, row + o] for offsets o in [-p, p]^d (x fastest),
 * into out (nrows * (2p+1)^d doubles).  0 for inactive rows and columns. */
int imgm_host_operator_rows(const imgm_handle* h, int level, int64_t nrows, const int64_t* rows, double* out);

/* Finest-level right-hand side (n_grid doubles). */
int imgm_host_rhs(const imgm_handle* h, double* out);

/* Schwarz data of level l >= 2: sizes first, then the arrays (block k holds rows
 * idx[ptr[k]:ptr[k+1]] and the column-major inverse val[vptr[k]:vptr[k+1]]; dinv[i] is
 * the sum of 1/A_ii over the one-function blocks that hold row i). */
int imgm_host_block_sizes(const imgm_handle* h, int level, int64_t* nblk, int64_t* nidx, int64_t* nval);
int imgm_host_blocks(const imgm_handle* h, int level, int64_t* ptr, int32_t* idx, int64_t* vptr, double* val,
                     double* dinv);

/* 1-D restriction table of level l >= 2: coarse function i of level l-1 equals
 * sum_k w[i*(p+2)+k] phi_{first[i]+k} of level l (m_{l-1} entries of first). */
int imgm_host_restriction(const imgm_handle* h, int level, int32_t* first, double* w);

/* Coarsest-level inverse: nc kept rows and the nc x nc row-major inverse on them. */
int imgm_host_coarse_size(const imgm_handle* h, int64_t* nc);
int imgm_host_coarse(const imgm_handle* h, int32_t* rows, double* inv);

#ifdef __cplusplus
}
#endif

#endif /* IMGM_H */
