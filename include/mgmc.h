/*
 * mgmc.h -- C ABI of the GB300 Multigrid Monte Carlo (MGMC) sampler.
 *
 * The sampler draws from the Gaussian posterior N(mu, A~^-1),
 *   A~ = A + B Gamma^-1 B^T,  mu = A~^-1 f,  f = B Gamma^-1 y,
 * (Sec. 2.2, Eqs. post-mean / post-cov / f_ell_definition of Kazashi, Mueller,
 * Scheichl, "Multigrid Monte Carlo Revisited", arXiv 2407.12149), where A is
 * the finite-difference precision s (kappa^2(x) I - Delta_h) on the interior
 * vertices of the unit square or cube with zero Dirichlet values and
 * s = h^d (default, the bilinear-form scaling of Sec. 2.3) or s = 1.
 * One call of mgmc_sample applies n_steps MGMC V-cycles (Alg. 1, gamma = 1)
 * with the paper's Gibbs smoother with low-rank correction (Alg. 3: nu1
 * forward sweeps before the coarse-grid correction, nu2 backward sweeps
 * after it), Galerkin coarse operators (Eq. galerkin_triple_product),
 * restriction = transpose of the multilinear prolongation, and an exact
 * Cholesky sampler on the coarsest grid (Sec. 3.5).
 *
 * Conventions used by every entry point:
 *   - Grids are cubes: n interior points per axis, n = 2^k - 1; level
 *     l-1 has (n_l - 1)/2 points per axis.  A dense field of a grid holds
 *     n^dim values, site s = i + n (j + n k), x fastest.
 *   - Host arrays passed to mgmc_create are copied; the caller keeps
 *     ownership.  Device buffers the handle needs are obtained from the
 *     caller's allocator (or cudaMalloc when the allocator is NULL) and are
 *     returned to it by mgmc_destroy.
 *   - Work is ordered on the CUDA stream passed in (a cudaStream_t given as
 *     void*; NULL = legacy default stream).  mgmc_sample returns once the
 *     work is queued unless a host pointer was passed; mgmc_mean_solve and
 *     mgmc_qoi_stats synchronise that stream.
 *   - No exception crosses this boundary.  Every function returns a status;
 *     mgmc_last_error() gives a message for the last failing call on the
 *     calling thread.  There is no CPU fallback: without a usable CUDA
 *     device the calls fail with MGMC_ERR_CUDA.
 *   - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef MGMC_H
#define MGMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MGMC_OK = 0,
    MGMC_ERR_ARG = 1,      /* invalid argument (size not 2^k-1, NaN input, bad pointer, ...) */
    MGMC_ERR_CUDA = 2,     /* CUDA runtime error or no device */
    MGMC_ERR_OOM = 3,      /* allocator returned NULL */
    MGMC_ERR_NOT_SPD = 4,  /* Gamma, a coarse operator or A~_0 is not symmetric positive definite */
    MGMC_ERR_TIMEOUT = 5,  /* a bounded device-side wait gave up */
    MGMC_ERR_STATE = 6,    /* handle in the wrong state for this call */
    MGMC_ERR_NUMERIC = 7   /* non-finite value produced */
} mgmc_status;

enum { MGMC_FP64 = 0, MGMC_FP32 = 1 };

/* Maximum number of observations (columns of B). */
#define MGMC_MAX_OBS 64
/* Maximum number of unknowns on the coarsest grid (dense Cholesky). */
#define MGMC_MAX_COARSEST 1024

typedef struct mgmc_ctx* mgmc_handle;

/* Device-memory provider.  alloc(bytes, stream, ctx) returns device memory
 * or NULL; free(ptr, stream, ctx) returns it.  Both are called only from
 * mgmc_create / mgmc_destroy on the caller's thread. */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void (*free)(void* ptr, void* stream, void* ctx);
    void* ctx;
} mgmc_allocator;

typedef struct {
    int dim;          /* 2 or 3 */
    int n;            /* interior points per axis of the finest grid, 2^k - 1 */
    int n_levels;     /* number of grids (>= 1); 0 = coarsen down to n = 1 */
    int nu1, nu2;     /* forward / backward smoothing sweeps per level (paper: 1, 1) */
    int precision;    /* MGMC_FP64 or MGMC_FP32: type of the smoother, transfer and
                         state arithmetic; the low-rank update, coarsest Cholesky
                         sample and QoI accumulation are FP64 in both */
    int scale_hd;     /* 1: A = h^d (kappa^2 - Delta_h) (default); 0: kappa^2 - Delta_h */
    int coarse_max_n; /* grids with n <= coarse_max_n run inside one single-CTA kernel;
                         0 selects the default (63 in 2D, 15 in 3D) */
    int gibbs;        /* 0: the MGMC V-cycle (Alg. 1).  1: the plain Gibbs sampler the
                         paper compares against (Sec. 5.1.3): one step is nu1 forward and
                         nu2 backward sweeps of the low-rank Gibbs smoother (Alg. 3) on
                         the finest grid alone, with the MGMC cycle's noise slots and no
                         coarse-grid correction.  Needs n_levels >= 2 (the finest grid's
                         low-rank data are those of MGMC); single-chain handles only
                         (mgmc_create_batch returns MGMC_ERR_ARG). */
    int disc;         /* discretisation of kappa^2 - Delta on the finest grid (Sec. 5.1.1):
                         MGMC_FD (default): the 5/7-point finite-difference stencil;
                         MGMC_Q1: the lowest-order conforming multilinear finite-element
                         matrix, a_ij = int grad phi_i . grad phi_j + kappa^2 phi_i phi_j
                         (9/27-point; constant kappa^2 only: kappa2 must be NULL), divided
                         by h^d when scale_hd = 0.  The coarse grids are Galerkin products
                         either way (for Q1 they are the Q1 matrices of the coarse grids).
                         MGMC_SSL: the squared shifted Laplacian (kappa^2 - Delta)^2 of
                         Eq. squared_shifted_laplace with u = du/dn = 0 (Sec. 5.1.1), the
                         13-point finite-difference stencil h^-4 [20, -8, 2, 1] with mirror
                         ghosts behind the boundary vertices, plus 2 kappa^2 (-Delta_h) and
                         kappa^4, times h^2 (scale_hd = 1); 2D, constant kappa^2, FP64.  Every
                         grid carries a radius-2 (5 x 5) stencil and is swept in the nine
                         colours (i mod 3, j mod 3); the general (one launch per colour) path
                         runs every grid but the coarsest, which is sampled exactly. */
    int band_min_n;   /* 2D FP32 V-cycles (nu1 = nu2 = 1): the 9-point grids below the finest
                         with n >= band_min_n (and above coarse_max_n) run in the streaming
                         band kernels, the smaller ones in shared-memory tile kernels.  0 selects
                         the default (255); a value above n keeps every grid on the tiles.  Both
                         kernel families give bitwise identical states; a batch takes the value
                         of its first configuration. */
    int gamma;        /* cycle index of Alg. 1: 1 V-cycle, 2 W-cycle (the finest grid calls the
                         next grid once, every coarser grid calls its coarse grid twice, the
                         coarse state carried from one call to the next; Sec. 5.1.3 uses it
                         for MGMC_SSL); 0 selects 2 for MGMC_SSL and 1 otherwise.  The v-th
                         visit of a grid within a cycle draws its sweep noise with slots
                         2 (v S + j) (pre) and 2 (v S + j) + 1 (post), S = max(nu1, nu2, 1),
                         and the coarsest grid's v-th sample with slot v; a W-cycle runs on
                         the general path with the coarsest grid alone in the coarse kernel.
                         Single-chain handles only (mgmc_create_batch takes 0 or 1). */
} mgmc_config;

enum { MGMC_FD = 0, MGMC_Q1 = 1, MGMC_SSL = 2 };

/* Fill cfg with the paper's defaults for a dim-dimensional n^dim grid. */
mgmc_status mgmc_config_default(mgmc_config* cfg, int dim, int n);

/* Create a sampler for one posterior (Sec. 2.2 / 2.3).
 *   kappa2:       host [n^dim] kappa^2 at the fine vertices, or NULL to use kappa2_const.
 *   m:            number of observations beta (0 <= m <= MGMC_MAX_OBS).
 *   obs_site/obs_w: host [m * nnz_per_obs]: row k of B^T as (fine site, weight);
 *                 site -1 marks an unused entry (e.g. a Dirichlet boundary vertex).
 *   Gamma:        host [m * m] row-major SPD observation-noise covariance.
 *   y:            host [m] observed values.
 *   n_qoi, qoi_site, qoi_w: host sparse F_L of the linear QoI F_L^T x (Eq. F_matrix).
 * Errors: MGMC_ERR_ARG (sizes, non-finite values, sites out of range),
 * MGMC_ERR_NOT_SPD, MGMC_ERR_OOM, MGMC_ERR_CUDA.  *out is NULL on error. */
mgmc_status mgmc_create(const mgmc_config* cfg, const mgmc_allocator* alloc, void* stream,
                        const double* kappa2, double kappa2_const,
                        int m, const int32_t* obs_site, const double* obs_w, int nnz_per_obs,
                        const double* Gamma, const double* y,
                        int n_qoi, const int32_t* qoi_site, const double* qoi_w,
                        mgmc_handle* out);

/* Rows of B for point observations at xyz (host [m * dim], each in (0,1)^dim):
 * the 2^dim multilinear interpolation weights of the enclosing cell
 * (Eq. B_ell_definition for point evaluation).  obs_site / obs_w: host
 * [m * 2^dim]; vertices on the boundary get site -1, weight 0.  Corner c's
 * bit a selects the upper vertex along axis a. */
mgmc_status mgmc_point_obs_rows(int dim, int n, int m, const double* xyz, int32_t* obs_site, double* obs_w);

/* Apply n_steps MGMC V-cycles to x_inout (dense n^dim field in the handle's
 * precision; device or host memory).  Cycle t uses the random numbers of
 * cycle index step_offset + t, so runs split at any point reproduce a single
 * run bit for bit.  chain (< 65536) selects an independent random stream.
 * qoi_out: NULL or [n_steps] doubles (device or host) receiving F_L^T x
 * after every cycle.  Host buffers are staged through device memory on the
 * stream and the call synchronises it before returning.
 * x_inout = NULL continues from the state the handle holds (the state after
 * the previous call, zero after mgmc_create) and leaves the new state there:
 * nothing is copied in or out; mgmc_get_state reads it. */
mgmc_status mgmc_sample(mgmc_handle h, int64_t n_steps, uint64_t seed, uint64_t step_offset,
                        uint32_t chain, void* x_inout, double* qoi_out, void* stream);

/* Posterior mean by noise-free V-cycles (deterministic multigrid; the multigrid / MGMC equivalence of Sec. 4):
 * iterates from mean_out (dense n^dim field, handle precision, device or
 * host) until ||f - A~ x||_2 <= rtol ||f||_2 or max_cycles.  Synchronous.
 * cycles_done / rel_residual may be NULL. */
mgmc_status mgmc_mean_solve(mgmc_handle h, double rtol, int max_cycles, void* mean_out,
                            int* cycles_done, double* rel_residual, void* stream);

typedef struct {
    double mean;      /* sample mean of the kept series */
    double var;       /* lag-0 autocovariance */
    double tau_int;   /* IACT, tau = 1 + 2 sum_{t=1}^{W} rho(t) (Sec. 5.3.2) */
    double tau_err;   /* its statistical error (Wolff 2004, Eq. 42) */
    double ess;       /* effective sample size n_used / tau_int */
    int64_t window;   /* Wolff's automatic window W */
    int64_t n_used;   /* n - burn_in */
} mgmc_stats;

/* Chain statistics of a QoI series on the device (Sec. 5.3.2): lagged
 * autocovariance with divisor n - t and Wolff's automatic window with
 * parameter S (1.5 if S <= 0), computed by CUDA kernels.  qoi: device
 * [n] doubles; the first burn_in entries are skipped.  Scratch of
 * (n - burn_in)/2 + 1 doubles comes from cudaMallocAsync on the stream.
 * Synchronous. */
mgmc_status mgmc_qoi_stats(const double* qoi, int64_t n, int64_t burn_in, double S, mgmc_stats* out,
                           void* stream);

/* Longest series (n - burn_in) mgmc_qoi_stats_noalloc accepts. */
#define MGMC_NOALLOC_MAX_SERIES 65536

/* The same statistics as mgmc_qoi_stats for callers that cannot allocate
 * device memory while they run: for example a process whose device memory
 * is held entirely by another framework's pool, or a latency-critical
 * monitoring loop that must not wait on an allocator.  The paper has no
 * counterpart; this is a library convenience.
 * Scratch lives in one fixed device array of about 264 KB inside the library
 * (every GPU that loads the library keeps it until the process exits); no
 * allocation or free of any kind is made.  All lags t <= (n - burn_in)/2 are
 * evaluated in one pass, so n - burn_in may be at most
 * MGMC_NOALLOC_MAX_SERIES (else MGMC_ERR_ARG).  The first call on a device
 * also looks up the scratch address for that device.  The call copies its
 * result to host memory and synchronises the stream, so it must not be made
 * while that stream is being captured into a CUDA graph.  All calls share the
 * one scratch array: calls that may overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller. */
mgmc_status mgmc_qoi_stats_noalloc(const double* qoi, int64_t n, int64_t burn_in, double S, mgmc_stats* out,
                                   void* stream);

/* The finest grid's operator A_L (without the observation term) exactly as
 * mgmc_create assembles it from cfg->dim, n, scale_hd and disc (Sec. 2.3 /
 * 5.1.1): out = host [n^dim * W^dim], W = 2R + 1 with the stencil radius R (2 for
 * MGMC_SSL, else 1), the coupling of site s to site s + o at out[s * W^dim + o],
 * offset o = (dx+R) + W (dy+R) [+ W^2 (dz+R)], 0 where the neighbour is a
 * boundary vertex.  kappa2: host [n^dim] or NULL (kappa2_const).
 * Host only: needs no device.  MGMC_ERR_ARG for bad sizes or values. */
mgmc_status mgmc_fine_operator(const mgmc_config* cfg, const double* kappa2, double kappa2_const, double* out);

/* Number of grids, unknowns per axis of grid l (0 = coarsest) and the
 * precision of a handle. */
mgmc_status mgmc_info(mgmc_handle h, int* n_levels, int* precision, int* dim);
mgmc_status mgmc_level_n(mgmc_handle h, int l, int* n);

/* Kernels launched per V-cycle by mgmc_sample (for launch accounting). */
mgmc_status mgmc_launches_per_cycle(mgmc_handle h, int* launches);

/* One posterior problem of a batch (the arguments of mgmc_create). */
typedef struct {
    const double* kappa2;
    double kappa2_const;
    int m;
    const int32_t* obs_site;
    const double* obs_w;
    int nnz_per_obs;
    const double* Gamma;
    const double* y;
    int n_qoi;
    const int32_t* qoi_site;
    const double* qoi_w;
} mgmc_problem;

/* A batch of independent chains (2D, nu1 = nu2 = 1, one precision; grid sizes,
 * kappa^2, observations and QoI may differ per chain) advanced together: each
 * phase of the V-cycle (Alg. 1) is one launch over the same grid depth of all
 * chains, the coarse grids of each chain run in one CTA of a batched launch.
 * Chain c uses the Philox chain id c, so it reproduces mgmc_sample with
 * chain = c on a handle created from cfgs[c] with the same coarse_max_n
 * (default 31 here).  All host arrays are copied. */
mgmc_status mgmc_create_batch(int n_chains, const mgmc_config* cfgs, const mgmc_problem* problems,
                              const mgmc_allocator* alloc, void* stream, mgmc_handle* out);

/* n_steps V-cycles of every chain of a batch handle.  x_inout: host array of
 * n_chains pointers to chain c's dense n_c^2 state -- all in device memory, or
 * all in host memory (copied in and out through the device inside the call, one
 * copy per chain and direction) -- or NULL to continue from the states the
 * handle holds (as in mgmc_sample); qoi_out: NULL, or device or host
 * [n_chains * n_steps] (row c = chain c).  Asynchronous on stream when every
 * buffer is device memory; with any host buffer the call synchronises the stream
 * and reports the chains' sticky status bits (as mgmc_check_status).
 * MGMC_ERR_ARG when host and device states are mixed. */
mgmc_status mgmc_sample_batch(mgmc_handle h, int64_t n_steps, uint64_t seed, uint64_t step_offset,
                              void* const* x_inout, double* qoi_out, void* stream);

/* Copy the state a handle holds for chain `chain` (0 for a single-chain handle,
 * 0 .. n_chains-1 for a batch) into x_out: dense n^dim field in the handle's
 * precision, device or host memory (host: the call synchronises the stream).
 * MGMC_ERR_ARG for a bad chain index or NULL x_out. */
mgmc_status mgmc_get_state(mgmc_handle h, int chain, void* x_out, void* stream);

/* The sticky status of every chain of a handle: the kernels set a bit when a
 * bounded wait for a staging copy gave up or a QoI was not finite, and the bits
 * stay set (across calls) until reported.  Synchronises the stream, returns
 * MGMC_ERR_TIMEOUT (a wait gave up; the chain's state is not a valid sample) or
 * MGMC_ERR_NUMERIC (non-finite QoI), else MGMC_OK, and clears the bits.
 * mgmc_sample, mgmc_sample_batch with host buffers and mgmc_mean_solve report
 * them the same way whenever they synchronise. */
mgmc_status mgmc_check_status(mgmc_handle h, void* stream);

/* Bound of the kernels' staging waits of every chain of a handle, for tests of
 * the timeout path: 0 restores the default (1 s), a positive value is that many
 * nanoseconds, a negative value makes every staging wait give up at once (the
 * kernel then flags MGMC_ERR_TIMEOUT, lets its copies in flight land within the
 * default bound and ends; the chain's state is garbage until it is re-set).
 * Synchronises the device. */
mgmc_status mgmc_set_wait_limit(mgmc_handle h, int64_t limit_ns);

/* Change band_min_n (see mgmc_config) of a handle after creation: the job tables
 * of both kernel families exist from mgmc_create / mgmc_create_batch on, so this
 * only selects, per grid depth, which one the captured cycle launches (the graph is
 * captured again on the next call that samples).  The states do not depend on the
 * choice.  Synchronises the device when the choice changes.  MGMC_ERR_ARG for a
 * negative value.  (An autotuner uses it to time the settings on one handle.) */
mgmc_status mgmc_set_band_min_n(mgmc_handle h, int band_min_n);

/* Threads per CTA of the 2D coarse-grid kernel (one CTA per chain, all grids with
 * n <= coarse_max_n in shared memory): 0 (default) chooses 1024 while the chains
 * leave SMs free and 256 once several chains share an SM; else a multiple of 32 in
 * [64, 1024].  The kernel's arithmetic does not depend on it (the states are bitwise
 * the same); only the time of its barrier-bound phases does.  The graph is captured
 * again on the next sampling call.  MGMC_ERR_ARG for other values. */
mgmc_status mgmc_set_coarse_threads(mgmc_handle h, int threads);

/* Benchmark timing: with enable != 0 the captured cycle records CUDA events
 * around the finest grid's forward sweep and its backward sweep (finest grid
 * above coarse_max_n only).  mgmc_profile_times synchronises the stream given
 * and writes ms[0] = forward sweep, ms[1] = backward sweep of the last cycle
 * run (n >= 2).  MGMC_ERR_STATE when profiling is off or the finest grid runs
 * inside the single-CTA kernel. */
mgmc_status mgmc_set_profiling(mgmc_handle h, int enable);
mgmc_status mgmc_profile_times(mgmc_handle h, float* ms, int n, void* stream);

mgmc_status mgmc_destroy(mgmc_handle h);

/* ------------------------------------------------------------------------
 * Learned warm start (not in the paper): a U-Net maps three input channels
 * on the (n+1) x (n+1) grid -- log(kappa^2 / 10), the summed observation row
 * weights sum_k B_{k,i} and the weighted data sum_k B_{k,i} y_k, with the last
 * row and column zero -- to an estimate of the posterior mean mu = A~^-1 f
 * (Sec. 2.2), to be used ONLY as a chain's initial state: the chain's law is
 * that of the sampler whatever x_0 is; a good x_0 shortens burn-in.
 * Channels-last BF16 activations and weights, FP32 accumulation on the tcgen05
 * tensor cores.  c0 channels at full resolution, doubling at each of three
 * 2x2 average poolings; two 3x3 conv + ReLU per level; nearest upsampling and
 * concatenation with the encoder output on the way up; a 1x1 output.  Loss:
 * mean squared error on the n x n interior; optimiser: Adam (beta 0.9, 0.999,
 * eps 1e-8).  Parameters as one flat FP32 vector: per 3x3 convolution W
 * [cout][3][3][cin] then b [cout] in the order e0a e0b e1a e1b e2a e2b ba bb
 * d2a d2b d1a d1b d0a d0b, then the output layer w [c0], b [1].
 * Data layouts: inputs [samples][n+1][n+1][3] BF16 (bits as uint16), device;
 * targets and predictions [samples][n*n] dense like mgmc_sample's x (site
 * i + n j), device.  Calls are synchronous on the handle's stream.
 * ------------------------------------------------------------------------ */
typedef struct mgmc_unet* mgmc_unet_handle;

/* n = 2^k - 1 >= 31, c0 in {8, 16, 32} (c0 = 32: 1 946 881 parameters),
 * max_batch <= 64 samples per step; He-normal initial weights from seed. */
mgmc_status mgmc_unet_create(int n, int c0, int max_batch, uint64_t seed, const mgmc_allocator* alloc, void* stream,
                             mgmc_unet_handle* out);
mgmc_status mgmc_unet_n_params(mgmc_unet_handle u, int64_t* count);
mgmc_status mgmc_unet_get_params(mgmc_unet_handle u, float* host_out);
/* also resets the Adam moments and step count */
mgmc_status mgmc_unet_set_params(mgmc_unet_handle u, const float* host_in);
/* host helper: the input channels of one problem (same arguments as mgmc_create's
 * kappa^2 and observation rows) into out [n+1][n+1][3] BF16 (host) */
mgmc_status mgmc_unet_inputs(int n, const double* kappa2, double kappa2_const, int m, const int32_t* obs_site,
                             const double* obs_w, int nnz_per_obs, const double* y, uint16_t* out);
/* loss (mean squared error) of `batch` samples and its gradient (host, flat
 * like the parameters); either output may be NULL */
mgmc_status mgmc_unet_gradient(mgmc_unet_handle u, int batch, const void* inputs_bf16, const float* targets,
                               float* loss_out, float* grad_out);
/* `epochs` passes of Adam over n_samples (seeded shuffles, n_samples / batch
 * steps each); epoch_loss: NULL or host [epochs] mean training loss */
mgmc_status mgmc_unet_train(mgmc_unet_handle u, int64_t n_samples, const void* inputs_bf16, const float* targets,
                            int epochs, int batch, float lr, uint64_t shuffle_seed, float* epoch_loss);
/* the estimate of mu for n_samples problems into x_out [n_samples][n*n], FP32
 * or FP64 (precision = MGMC_FP32 / MGMC_FP64) */
mgmc_status mgmc_unet_predict(mgmc_unet_handle u, int64_t n_samples, const void* inputs_bf16, void* x_out,
                              int precision);
mgmc_status mgmc_unet_destroy(mgmc_unet_handle u);

/* ------------------------------------------------------------------------
 * Tensor-core GEMM (BF16 in, FP32 accumulate) on which the learned warm
 * start's convolutions run; exported for testing and reuse:
 *   C[M][N] = A[M][K] * B[N][K]^T  (+ bias[n]) (ReLU)
 * A: device BF16 row-major [M][lda], B: device BF16 row-major [N][ldb]
 * (lda, ldb >= K and multiples of 8; base addresses 16-byte aligned).
 * epilogue: bit 0 add bias (device float [N]), bit 1 ReLU, bit 2 store BF16
 * (else float).  splits > 1 (FP32 output only): the K range is cut into
 * `splits` parts summed in a fixed order (deterministic).  C: device [M][N].
 * Asynchronous on stream; MGMC_ERR_TIMEOUT is reported by the next call that
 * synchronises (a bounded wait inside the kernel gave up).
 * ------------------------------------------------------------------------ */
mgmc_status mgmc_tc_gemm(const void* A, int lda, const void* B, int ldb, void* C, int M, int N, int K, int splits,
                         int epilogue, const float* bias, void* stream);

/* Message of the last failing call on this thread; valid until the next call. */
const char* mgmc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
