/*
 * mgmc_oracle.h -- plain, slow, FP64 CPU reference of the Multigrid Monte
 * Carlo (MGMC) sampler of Kazashi, Mueller & Scheichl (arXiv 2407.12149).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads
 * or calls this code; only the test-suite, the smoke check and the
 * benchmark's CPU-baseline / reference arm do.  It shares no source with
 * the CUDA path.
 *
 * Conventions (all of them also stated in the header of mgmc_oracle.c):
 *   - levels are numbered as in the paper: 0 = coarsest, L = finest;
 *   - a level with n interior points per axis stores n^d values in
 *     lexicographic order (x fastest);
 *   - every function returns 0 on success and a negative code on error.
 */
#ifndef MGMC_ORACLE_H
#define MGMC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct oracle_problem oracle_problem;

/* Build the hierarchy, Galerkin operators, low-rank precompute and the
 * coarsest Cholesky factor.  kappa2 may be NULL (then kappa2_const is used).
 * obs_site/obs_w hold m rows of nnz_per_obs (fine site, weight); site -1 is
 * an ignored (boundary) entry.  Gamma is m x m row-major SPD, y has m
 * entries.  qoi_site/qoi_w: n_qoi entries of the QoI vector F_L.
 * disc: fine-grid discretisation, 0 the finite-difference stencil of
 * kappa^2 - Delta, 1 its Q1 finite-element matrix (constant kappa^2: kappa2 =
 * NULL), 2 the 13-point finite-difference matrix of the squared operator
 * (kappa^2 - Delta)^2 with u = du/dn = 0 (2D, constant kappa^2; radius-2
 * stencils on every level). */
int oracle_create(int dim, int n, int n_levels, int scale_hd, int disc, int nu1, int nu2,
                  const double* kappa2, double kappa2_const,
                  int m, const int32_t* obs_site, const double* obs_w, int nnz_per_obs,
                  const double* Gamma, const double* y,
                  int n_qoi, const int32_t* qoi_site, const double* qoi_w,
                  oracle_problem** out);
void oracle_destroy(oracle_problem* p);

/* Cycle index of Alg. 1: gamma = 1 (V-cycle, the default) or 2 (W-cycle: the
 * finest level calls the next grid once, every coarser level calls its coarse
 * grid twice). */
int oracle_set_gamma(oracle_problem* p, int gamma);

/* Level queries (l = 0 coarsest .. n_levels-1 finest). */
int oracle_level_n(const oracle_problem* p, int l);
/* Full W^d stencil of level l, W = 2R + 1 (R = 2 for disc 2, else 1):
 * out[N * W^d], offset index (3D form; 2D drops the dz term)
 * (dx+R) + W (dy+R) + W^2 (dz+R); out-of-domain couplings are 0. */
int oracle_level_stencil(const oracle_problem* p, int l, double* out);
/* Dense B_l (N x m, row-major). */
int oracle_level_B_dense(const oracle_problem* p, int l, double* out);
/* Low-rank matrix G_l of Eq. (Bellstar_definition) for direction dir
 * (0 forward, 1 backward) written densely: out[N x m] row-major. */
int oracle_level_G_dense(const oracle_problem* p, int l, int dir, double* out);
/* Number of rows in the support of G_l(dir). */
int oracle_level_G_support(const oracle_problem* p, int l, int dir);
/* Dense coarsest operator A~_0 = A_0 + B_0 Gamma^-1 B_0^T (n0 x n0). */
int oracle_coarsest_dense(const oracle_problem* p, double* out);

/* One Alg. 3 step (Gibbs smoother with low-rank correction) on level l
 * for the right-hand side f = fd + B_l Gamma^-1 d, with the random numbers
 * supplied: zdiag[N] standard normals for xi_diag = D^{1/2} zdiag and zlr[m]
 * standard normals for xi_LR = L_Gamma^{-T} zlr.  x (in/out) and fd are
 * dense level vectors, d has m entries. */
int oracle_smoother_step_given(const oracle_problem* p, int l, int dir,
                               double* x, const double* fd, const double* d,
                               const double* zdiag, const double* zlr);

/* Run n_steps MGMC cycles (Alg. 1 with the cycle index of oracle_set_gamma) on
 * the finest level.
 * x (in/out) is the dense fine state.  Cycle m uses the Philox counters of
 * cycle index step_offset + m.  noise = 0 gives the deterministic
 * multigrid iteration.  qoi_out (may be NULL) receives F_L^T x after each
 * cycle. */
int oracle_sample(oracle_problem* p, int64_t n_steps, uint64_t seed, uint64_t step_offset,
                  uint32_t chain, int noise, double* x, double* qoi_out);

/* The plain Gibbs sampler the paper compares MGMC with (Sec. 5.1.3, "Gibbs
 * sampler"): each step is nu1 forward then nu2 backward sweeps of the
 * low-rank Gibbs smoother (Alg. 3) on the finest level, with the right-hand
 * side f_L = B Gamma^-1 y held as fd = 0, d = y, and the noise slots of the
 * MGMC cycle's finest level (2 j forward, 2 j + 1 backward).  Needs
 * n_levels >= 2.  Arguments as oracle_sample. */
int oracle_sample_gibbs(oracle_problem* p, int64_t n_steps, uint64_t seed, uint64_t step_offset,
                        uint32_t chain, int noise, double* x, double* qoi_out);

/* Noise-free V-cycles from the given x until ||f - A~ x|| <= rtol ||f||. */
int oracle_mean_solve(oracle_problem* p, double rtol, int max_cycles, double* x,
                      int* cycles_done, double* rel_residual);

/* Fine-level right-hand side f_L = B Gamma^-1 y (dense, N entries). */
int oracle_fine_rhs(const oracle_problem* p, double* out);
/* Residual norm ratio ||f_L - A~_L x|| / ||f_L||. */
double oracle_rel_residual(const oracle_problem* p, const double* x);

/* Philox4x32-10 block and the Box-Muller pair used everywhere. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void oracle_normal_pair(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                        double* z0, double* z1);
/* The four standard normals of one site-noise block (kind 0): two Box-Muller
 * pairs from 32-bit uniforms u = (w + 0.5) 2^-32 of the Philox words
 * (w0, w1) -> z[0], z[1] and (w2, w3) -> z[2], z[3]. */
void oracle_normal_quad(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double z[4]);

/* Chain statistics: sample mean/variance, lagged autocovariance and the
 * integrated autocorrelation time with Wolff's automatic window (S given).
 * tau and tau_err are in the paper's convention (tau = 1 + 2 sum rho). */
int oracle_chain_stats(const double* series, int64_t n, double S,
                       double* mean, double* var, double* tau, double* tau_err,
                       int64_t* window);

#ifdef __cplusplus
}
#endif
#endif
