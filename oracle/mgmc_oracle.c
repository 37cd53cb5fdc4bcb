/*
 * mgmc_oracle.c -- plain FP64 CPU reference of the Multigrid Monte Carlo
 * sampler (Kazashi, Mueller, Scheichl, "Multigrid Monte Carlo Revisited",
 * arXiv 2407.12149).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, by the smoke check and by the
 * benchmark's CPU baseline.  The product library never includes, links or
 * executes this file and shares no code with it.
 *
 * What it computes, step by step in the paper's order and notation:
 *
 *  Sec. 2.3 / Eq. (def-A_ell), (A_ell_1_B_ell_1):
 *    finest A_L = s (kappa^2 I - Delta_h) on the interior vertices of the
 *    unit square/cube (zero Dirichlet), s = h^d (bilinear-form scaling,
 *    Phi(l) = h^{d/2}) or s = 1 (literal reading); or its Q1 finite-element
 *    matrix; or (Sec. 5.1.1, Eq. squared_shifted_laplace) the 13-point
 *    finite-difference matrix of (kappa^2 - Delta)^2 with u = du/dn = 0 in
 *    2D (radius-2 stencils on every grid); A_{l-1} = P^T A_l P,
 *    B_{l-1} = P^T B_l with the canonical multilinear prolongation
 *    P = I_{l-1}^l (Eq. definition_prolongation), restriction = P^T unscaled.
 *  Eq. (f_ell_definition):  f_L = B Gamma^-1 y.
 *  Eq. (galerkin_triple_product): A~_l = A_l + B_l Gamma^-1 B_l^T.
 *  Alg. 3 + Eq. (lowrank_gibbs_two_steps), (Bellstar_definition):
 *    theta* = theta + (D + L)^-1 (f + xi - A theta),
 *    xi = D^{1/2} z + B xi_LR, xi_LR = L_Gamma^-T z',
 *    theta' = theta* - G (B^T theta*),  G = C (Gamma + B^T C)^-1,
 *    C = (D + L)^-1 B; backward direction swaps L <-> L^T.
 *    (Alg. 3's triangular solve is read as the increment form of
 *    Eq. lowrank_gibbs_two_steps.)
 *    Evaluation: every level's right-hand side is held as
 *    f_l = fd_l + B_l Gamma^-1 d_l (dense fd_l, data vector d_l; on the
 *    finest level fd_L = 0, d_L = y, Eq. f_ell_definition).  Splitting the
 *    sweep's right-hand side into its dense part s and B u,
 *    u = Gamma^-1 d + xi_LR, gives theta* = theta*_s + C u with theta*_s the
 *    Gauss-Seidel sweep of the dense part alone, and since
 *    C - G B^T C = G Gamma (from Eq. Bellstar_definition),
 *        theta' = theta*_s - G (B^T theta*_s - d - L_Gamma z').
 *    This is the same update; it avoids forming theta*, whose entries near
 *    an observation reach |Gamma^-1 y| w / a_ii and cancel in theta'.
 *  Alg. 1 with gamma = 1 (V-cycle) or gamma = 2 (W-cycle: the finest grid
 *    calls the next one once, every coarser grid calls its coarse grid
 *    twice, the coarse state carried from one call to the next),
 *    nu1 forward / nu2 backward sweeps,
 *    f_{l-1} = P^T (f_l - A~_l theta), coarse start psi = 0, theta += P psi.
 *    With the split: fd_{l-1} = P^T (fd_l - A_l theta) and
 *    d_{l-1} = d_l - B_l^T theta (because P^T B_l = B_{l-1}).
 *  Sec. 3.4 / Sec. 5.1.3: exact coarsest sampler
 *    theta_0 = A~_0^-1 f_0 + L_0^-T z  with A~_0 = L_0 L_0^T,
 *    f_0 = fd_0 + B_0 Gamma^-1 d_0.
 *  Eq. (MGMC_estimator), Sec. 5.3.2: QoI series F^T theta, lagged
 *    autocovariance with divisor n - t, IACT with Wolff's automatic window.
 *
 * Readings where the paper is silent (shared with the CUDA path by
 * definition only, not by code):
 *   - unknown order: 2^d parity colours, 2D order (0,0),(1,1),(0,1),(1,0);
 *     3D the four even colours (i+j+k even) in lexicographic order of
 *     (i mod 2, j mod 2, k mod 2) then the four odd ones; radius-2 stencils
 *     the nine classes (i mod 3, j mod 3) by code (i mod 3) + 3 (j mod 3);
 *     lexicographic within a colour.  Backward sweep = reverse colour order.
 *   - omega = 1.
 *   - random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed,
 *     counter (c0 = pair, c1 = cycle low 32 bits,
 *     c2 = (cycle bits 32..47) | chain << 16, c3 = kind << 24 | level << 16 | slot);
 *     kind 0 (site noise): one block per 4-site group of a grid row,
 *       c0 = (k n + j) nq + (i >> 2), nq = (n + 3) / 4; its four words give
 *       two Box-Muller pairs from 32-bit uniforms u = (w + 0.5) 2^-32:
 *       (w0, w1) for the sites with i even, (w2, w3) for i odd, member
 *       (i >> 1) & 1, z0 = r cos(2 pi u2), z1 = r sin(2 pi u2),
 *       r = sqrt(-2 ln u1); slot = 2 (v S + j) for the j-th pre sweep and
 *       2 (v S + j) + 1 for the j-th post sweep of the v-th visit of the
 *       level within the cycle, S = max(nu1, nu2, 1) (v = 0 in a V-cycle).
 *     kinds 1 and 2: one Box-Muller pair per block from 53-bit uniforms
 *       u = (k53 + 0.5) 2^-53 of the top 53 bits of (w0,w1) resp. (w2,w3);
 *       kind 1 (low-rank noise z'): c0 = k >> 1, member k & 1;
 *       kind 2 (coarsest sample): c0 = s >> 1, member s & 1, slot = the
 *       visit index v of the coarsest grid.
 *
 * Compile with -ffp-contract=off so that x86 and Arm builds round alike.
 */
#include "mgmc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ERR_ARG (-1)
#define ERR_NOT_SPD (-3)
#define ERR_OOM (-4)

typedef struct {
    int n;          /* interior points per axis */
    int N;          /* n^d */
    double* a;      /* [N * NS] full stencil */
    /* B_l stored column-wise: column k has entries b_ptr[k] .. b_ptr[k+1]-1 */
    int* b_ptr;
    int* b_site;
    double* b_w;
    /* G_l(dir) on its support: g_rows[dir] sites, g_val[dir][r * m + k] */
    int g_nrows[2];
    int* g_site[2];
    double* g_val[2];
    /* work vectors for the cycle: dense right-hand side fd, data vector d */
    double* f;
    double* dv;
    double* x;
    double* r;
    double* e;
} olevel;

struct oracle_problem {
    int d, NS, centre;
    int R, W;              /* stencil radius (1, or 2 for the squared operator) and width 2R+1 */
    int gamma;             /* recursive calls on the coarser grids below the finest (1 V, 2 W) */
    int visit[32];         /* visits of each level within the current cycle */
    int n_levels;
    int scale_hd;
    int disc;              /* fine-grid discretisation: 0 finite differences, 1 Q1 finite elements */
    int nu1, nu2;
    int m;                 /* beta: number of observations */
    olevel* lev;           /* lev[0] coarsest ... lev[n_levels-1] finest */
    double* Gamma;         /* m x m */
    double* Gamma_inv;     /* m x m */
    double* LG;            /* Cholesky factor of Gamma (lower) */
    double* LGinvT;        /* L_Gamma^-T, m x m */
    double* y;
    double* fL;            /* f_L = B Gamma^-1 y, dense */
    int n0;                /* unknowns on the coarsest level */
    double* A0;            /* dense A~_0 */
    double* L0;            /* its Cholesky factor (lower) */
    int n_qoi;
    int* q_site;
    double* q_w;
    /* counters of the current cycle */
    uint64_t seed;
    uint64_t cycle;
    uint32_t chain;
    int noise;
};

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller    */
/* ------------------------------------------------------------------ */

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

static double uniform53(uint32_t hi, uint32_t lo)
{
    uint64_t k = ((((uint64_t)hi) << 32) | (uint64_t)lo) >> 11;
    double u = (double)k + 0.5;
    return u * 0x1p-53;
}

void oracle_normal_pair(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                        double* z0, double* z1)
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    oracle_philox4x32_10(ctr, key, w);
    double u1 = uniform53(w[0], w[1]);
    double u2 = uniform53(w[2], w[3]);
    double r = sqrt(-2.0 * log(u1));
    double phi = 2.0 * M_PI * u2;
    *z0 = r * cos(phi);
    *z1 = r * sin(phi);
}

void oracle_normal_quad(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double z[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    oracle_philox4x32_10(ctr, key, w);
    for (int h = 0; h < 2; ++h) {
        double u1 = ((double)w[2 * h] + 0.5) * 0x1p-32;
        double u2 = ((double)w[2 * h + 1] + 0.5) * 0x1p-32;
        double r = sqrt(-2.0 * log(u1));
        double phi = 2.0 * M_PI * u2;
        z[2 * h] = r * cos(phi);
        z[2 * h + 1] = r * sin(phi);
    }
}

/* site noise (kind 0) of column i in block c0 of level `level` */
static double draw_site(const oracle_problem* p, int level, uint32_t slot, uint32_t block, int i)
{
    if (!p->noise) return 0.0;
    uint32_t c1 = (uint32_t)p->cycle;
    uint32_t c2 = ((uint32_t)(p->cycle >> 32) & 0xFFFFu) | (p->chain << 16);
    uint32_t c3 = ((uint32_t)level << 16) | slot;
    double z[4];
    oracle_normal_quad(p->seed, block, c1, c2, c3, z);
    return z[2 * (i & 1) + ((i >> 1) & 1)];
}

static double draw(const oracle_problem* p, uint32_t kind, int level, uint32_t slot,
                   uint32_t pair, int member)
{
    if (!p->noise) return 0.0;
    uint32_t c1 = (uint32_t)p->cycle;
    uint32_t c2 = ((uint32_t)(p->cycle >> 32) & 0xFFFFu) | (p->chain << 16);
    uint32_t c3 = (kind << 24) | ((uint32_t)level << 16) | slot;
    double z0, z1;
    oracle_normal_pair(p->seed, pair, c1, c2, c3, &z0, &z1);
    return member ? z1 : z0;
}

/* ------------------------------------------------------------------ */
/* small dense helpers                                                 */
/* ------------------------------------------------------------------ */

/* Cholesky A = L L^T of an SPD k x k matrix (row-major); L lower. */
static int cholesky(int k, const double* A, double* L)
{
    memset(L, 0, sizeof(double) * (size_t)k * k);
    for (int i = 0; i < k; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[i * k + j];
            for (int t = 0; t < j; ++t) s -= L[i * k + t] * L[j * k + t];
            if (i == j) {
                if (!(s > 0.0)) return ERR_NOT_SPD;
                L[i * k + i] = sqrt(s);
            } else {
                L[i * k + j] = s / L[j * k + j];
            }
        }
    }
    return 0;
}

/* Inverse of a general k x k matrix by Gauss-Jordan with partial pivoting. */
static int invert(int k, const double* A, double* Ainv)
{
    double* W = malloc(sizeof(double) * (size_t)k * 2 * k);
    if (!W) return ERR_OOM;
    for (int i = 0; i < k; ++i) {
        for (int j = 0; j < k; ++j) {
            W[i * 2 * k + j] = A[i * k + j];
            W[i * 2 * k + k + j] = (i == j) ? 1.0 : 0.0;
        }
    }
    for (int c = 0; c < k; ++c) {
        int piv = c;
        for (int i = c + 1; i < k; ++i)
            if (fabs(W[i * 2 * k + c]) > fabs(W[piv * 2 * k + c])) piv = i;
        if (W[piv * 2 * k + c] == 0.0) {
            free(W);
            return ERR_NOT_SPD;
        }
        if (piv != c) {
            for (int j = 0; j < 2 * k; ++j) {
                double t = W[c * 2 * k + j];
                W[c * 2 * k + j] = W[piv * 2 * k + j];
                W[piv * 2 * k + j] = t;
            }
        }
        double d = W[c * 2 * k + c];
        for (int j = 0; j < 2 * k; ++j) W[c * 2 * k + j] /= d;
        for (int i = 0; i < k; ++i) {
            if (i == c) continue;
            double fct = W[i * 2 * k + c];
            if (fct == 0.0) continue;
            for (int j = 0; j < 2 * k; ++j) W[i * 2 * k + j] -= fct * W[c * 2 * k + j];
        }
    }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) Ainv[i * k + j] = W[i * 2 * k + k + j];
    free(W);
    return 0;
}

/* ------------------------------------------------------------------ */
/* grid helpers                                                        */
/* ------------------------------------------------------------------ */

static void site_coords(int d, int n, int s, int c[3])
{
    c[0] = s % n;
    c[1] = (d >= 2) ? (s / n) % n : 0;
    c[2] = (d >= 3) ? s / (n * n) : 0;
}

static int site_index(int d, int n, const int c[3])
{
    for (int a = 0; a < d; ++a)
        if (c[a] < 0 || c[a] >= n) return -1;
    int s = c[0];
    if (d >= 2) s += n * c[1];
    if (d >= 3) s += n * n * c[2];
    return s;
}

static void offset_of(int d, int W, int o, int off[3])
{
    int R = W / 2;
    off[0] = o % W - R;
    off[1] = (d >= 2) ? (o / W) % W - R : 0;
    off[2] = (d >= 3) ? o / (W * W) - R : 0;
}

static int offset_index(const oracle_problem* p, int dx, int dy, int dz)
{
    return (dx + p->R) + p->W * (dy + p->R) + (p->d == 3 ? p->W * p->W * (dz + p->R) : 0);
}

/* Entry of the 1D canonical prolongation: fine interior index i, coarse j.
 * Coarse vertex j sits on fine vertex 2j+1; its hat function is 1/2 on the
 * two fine neighbours (Sec. 5.1.3: multilinear interpolation). */
static double p1d(int i, int j)
{
    if (i == 2 * j + 1) return 1.0;
    if (i == 2 * j || i == 2 * j + 2) return 0.5;
    return 0.0;
}

/* Colour sequence; returns the number of colours.  Radius-2 stencils (2D): the
 * nine classes (i mod 3, j mod 3) with code (i mod 3) + 3 (j mod 3) in increasing
 * code order -- sites of one class are at least 3 apart along an axis and so
 * never coupled by a 5 x 5 stencil. */
static int colour_sequence(const oracle_problem* p, int seq[27])
{
    int d = p->d;
    if (p->R == 2) {
        for (int c = 0; c < 9; ++c) seq[c] = c;
        return 9;
    }
    if (d == 2) {
        /* (0,0), (1,1), (0,1), (1,0) with code px + 2 py */
        seq[0] = 0; seq[1] = 3; seq[2] = 2; seq[3] = 1;
        return 4;
    }
    /* even: (0,0,0),(0,1,1),(1,0,1),(1,1,0); odd: (0,0,1),(0,1,0),(1,0,0),(1,1,1)
       with code px + 2 py + 4 pz */
    seq[0] = 0; seq[1] = 6; seq[2] = 5; seq[3] = 3;
    seq[4] = 4; seq[5] = 2; seq[6] = 1; seq[7] = 7;
    return 8;
}

static int parity_code(const oracle_problem* p, const int c[3])
{
    int d = p->d;
    if (p->R == 2) return c[0] % 3 + 3 * (c[1] % 3);
    int code = (c[0] & 1) + 2 * (c[1] & 1);
    if (d == 3) code += 4 * (c[2] & 1);
    return code;
}

/* y += A x for level l (plain definition sum_j a_ij x_j). */
static void apply_A(const oracle_problem* p, const olevel* L, const double* x, double* out)
{
    int d = p->d, n = L->n;
    for (int s = 0; s < L->N; ++s) {
        int c[3];
        site_coords(d, n, s, c);
        double acc = 0.0;
        for (int o = 0; o < p->NS; ++o) {
            double a = L->a[(size_t)s * p->NS + o];
            if (a == 0.0) continue;
            int off[3], nc[3];
            offset_of(d, p->W, o, off);
            for (int t = 0; t < 3; ++t) nc[t] = c[t] + off[t];
            int j = site_index(d, n, nc);
            if (j < 0) continue;
            acc += a * x[j];
        }
        out[s] = acc;
    }
}

/* B^T x (m entries). */
static void apply_Bt(const oracle_problem* p, const olevel* L, const double* x, double* z)
{
    for (int k = 0; k < p->m; ++k) {
        double acc = 0.0;
        for (int e = L->b_ptr[k]; e < L->b_ptr[k + 1]; ++e) acc += L->b_w[e] * x[L->b_site[e]];
        z[k] = acc;
    }
}

/* out = B v (dense N). */
static void apply_B(const oracle_problem* p, const olevel* L, const double* v, double* out)
{
    memset(out, 0, sizeof(double) * (size_t)L->N);
    for (int k = 0; k < p->m; ++k)
        for (int e = L->b_ptr[k]; e < L->b_ptr[k + 1]; ++e) out[L->b_site[e]] += L->b_w[e] * v[k];
}

/* out = A~ x = A x + B Gamma^-1 B^T x */
static void apply_Atilde(const oracle_problem* p, const olevel* L, const double* x, double* out)
{
    apply_A(p, L, x, out);
    if (p->m == 0) return;
    double* z = malloc(sizeof(double) * p->m * 2);
    double* w = z + p->m;
    apply_Bt(p, L, x, z);
    for (int k = 0; k < p->m; ++k) {
        double acc = 0.0;
        for (int l = 0; l < p->m; ++l) acc += p->Gamma_inv[k * p->m + l] * z[l];
        w[k] = acc;
    }
    for (int k = 0; k < p->m; ++k)
        for (int e = L->b_ptr[k]; e < L->b_ptr[k + 1]; ++e) out[L->b_site[e]] += L->b_w[e] * w[k];
    free(z);
}

/* ------------------------------------------------------------------ */
/* colour-ordered Gauss-Seidel sweep                                   */
/*   x_i <- (rhs_i + noise_i - sum_{j != i} a_ij x_j) / a_ii           */
/* over the colours in order (dir = 0) or reverse order (dir = 1).     */
/* rhs may include the dense low-rank noise B xi_LR (passed in e).     */
/* zdiag: optional explicit standard normals; otherwise Philox.        */
/* ------------------------------------------------------------------ */
static void gs_sweep(const oracle_problem* p, int l, const olevel* L, int dir, double* x,
                     const double* rhs, const double* e, const double* zdiag, uint32_t slot,
                     int use_noise)
{
    int d = p->d, n = L->n;
    int seq[27];
    int nc = colour_sequence(p, seq);
    int nq = (n + 3) / 4;
    for (int ci = 0; ci < nc; ++ci) {
        int colour = dir == 0 ? seq[ci] : seq[nc - 1 - ci];
        for (int s = 0; s < L->N; ++s) {
            int c[3];
            site_coords(d, n, s, c);
            if (parity_code(p, c) != colour) continue;
            const double* a = L->a + (size_t)s * p->NS;
            double aii = a[p->centre];
            double z = 0.0;
            if (use_noise) {
                if (zdiag) {
                    z = zdiag[s];
                } else {
                    uint32_t block = (uint32_t)(((int64_t)c[2] * n + c[1]) * nq + (c[0] >> 2));
                    z = draw_site(p, l, slot, block, c[0]);
                }
            }
            double acc = rhs ? rhs[s] : 0.0;
            acc += sqrt(aii) * z;
            if (e) acc += e[s];
            for (int o = 0; o < p->NS; ++o) {
                if (o == p->centre) continue;
                double aij = a[o];
                if (aij == 0.0) continue;
                int off[3], cc[3];
                offset_of(d, p->W, o, off);
                for (int t = 0; t < 3; ++t) cc[t] = c[t] + off[t];
                int j = site_index(d, n, cc);
                if (j < 0) continue;
                acc -= aij * x[j];
            }
            x[s] = acc / aii;
        }
    }
}

/* Gamma xi_LR = L_Gamma z' (z' standard normal), the low-rank noise of Sec. 3.4
 * in the units of the data vector. */
static void lowrank_noise(const oracle_problem* p, int l, uint32_t slot, const double* zgiven, double* gxi)
{
    int m = p->m;
    double* zp = malloc(sizeof(double) * (m > 0 ? m : 1));
    for (int k = 0; k < m; ++k)
        zp[k] = zgiven ? zgiven[k] : draw(p, 1u, l, slot, (uint32_t)(k >> 1), k & 1);
    for (int k = 0; k < m; ++k) {
        double acc = 0.0;
        for (int t = 0; t <= k; ++t) acc += p->LG[k * m + t] * zp[t];
        gxi[k] = acc;
    }
    free(zp);
}

/* Alg. 3: one Gibbs smoother step with low-rank correction on level l,
 * right-hand side fd + B Gamma^-1 d:
 *   theta*_s = Gauss-Seidel sweep of fd + D^{1/2} z,
 *   theta'   = theta*_s - G (B^T theta*_s - d - L_Gamma z'). */
static void lowrank_gibbs(const oracle_problem* p, int l, int dir, double* x, const double* fd, const double* d,
                          uint32_t slot, const double* zdiag, const double* zlr, int use_noise)
{
    olevel* L = &p->lev[l];
    int m = p->m;
    gs_sweep(p, l, L, dir, x, fd, NULL, zdiag, slot, use_noise);
    if (m == 0) return;
    double* v = malloc(sizeof(double) * m * 2);
    double* gxi = v + m;
    apply_Bt(p, L, x, v);
    if (use_noise) {
        lowrank_noise(p, l, slot, zlr, gxi);
        for (int k = 0; k < m; ++k) v[k] = v[k] - d[k] - gxi[k];
    } else {
        for (int k = 0; k < m; ++k) v[k] = v[k] - d[k];
    }
    for (int r = 0; r < L->g_nrows[dir]; ++r) {
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc += L->g_val[dir][(size_t)r * m + k] * v[k];
        x[L->g_site[dir][r]] -= acc;
    }
    free(v);
}

/* ------------------------------------------------------------------ */
/* setup                                                               */
/* ------------------------------------------------------------------ */

static void free_level(olevel* L)
{
    free(L->a);
    free(L->b_ptr);
    free(L->b_site);
    free(L->b_w);
    for (int dir = 0; dir < 2; ++dir) {
        free(L->g_site[dir]);
        free(L->g_val[dir]);
    }
    free(L->f);
    free(L->dv);
    free(L->x);
    free(L->r);
    free(L->e);
}

void oracle_destroy(oracle_problem* p)
{
    if (!p) return;
    if (p->lev)
        for (int l = 0; l < p->n_levels; ++l) free_level(&p->lev[l]);
    free(p->lev);
    free(p->Gamma);
    free(p->Gamma_inv);
    free(p->LG);
    free(p->LGinvT);
    free(p->y);
    free(p->fL);
    free(p->A0);
    free(p->L0);
    free(p->q_site);
    free(p->q_w);
    free(p);
}

static int alloc_level(oracle_problem* p, olevel* L, int n)
{
    L->n = n;
    L->N = n;
    for (int a = 1; a < p->d; ++a) L->N *= n;
    L->a = calloc((size_t)L->N * p->NS, sizeof(double));
    L->f = calloc((size_t)L->N, sizeof(double));
    L->dv = calloc((size_t)(p->m > 0 ? p->m : 1), sizeof(double));
    L->x = calloc((size_t)L->N, sizeof(double));
    L->r = calloc((size_t)L->N, sizeof(double));
    L->e = calloc((size_t)L->N, sizeof(double));
    L->b_ptr = calloc((size_t)p->m + 1, sizeof(int));
    if (!L->a || !L->f || !L->dv || !L->x || !L->r || !L->e || !L->b_ptr) return ERR_OOM;
    return 0;
}

/* Fine-level FD operator: s (kappa^2 I - Delta_h), s = h^d or 1. */
static void build_fine_operator(oracle_problem* p, olevel* L, const double* kappa2,
                                double kappa2_const)
{
    int d = p->d, n = L->n;
    double h = 1.0 / (double)(n + 1);
    double scale = 1.0;
    if (p->scale_hd)
        for (int a = 0; a < d; ++a) scale *= h;
    double inv_h2 = 1.0 / (h * h);
    for (int s = 0; s < L->N; ++s) {
        int c[3];
        site_coords(d, n, s, c);
        double k2 = kappa2 ? kappa2[s] : kappa2_const;
        double* a = L->a + (size_t)s * p->NS;
        a[p->centre] = scale * (k2 + 2.0 * d * inv_h2);
        for (int ax = 0; ax < d; ++ax) {
            for (int sg = -1; sg <= 1; sg += 2) {
                int cc[3] = {c[0], c[1], c[2]};
                cc[ax] += sg;
                if (site_index(d, n, cc) < 0) continue;
                int off[3] = {0, 0, 0};
                off[ax] = sg;
                int o = offset_index(p, off[0], off[1], off[2]);
                a[o] = -scale * inv_h2;
            }
        }
    }
}

/* Fine-level lowest-order conforming Q1 (multilinear) finite-element matrix of
 * kappa^2 I - Delta with zero Dirichlet values (Sec. 5.1.1, FE discretisation):
 * a_ij = int grad phi_i . grad phi_j + kappa^2 phi_i phi_j over the unit
 * square / cube for the nodal hat functions phi of the uniform grid, constant
 * kappa^2.  A hat function is a product of 1D hats, so each entry is a sum of
 * products of the 1D integrals
 *   stiffness  int phi_a' phi_b'  = (2 / h, -1 / h)  for |a - b| = (0, 1),
 *   mass       int phi_a  phi_b   = (4 h / 6, h / 6),
 * one derivative factor per axis: a(o) = sum_ax K(o_ax) prod_{t != ax} M(o_t)
 * + kappa^2 prod_t M(o_t).  scale_hd = 0 divides by h^d (the literal scaling
 * of the finite-difference option). */
static void build_fine_operator_q1(oracle_problem* p, olevel* L, double kappa2_const)
{
    int d = p->d, n = L->n;
    double h = 1.0 / (double)(n + 1);
    double scale = 1.0;
    if (!p->scale_hd)
        for (int a = 0; a < d; ++a) scale /= h;
    for (int s = 0; s < L->N; ++s) {
        int c[3];
        site_coords(d, n, s, c);
        double* a = L->a + (size_t)s * p->NS;
        for (int o = 0; o < p->NS; ++o) {
            int off[3], cc[3] = {0, 0, 0};
            offset_of(d, p->W, o, off);
            for (int t = 0; t < d; ++t) cc[t] = c[t] + off[t];
            if (site_index(d, n, cc) < 0) continue;
            double K[3], M[3];
            for (int t = 0; t < d; ++t) {
                K[t] = off[t] == 0 ? 2.0 / h : -1.0 / h;
                M[t] = off[t] == 0 ? 4.0 * h / 6.0 : h / 6.0;
            }
            double stiff = 0.0, mass = 1.0;
            for (int ax = 0; ax < d; ++ax) {
                double term = K[ax];
                for (int t = 0; t < d; ++t)
                    if (t != ax) term *= M[t];
                stiff += term;
                mass *= M[ax];
            }
            a[o] = scale * (stiff + kappa2_const * mass);
        }
    }
}

/* Fine-level finite-difference matrix of the squared shifted Laplacian
 * (kappa^2 - Delta)^2 = Delta^2 - 2 kappa^2 Delta + kappa^4 (Eq.
 * squared_shifted_laplace, Sec. 5.1.1, boundary conditions u = du/dn = 0), 2D,
 * constant kappa^2:
 *   Delta_h^2 -- the 13-point stencil h^-4 [20 at the centre, -8 at the four axis
 *     neighbours, 2 at the four diagonal neighbours, 1 at distance 2 along the
 *     axes]; a coupling that lands on a boundary vertex is dropped (u = 0 there),
 *     one that lands on the ghost vertex behind it takes the value of its mirror
 *     image across the boundary vertex (the centred difference of du/dn = 0);
 *   -2 kappa^2 Delta_h -- the 5-point stencil 2 kappa^2 h^-2 [4 at the centre, -1 at
 *     the axis neighbours] with u = 0 on the boundary;
 *   kappa^4 on the diagonal;
 * all times s = h^2 (scale_hd = 1) or 1. */
static void build_fine_operator_ssl(oracle_problem* p, olevel* L, double kappa2)
{
    int n = L->n;
    double h = 1.0 / (double)(n + 1);
    double scale = p->scale_hd ? h * h : 1.0;
    double ih2 = 1.0 / (h * h), ih4 = ih2 * ih2;
    static const int bih[13][3] = {{0, 0, 20},  {-1, 0, -8}, {1, 0, -8}, {0, -1, -8}, {0, 1, -8},
                                   {-1, -1, 2}, {1, -1, 2},  {-1, 1, 2}, {1, 1, 2},   {-2, 0, 1},
                                   {2, 0, 1},   {0, -2, 1},  {0, 2, 1}};
    for (int s = 0; s < L->N; ++s) {
        int c[3];
        site_coords(2, n, s, c);
        double* a = L->a + (size_t)s * p->NS;
        for (int t = 0; t < 13; ++t) {
            int g[2] = {c[0] + bih[t][0], c[1] + bih[t][1]};
            int drop = 0;
            for (int ax = 0; ax < 2; ++ax) {
                if (g[ax] == -1 || g[ax] == n)
                    drop = 1;               /* boundary vertex */
                else if (g[ax] == -2)
                    g[ax] = 0;              /* ghost behind x = 0: mirror image */
                else if (g[ax] == n + 1)
                    g[ax] = n - 1;          /* ghost behind x = 1: mirror image */
            }
            if (drop) continue;
            a[offset_index(p, g[0] - c[0], g[1] - c[1], 0)] += scale * (double)bih[t][2] * ih4;
        }
        a[p->centre] += scale * (2.0 * kappa2 * 4.0 * ih2 + kappa2 * kappa2);
        for (int t = 1; t <= 4; ++t) {
            int g0 = c[0] + bih[t][0], g1 = c[1] + bih[t][1];
            if (g0 < 0 || g0 >= n || g1 < 0 || g1 >= n) continue;
            a[offset_index(p, bih[t][0], bih[t][1], 0)] += -scale * 2.0 * kappa2 * ih2;
        }
    }
}

/* Galerkin triple product A_c = P^T A_f P (Eq. A_ell_1_B_ell_1). */
static void build_galerkin(oracle_problem* p, const olevel* F, olevel* C)
{
    int d = p->d;
    for (int J = 0; J < C->N; ++J) {
        int cj[3];
        site_coords(d, C->n, J, cj);
        double* ac = C->a + (size_t)J * p->NS;
        for (int po = 0; po < p->NS; ++po) {
            int pp[3];
            offset_of(d, p->W, po, pp);
            int ci[3] = {0, 0, 0};
            double wP = 1.0;
            for (int t = 0; t < d; ++t) {
                ci[t] = 2 * cj[t] + 1 + pp[t];
                wP *= p1d(ci[t], cj[t]);
            }
            int i = site_index(d, F->n, ci);
            if (i < 0 || wP == 0.0) continue;
            const double* af = F->a + (size_t)i * p->NS;
            for (int o = 0; o < p->NS; ++o) {
                double aij = af[o];
                if (aij == 0.0) continue;
                int off[3], cjf[3] = {0, 0, 0};
                offset_of(d, p->W, o, off);
                for (int t = 0; t < d; ++t) cjf[t] = ci[t] + off[t];
                if (site_index(d, F->n, cjf) < 0) continue;
                for (int q = 0; q < p->NS; ++q) {
                    int qq[3], ck[3] = {0, 0, 0};
                    offset_of(d, p->W, q, qq);
                    double w = 1.0;
                    for (int t = 0; t < d; ++t) {
                        ck[t] = cj[t] + qq[t];
                        w *= p1d(cjf[t], ck[t]);
                    }
                    if (w == 0.0 || site_index(d, C->n, ck) < 0) continue;
                    ac[q] += wP * aij * w;
                }
            }
        }
    }
}

/* B_c = P^T B_f (Eq. A_ell_1_B_ell_1), column by column. */
static int build_coarse_B(oracle_problem* p, const olevel* F, olevel* C)
{
    int d = p->d, m = p->m;
    double* col = calloc((size_t)C->N, sizeof(double));
    char* mark = calloc((size_t)C->N, 1);
    int cap = 64, nnz = 0;
    int* sites = malloc(sizeof(int) * cap);
    double* ws = malloc(sizeof(double) * cap);
    int tcap = 64;
    int* touched = malloc(sizeof(int) * tcap);
    if (!col || !mark || !sites || !ws || !touched) return ERR_OOM;
    for (int k = 0; k < m; ++k) {
        C->b_ptr[k] = nnz;
        int nt = 0;
        for (int e = F->b_ptr[k]; e < F->b_ptr[k + 1]; ++e) {
            int cf[3];
            site_coords(d, F->n, F->b_site[e], cf);
            for (int q = 0; q < p->NS; ++q) {
                int qq[3], ck[3] = {0, 0, 0};
                offset_of(d, p->W, q, qq);
                double w = 1.0;
                for (int t = 0; t < d; ++t) {
                    /* the coarse vertices whose hat function covers fine index cf */
                    ck[t] = (cf[t] >> 1) + qq[t];
                    w *= p1d(cf[t], ck[t]);
                }
                int K = site_index(d, C->n, ck);
                if (w == 0.0 || K < 0) continue;
                if (!mark[K]) {
                    mark[K] = 1;
                    if (nt == tcap) {
                        tcap *= 2;
                        touched = realloc(touched, sizeof(int) * tcap);
                    }
                    touched[nt++] = K;
                }
                col[K] += w * F->b_w[e];
            }
        }
        /* emit in increasing site order */
        for (int a = 0; a < nt; ++a)
            for (int b = a + 1; b < nt; ++b)
                if (touched[b] < touched[a]) {
                    int t = touched[a];
                    touched[a] = touched[b];
                    touched[b] = t;
                }
        for (int t = 0; t < nt; ++t) {
            int K = touched[t];
            if (col[K] != 0.0) {
                if (nnz == cap) {
                    cap *= 2;
                    sites = realloc(sites, sizeof(int) * cap);
                    ws = realloc(ws, sizeof(double) * cap);
                }
                sites[nnz] = K;
                ws[nnz] = col[K];
                ++nnz;
            }
            col[K] = 0.0;
            mark[K] = 0;
        }
    }
    C->b_ptr[m] = nnz;
    C->b_site = sites;
    C->b_w = ws;
    free(col);
    free(mark);
    free(touched);
    return 0;
}

/* Low-rank precompute for level l, direction dir (Alg. 3 lines 7-8):
 * C = M^-1 B column by column (a noise-free sweep from zero with rhs B_k),
 * S = Gamma + B^T C, G = C S^-1 stored on the union support of C. */
static int build_lowrank(oracle_problem* p, int l, int dir)
{
    olevel* L = &p->lev[l];
    int m = p->m, N = L->N;
    L->g_nrows[dir] = 0;
    if (m == 0) return 0;
    double* col = calloc((size_t)N, sizeof(double));
    int* rowof = malloc(sizeof(int) * (size_t)N);
    if (!col || !rowof) return ERR_OOM;
    for (int s = 0; s < N; ++s) rowof[s] = -1;
    /* pass 1: union support */
    int nrows = 0;
    int cap = 1024;
    int* sup = malloc(sizeof(int) * cap);
    for (int k = 0; k < m; ++k) {
        double* bk = L->r;
        memset(bk, 0, sizeof(double) * N);
        for (int e = L->b_ptr[k]; e < L->b_ptr[k + 1]; ++e) bk[L->b_site[e]] += L->b_w[e];
        memset(col, 0, sizeof(double) * N);
        gs_sweep(p, l, L, dir, col, bk, NULL, NULL, 0, 0);
        for (int s = 0; s < N; ++s) {
            if (col[s] != 0.0 && rowof[s] < 0) {
                if (nrows == cap) {
                    cap *= 2;
                    sup = realloc(sup, sizeof(int) * cap);
                }
                rowof[s] = nrows;
                sup[nrows++] = s;
            }
        }
    }
    /* sort support sites ascending and renumber */
    for (int s = 0, r = 0; s < N; ++s)
        if (rowof[s] >= 0) sup[r++] = s;
    for (int r = 0; r < nrows; ++r) rowof[sup[r]] = r;
    double* Cs = calloc((size_t)nrows * m + 1, sizeof(double));
    for (int k = 0; k < m; ++k) {
        double* bk = L->r;
        memset(bk, 0, sizeof(double) * N);
        for (int e = L->b_ptr[k]; e < L->b_ptr[k + 1]; ++e) bk[L->b_site[e]] += L->b_w[e];
        memset(col, 0, sizeof(double) * N);
        gs_sweep(p, l, L, dir, col, bk, NULL, NULL, 0, 0);
        for (int r = 0; r < nrows; ++r) Cs[(size_t)r * m + k] = col[sup[r]];
    }
    /* S = Gamma + B^T C */
    double* S = malloc(sizeof(double) * m * m);
    double* Sinv = malloc(sizeof(double) * m * m);
    for (int k = 0; k < m; ++k) {
        for (int j = 0; j < m; ++j) {
            double acc = p->Gamma[k * m + j];
            for (int e = L->b_ptr[k]; e < L->b_ptr[k + 1]; ++e) {
                int r = rowof[L->b_site[e]];
                if (r >= 0) acc += L->b_w[e] * Cs[(size_t)r * m + j];
            }
            S[k * m + j] = acc;
        }
    }
    int rc = invert(m, S, Sinv);
    if (rc) return rc;
    /* G = C S^-1 */
    double* G = calloc((size_t)nrows * m + 1, sizeof(double));
    for (int r = 0; r < nrows; ++r)
        for (int j = 0; j < m; ++j) {
            double acc = 0.0;
            for (int k = 0; k < m; ++k) acc += Cs[(size_t)r * m + k] * Sinv[k * m + j];
            G[(size_t)r * m + j] = acc;
        }
    L->g_nrows[dir] = nrows;
    L->g_site[dir] = realloc(sup, sizeof(int) * (nrows > 0 ? nrows : 1));
    L->g_val[dir] = G;
    free(Cs);
    free(S);
    free(Sinv);
    free(col);
    free(rowof);
    return 0;
}

int oracle_create(int dim, int n, int n_levels, int scale_hd, int disc, int nu1, int nu2,
                  const double* kappa2, double kappa2_const,
                  int m, const int32_t* obs_site, const double* obs_w, int nnz_per_obs,
                  const double* Gamma, const double* y,
                  int n_qoi, const int32_t* qoi_site, const double* qoi_w,
                  oracle_problem** out)
{
    if (!out || (dim != 2 && dim != 3) || n < 1 || n_levels < 1 || m < 0 || nu1 < 0 || nu2 < 0)
        return ERR_ARG;
    /* the Q1 and squared-operator options take a constant kappa^2; the squared
       operator is two-dimensional */
    if (disc != 0 && ((disc != 1 && disc != 2) || kappa2)) return ERR_ARG;
    if (disc == 2 && dim != 2) return ERR_ARG;
    if (n_levels > 32) return ERR_ARG;
    /* n_levels grids: n_{l-1} = (n_l - 1) / 2 must stay >= 1 and exact */
    {
        int nn = n;
        for (int l = 1; l < n_levels; ++l) {
            if (nn < 3 || (nn - 1) % 2 != 0) return ERR_ARG;
            nn = (nn - 1) / 2;
        }
    }
    if (m > 0 && (!obs_site || !obs_w || !Gamma || !y || nnz_per_obs < 1)) return ERR_ARG;
    oracle_problem* p = calloc(1, sizeof(oracle_problem));
    if (!p) return ERR_OOM;
    p->d = dim;
    p->R = disc == 2 ? 2 : 1;
    p->W = 2 * p->R + 1;
    p->NS = dim == 2 ? p->W * p->W : p->W * p->W * p->W;
    p->centre = (p->NS - 1) / 2;
    p->gamma = 1;
    p->n_levels = n_levels;
    p->scale_hd = scale_hd;
    p->disc = disc;
    p->nu1 = nu1;
    p->nu2 = nu2;
    p->m = m;
    p->lev = calloc((size_t)n_levels, sizeof(olevel));
    int mm = m > 0 ? m : 1;
    p->Gamma = calloc((size_t)mm * mm, sizeof(double));
    p->Gamma_inv = calloc((size_t)mm * mm, sizeof(double));
    p->LG = calloc((size_t)mm * mm, sizeof(double));
    p->LGinvT = calloc((size_t)mm * mm, sizeof(double));
    p->y = calloc((size_t)mm, sizeof(double));
    int rc = 0;
    if (m > 0) {
        memcpy(p->Gamma, Gamma, sizeof(double) * m * m);
        memcpy(p->y, y, sizeof(double) * m);
        rc = cholesky(m, p->Gamma, p->LG);
        if (rc) goto fail;
        rc = invert(m, p->Gamma, p->Gamma_inv);
        if (rc) goto fail;
        double* LGinv = malloc(sizeof(double) * m * m);
        rc = invert(m, p->LG, LGinv);
        if (rc) {
            free(LGinv);
            goto fail;
        }
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) p->LGinvT[i * m + j] = LGinv[j * m + i];
        free(LGinv);
    }
    /* levels */
    {
        int nn = n;
        for (int l = n_levels - 1; l >= 0; --l) {
            rc = alloc_level(p, &p->lev[l], nn);
            if (rc) goto fail;
            nn = (nn - 1) / 2;
        }
    }
    olevel* Lf = &p->lev[n_levels - 1];
    if (p->disc == 1)
        build_fine_operator_q1(p, Lf, kappa2_const);
    else if (p->disc == 2)
        build_fine_operator_ssl(p, Lf, kappa2_const);
    else
        build_fine_operator(p, Lf, kappa2, kappa2_const);
    /* fine B from the given rows (duplicates are summed) */
    {
        int nnz = 0;
        Lf->b_site = malloc(sizeof(int) * ((size_t)mm * nnz_per_obs + 1));
        Lf->b_w = malloc(sizeof(double) * ((size_t)mm * nnz_per_obs + 1));
        for (int k = 0; k < m; ++k) {
            Lf->b_ptr[k] = nnz;
            for (int t = 0; t < nnz_per_obs; ++t) {
                int s = obs_site[k * nnz_per_obs + t];
                double w = obs_w[k * nnz_per_obs + t];
                if (s < 0) continue;
                if (s >= Lf->N || !isfinite(w)) {
                    rc = ERR_ARG;
                    goto fail;
                }
                int found = -1;
                for (int e = Lf->b_ptr[k]; e < nnz; ++e)
                    if (Lf->b_site[e] == s) found = e;
                if (found >= 0) {
                    Lf->b_w[found] += w;
                } else {
                    Lf->b_site[nnz] = s;
                    Lf->b_w[nnz] = w;
                    ++nnz;
                }
            }
        }
        Lf->b_ptr[m] = nnz;
    }
    for (int l = n_levels - 1; l >= 1; --l) {
        build_galerkin(p, &p->lev[l], &p->lev[l - 1]);
        rc = build_coarse_B(p, &p->lev[l], &p->lev[l - 1]);
        if (rc) goto fail;
    }
    for (int l = 1; l < n_levels; ++l)
        for (int dir = 0; dir < 2; ++dir) {
            rc = build_lowrank(p, l, dir);
            if (rc) goto fail;
        }
    /* f_L = B Gamma^-1 y */
    p->fL = calloc((size_t)Lf->N, sizeof(double));
    if (m > 0) {
        double* w = malloc(sizeof(double) * m);
        for (int k = 0; k < m; ++k) {
            double acc = 0.0;
            for (int j = 0; j < m; ++j) acc += p->Gamma_inv[k * m + j] * p->y[j];
            w[k] = acc;
        }
        apply_B(p, Lf, w, p->fL);
        free(w);
    }
    /* coarsest dense A~_0 and its Cholesky factor */
    {
        olevel* L0 = &p->lev[0];
        int n0 = L0->N;
        p->n0 = n0;
        p->A0 = calloc((size_t)n0 * n0, sizeof(double));
        p->L0 = calloc((size_t)n0 * n0, sizeof(double));
        for (int s = 0; s < n0; ++s) {
            int c[3];
            site_coords(p->d, L0->n, s, c);
            for (int o = 0; o < p->NS; ++o) {
                int off[3], cc[3];
                offset_of(p->d, p->W, o, off);
                for (int t = 0; t < 3; ++t) cc[t] = c[t] + off[t];
                int j = site_index(p->d, L0->n, cc);
                if (j < 0) continue;
                p->A0[(size_t)s * n0 + j] += L0->a[(size_t)s * p->NS + o];
            }
        }
        double* Bd = calloc((size_t)n0 * mm, sizeof(double));
        for (int k = 0; k < m; ++k)
            for (int e = L0->b_ptr[k]; e < L0->b_ptr[k + 1]; ++e) Bd[(size_t)L0->b_site[e] * m + k] += L0->b_w[e];
        for (int i = 0; i < n0; ++i)
            for (int j = 0; j < n0; ++j) {
                double acc = 0.0;
                for (int k = 0; k < m; ++k)
                    for (int t = 0; t < m; ++t)
                        acc += Bd[(size_t)i * m + k] * p->Gamma_inv[k * m + t] * Bd[(size_t)j * m + t];
                p->A0[(size_t)i * n0 + j] += acc;
            }
        free(Bd);
        rc = cholesky(n0, p->A0, p->L0);
        if (rc) goto fail;
    }
    /* QoI */
    p->n_qoi = n_qoi;
    p->q_site = malloc(sizeof(int) * (n_qoi > 0 ? n_qoi : 1));
    p->q_w = malloc(sizeof(double) * (n_qoi > 0 ? n_qoi : 1));
    for (int t = 0; t < n_qoi; ++t) {
        if (qoi_site[t] < 0 || qoi_site[t] >= Lf->N) {
            rc = ERR_ARG;
            goto fail;
        }
        p->q_site[t] = qoi_site[t];
        p->q_w[t] = qoi_w[t];
    }
    *out = p;
    return 0;
fail:
    oracle_destroy(p);
    return rc;
}

/* ------------------------------------------------------------------ */
/* coarsest exact sampler and the V-cycle (Alg. 1)                     */
/* ------------------------------------------------------------------ */

static void coarsest_sample(oracle_problem* p, double* x, const double* fd, const double* d, uint32_t slot)
{
    int n0 = p->n0, m = p->m;
    olevel* L0 = &p->lev[0];
    double* yv = malloc(sizeof(double) * n0);
    double* f0 = malloc(sizeof(double) * n0);
    /* f_0 = fd_0 + B_0 Gamma^-1 d_0 */
    memcpy(f0, fd, sizeof(double) * n0);
    for (int k = 0; k < m; ++k) {
        double gk = 0.0;
        for (int t = 0; t < m; ++t) gk += p->Gamma_inv[k * m + t] * d[t];
        for (int e = L0->b_ptr[k]; e < L0->b_ptr[k + 1]; ++e) f0[L0->b_site[e]] += L0->b_w[e] * gk;
    }
    /* L y = f */
    for (int i = 0; i < n0; ++i) {
        double acc = f0[i];
        for (int t = 0; t < i; ++t) acc -= p->L0[(size_t)i * n0 + t] * yv[t];
        yv[i] = acc / p->L0[(size_t)i * n0 + i];
    }
    /* y += z */
    for (int i = 0; i < n0; ++i) yv[i] += draw(p, 2u, 0, slot, (uint32_t)(i >> 1), i & 1);
    /* L^T x = y */
    for (int i = n0 - 1; i >= 0; --i) {
        double acc = yv[i];
        for (int t = i + 1; t < n0; ++t) acc -= p->L0[(size_t)t * n0 + i] * x[t];
        x[i] = acc / p->L0[(size_t)i * n0 + i];
    }
    free(yv);
    free(f0);
}

static void restrict_to(const oracle_problem* p, const olevel* F, const olevel* C,
                        const double* r, double* fc)
{
    int d = p->d;
    for (int J = 0; J < C->N; ++J) {
        int cj[3];
        site_coords(d, C->n, J, cj);
        double acc = 0.0;
        for (int po = 0; po < p->NS; ++po) {
            int pp[3], ci[3] = {0, 0, 0};
            offset_of(d, p->W, po, pp);
            double w = 1.0;
            for (int t = 0; t < d; ++t) {
                ci[t] = 2 * cj[t] + 1 + pp[t];
                w *= p1d(ci[t], cj[t]);
            }
            int i = site_index(d, F->n, ci);
            if (i < 0) continue;
            acc += w * r[i];
        }
        fc[J] = acc;
    }
}

static void prolong_add(const oracle_problem* p, const olevel* C, const olevel* F,
                        const double* psi, double* x)
{
    int d = p->d;
    for (int i = 0; i < F->N; ++i) {
        int cf[3];
        site_coords(d, F->n, i, cf);
        double acc = 0.0;
        for (int q = 0; q < p->NS; ++q) {
            int qq[3], ck[3] = {0, 0, 0};
            offset_of(d, p->W, q, qq);
            double w = 1.0;
            for (int t = 0; t < d; ++t) {
                ck[t] = (cf[t] >> 1) + qq[t];
                w *= p1d(cf[t], ck[t]);
            }
            int K = site_index(d, C->n, ck);
            if (w == 0.0 || K < 0) continue;
            acc += w * psi[K];
        }
        x[i] += acc;
    }
}

/* Alg. 1 on level l.  The v-th visit of level l within a cycle (v = 0, 1, ...
 * in call order) draws with slots 2 (v S + j) for its j-th pre sweep and
 * 2 (v S + j) + 1 for its j-th post sweep, S = max(nu1, nu2, 1), and the coarsest
 * level's v-th visit with slot v; a V-cycle has v = 0 throughout.  The finest
 * level makes one coarse call, every other level gamma (Alg. 1: gamma_L = 1,
 * gamma_l = gamma below). */
static void mgmc_level(oracle_problem* p, int l, double* x, const double* fd, const double* d)
{
    const int v = p->visit[l]++;
    if (l == 0) {
        coarsest_sample(p, x, fd, d, (uint32_t)v);
        return;
    }
    olevel* L = &p->lev[l];
    olevel* C = &p->lev[l - 1];
    int S = p->nu1 > p->nu2 ? p->nu1 : p->nu2;
    if (S < 1) S = 1;
    for (int j = 0; j < p->nu1; ++j)
        lowrank_gibbs(p, l, 0, x, fd, d, (uint32_t)(2 * (v * S + j)), NULL, NULL, p->noise);
    /* f_{l-1} = P^T (f_l - A~_l theta):  fd_{l-1} = P^T (fd_l - A_l theta),
       d_{l-1} = d_l - B_l^T theta */
    apply_A(p, L, x, L->r);
    for (int s = 0; s < L->N; ++s) L->r[s] = fd[s] - L->r[s];
    restrict_to(p, L, C, L->r, C->f);
    if (p->m > 0) {
        apply_Bt(p, L, x, C->dv);
        for (int k = 0; k < p->m; ++k) C->dv[k] = d[k] - C->dv[k];
    }
    memset(C->x, 0, sizeof(double) * C->N);
    const int calls = l == p->n_levels - 1 ? 1 : p->gamma;
    for (int g = 0; g < calls; ++g) mgmc_level(p, l - 1, C->x, C->f, C->dv);
    prolong_add(p, C, L, C->x, x);
    for (int j = 0; j < p->nu2; ++j)
        lowrank_gibbs(p, l, 1, x, fd, d, (uint32_t)(2 * (v * S + j) + 1), NULL, NULL, p->noise);
}

static double qoi_of(const oracle_problem* p, const double* x)
{
    double acc = 0.0;
    for (int t = 0; t < p->n_qoi; ++t) acc += p->q_w[t] * x[p->q_site[t]];
    return acc;
}

int oracle_sample(oracle_problem* p, int64_t n_steps, uint64_t seed, uint64_t step_offset,
                  uint32_t chain, int noise, double* x, double* qoi_out)
{
    if (!p || !x || n_steps < 0) return ERR_ARG;
    p->seed = seed;
    p->chain = chain;
    p->noise = noise ? 1 : 0;
    for (int64_t s = 0; s < n_steps; ++s) {
        p->cycle = step_offset + (uint64_t)s;
        olevel* Lf = &p->lev[p->n_levels - 1];
        memset(Lf->f, 0, sizeof(double) * Lf->N);      /* fd_L = 0 */
        if (p->m > 0) memcpy(Lf->dv, p->y, sizeof(double) * p->m);   /* d_L = y */
        memset(p->visit, 0, sizeof(p->visit));
        mgmc_level(p, p->n_levels - 1, x, Lf->f, Lf->dv);
        if (qoi_out) qoi_out[s] = qoi_of(p, x);
    }
    return 0;
}

/* Sec. 5.1.3, "Gibbs sampler": the symmetric low-rank Gibbs sweeps of the finest
 * level alone (Alg. 3 forward nu1 times, then backward nu2 times). */
int oracle_sample_gibbs(oracle_problem* p, int64_t n_steps, uint64_t seed, uint64_t step_offset,
                        uint32_t chain, int noise, double* x, double* qoi_out)
{
    if (!p || !x || n_steps < 0 || p->n_levels < 2) return ERR_ARG;
    p->seed = seed;
    p->chain = chain;
    p->noise = noise ? 1 : 0;
    const int l = p->n_levels - 1;
    olevel* Lf = &p->lev[l];
    for (int64_t s = 0; s < n_steps; ++s) {
        p->cycle = step_offset + (uint64_t)s;
        memset(Lf->f, 0, sizeof(double) * Lf->N);      /* fd_L = 0 */
        if (p->m > 0) memcpy(Lf->dv, p->y, sizeof(double) * p->m);   /* d_L = y */
        for (int j = 0; j < p->nu1; ++j)
            lowrank_gibbs(p, l, 0, x, Lf->f, Lf->dv, (uint32_t)(2 * j), NULL, NULL, p->noise);
        for (int j = 0; j < p->nu2; ++j)
            lowrank_gibbs(p, l, 1, x, Lf->f, Lf->dv, (uint32_t)(2 * j + 1), NULL, NULL, p->noise);
        if (qoi_out) qoi_out[s] = qoi_of(p, x);
    }
    return 0;
}

double oracle_rel_residual(const oracle_problem* p, const double* x)
{
    const olevel* L = &p->lev[p->n_levels - 1];
    double* r = malloc(sizeof(double) * L->N);
    apply_Atilde(p, L, x, r);
    double num = 0.0, den = 0.0;
    for (int s = 0; s < L->N; ++s) {
        double t = p->fL[s] - r[s];
        num += t * t;
        den += p->fL[s] * p->fL[s];
    }
    free(r);
    if (den == 0.0) return num == 0.0 ? 0.0 : INFINITY;
    return sqrt(num / den);
}

int oracle_mean_solve(oracle_problem* p, double rtol, int max_cycles, double* x,
                      int* cycles_done, double* rel_residual)
{
    if (!p || !x || max_cycles < 0) return ERR_ARG;
    int c = 0;
    double rr = oracle_rel_residual(p, x);
    while (rr > rtol && c < max_cycles) {
        oracle_sample(p, 1, 0, (uint64_t)c, 0, 0, x, NULL);
        ++c;
        rr = oracle_rel_residual(p, x);
    }
    if (cycles_done) *cycles_done = c;
    if (rel_residual) *rel_residual = rr;
    return 0;
}

int oracle_fine_rhs(const oracle_problem* p, double* out)
{
    memcpy(out, p->fL, sizeof(double) * p->lev[p->n_levels - 1].N);
    return 0;
}

/* ------------------------------------------------------------------ */
/* queries                                                             */
/* ------------------------------------------------------------------ */

int oracle_level_n(const oracle_problem* p, int l)
{
    if (!p || l < 0 || l >= p->n_levels) return ERR_ARG;
    return p->lev[l].n;
}

int oracle_set_gamma(oracle_problem* p, int gamma)
{
    if (!p || gamma < 1 || gamma > 2) return ERR_ARG;
    /* the slots of the last visit of the coarsest level must fit 16 bits */
    double visits = 1.0;
    for (int l = p->n_levels - 2; l >= 1; --l) visits *= gamma;
    int S = p->nu1 > p->nu2 ? p->nu1 : p->nu2;
    if (S < 1) S = 1;
    if (2.0 * visits * S > 65536.0) return ERR_ARG;
    p->gamma = gamma;
    return 0;
}

int oracle_level_stencil(const oracle_problem* p, int l, double* out)
{
    if (!p || l < 0 || l >= p->n_levels) return ERR_ARG;
    memcpy(out, p->lev[l].a, sizeof(double) * (size_t)p->lev[l].N * p->NS);
    return 0;
}

int oracle_level_B_dense(const oracle_problem* p, int l, double* out)
{
    if (!p || l < 0 || l >= p->n_levels) return ERR_ARG;
    const olevel* L = &p->lev[l];
    memset(out, 0, sizeof(double) * (size_t)L->N * (p->m > 0 ? p->m : 1));
    for (int k = 0; k < p->m; ++k)
        for (int e = L->b_ptr[k]; e < L->b_ptr[k + 1]; ++e) out[(size_t)L->b_site[e] * p->m + k] += L->b_w[e];
    return 0;
}

int oracle_level_G_dense(const oracle_problem* p, int l, int dir, double* out)
{
    if (!p || l < 1 || l >= p->n_levels || dir < 0 || dir > 1) return ERR_ARG;
    const olevel* L = &p->lev[l];
    int m = p->m;
    memset(out, 0, sizeof(double) * (size_t)L->N * (m > 0 ? m : 1));
    for (int r = 0; r < L->g_nrows[dir]; ++r)
        for (int k = 0; k < m; ++k) out[(size_t)L->g_site[dir][r] * m + k] = L->g_val[dir][(size_t)r * m + k];
    return 0;
}

int oracle_level_G_support(const oracle_problem* p, int l, int dir)
{
    if (!p || l < 1 || l >= p->n_levels || dir < 0 || dir > 1) return ERR_ARG;
    return p->lev[l].g_nrows[dir];
}

int oracle_coarsest_dense(const oracle_problem* p, double* out)
{
    if (!p) return ERR_ARG;
    memcpy(out, p->A0, sizeof(double) * (size_t)p->n0 * p->n0);
    return 0;
}

int oracle_smoother_step_given(const oracle_problem* p, int l, int dir, double* x, const double* fd,
                               const double* d, const double* zdiag, const double* zlr)
{
    if (!p || l < 1 || l >= p->n_levels || !x || !fd || !zdiag || (p->m > 0 && (!zlr || !d))) return ERR_ARG;
    lowrank_gibbs(p, l, dir, x, fd, d, 0u, zdiag, zlr, 1);
    return 0;
}

/* ------------------------------------------------------------------ */
/* chain statistics (Sec. 5.3.2; Wolff, Comput. Phys. Commun. 156     */
/* (2004) 143, Sec. 3.3 automatic windowing)                           */
/* ------------------------------------------------------------------ */
int oracle_chain_stats(const double* a, int64_t n, double S, double* mean, double* var,
                       double* tau, double* tau_err, int64_t* window)
{
    if (!a || n < 2) return ERR_ARG;
    double abar = 0.0;
    for (int64_t i = 0; i < n; ++i) abar += a[i];
    abar /= (double)n;
    /* Gamma(t) = 1/(n - t) sum_i (a_i - abar)(a_{i+t} - abar), evaluated for t = 0, 1, ...
       only as far as the window search needs it */
    int64_t tmax = n / 2;
    double G0 = 0.0;
    for (int64_t i = 0; i < n; ++i) G0 += (a[i] - abar) * (a[i] - abar);
    G0 /= (double)n;
    if (mean) *mean = abar;
    if (var) *var = G0;
    if (G0 <= 0.0) {
        if (tau) *tau = 1.0;
        if (tau_err) *tau_err = 0.0;
        if (window) *window = 0;
        return 0;
    }
    double tint = 0.5;
    int64_t W = tmax;
    for (int64_t w = 1; w <= tmax; ++w) {
        double acc = 0.0;
        for (int64_t i = 0; i + w < n; ++i) acc += (a[i] - abar) * (a[i + w] - abar);
        tint += acc / (double)(n - w) / G0;
        double ttilde;
        if (tint <= 0.5)
            ttilde = 1e-6;
        else
            ttilde = S / log((2.0 * tint + 1.0) / (2.0 * tint - 1.0));
        double g = exp(-(double)w / ttilde) - ttilde / sqrt((double)w * (double)n);
        if (g < 0.0) {
            W = w;
            break;
        }
    }
    /* error of tau_int (Wolff 2004, Eq. 42) */
    double err = 2.0 * tint * sqrt(((double)W + 0.5 - tint) / (double)n);
    if (tau) *tau = 2.0 * tint;
    if (tau_err) *tau_err = 2.0 * err;
    if (window) *window = W;
    return 0;
}
