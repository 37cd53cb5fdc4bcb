// common.cuh -- device-side data layout and helpers of the MGMC sampler.
//
// Grid storage (every level, every field): a padded array with one ring of
// zero ghost values.  Interior site (i, j[, k]) lives at element
//   base + i + pitch * j [+ plane * k],
//   base = 4 + pitch [+ plane],
// so each row starts at a 16-byte boundary (4 FP32 / 2 FP64 sites), the
// left ghost sits at column 3 and the right ghost at column n + 4.  The
// ghosts are never written and stay zero (zero Dirichlet values, Sec. 5.1.1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/mgmc.h"

namespace mgmc {

constexpr int kMaxObs = MGMC_MAX_OBS;

// sets the message returned by mgmc_last_error() on this thread
void set_last_error(const char* msg);

// Per-cycle values read by the kernels of a captured cycle graph.
struct CycleState {
    unsigned long long seed;
    unsigned long long cycle;   // Philox cycle index of the running V-cycle
    unsigned int chain;
    int noise;                  // 0: deterministic multigrid (mean solve)
    double* qoi;                // NULL or [n_steps] QoI series
    long long step;             // index into qoi of the running cycle
    int status;                 // sticky error bits, kept until the host reports them:
                                // 1 a non-finite QoI, 2 a bounded wait gave up
    long long wait_ns;          // bound of the kernels' staging waits: 0 the default
                                // (1 s), > 0 that many ns, < 0 give up at once (tests)
};

constexpr int kStatusNumeric = 1;
constexpr int kStatusTimeout = 2;
constexpr int kStatusLayout = 4;   // a kernel's shared-memory layout exceeded its launch (not run)

// One grid level on the device.  T = float or double.
template <typename T>
struct DevLevel {
    int level;          // paper numbering: 0 coarsest
    int dim;
    int n;              // interior points per axis
    int pitch;          // elements per padded row
    long long plane;    // elements per padded plane
    long long base;     // element offset of interior site 0
    long long alloc;    // elements per padded field
    T* x;               // state theta_l / psi_l
    T* f;               // dense part of the right-hand side (NULL on the finest level)
    // finest level: 5/7-point operator s (kappa^2 - Delta_h)
    int fine;
    T* diag;            // FP64: a_ii ; FP32: s kappa^2_i (the row-sum part)
    T woff;             // s / h^2 (off-diagonal magnitude)
    // coarse levels: symmetric 9/27-point Galerkin stencil, structure of arrays;
    // slot 0 = a_ii (FP64) or the row sum sum_j a_ij (FP32), slot t >= 1 = a(i, i + o_t)
    // for the t-th positive stencil offset o_t
    T* coef;
    int ncoef;
    // stencil radius of the coefficient form: 1 (9/27-point) or 2 (2D 25-point grids of
    // the squared shifted Laplacian: offsets o = (dx+2) + 5 (dy+2), centre 12, slot t >= 1
    // = a(i, i + o_{12+t}); two halo rows and columns around the interior)
    int rad;
    // FP64 25-point grids: 1 / a_ii at [e] and sqrt(a_ii) at [alloc + e] (correctly rounded on
    // the host), so that a site update needs neither a division nor a square root
    const double* inv_sqrt25;
    // B_l rows grouped by grid row (finest level; used by the residual norm)
    const int* brow_ptr;    // [n^(dim-1) + 1]
    const int* bent_i;      // x index of the entry
    const int* bent_k;      // observation index
    const double* bent_w;   // weight
    // B_l columns (for z = B^T x)
    const int* bcol_ptr;          // [m + 1]
    const long long* bcol_site;   // padded element offset
    const double* bcol_w;
    const int* bcol_ss;           // grids inside the coarse kernel: shared-memory index of the site
    const int* bcol_dense;        // coarsest grid: dense site index
    const int* g_ss[2];           // grids inside the coarse kernel: shared-memory index of G's sites
    // G_l on its support, per direction (0 forward, 1 backward)
    int g_rows[2];
    const long long* g_site[2];   // padded element offsets
    const double* g_val[2];       // [rows * m]
    // the level's right-hand side is f_l = fdense_l + B_l Gamma^-1 d_l
    double* d;                    // [m] data vector d_l (d_L = y)
    double* dnext;                // [m] d_{l-1} = d_l - B_l^T theta, written on the way down
    // fused 2D tile path (see tile2d.cu)
    T* x2;                        // second state buffer: theta*_s after the forward sweep
    int ntx;                      // tiles per row
    const int* tile_ptr;          // [ntiles + 1]: B entries inside each tile
    const int* tile_loc;          // local site of the entry, lx | ly << 16, relative to the tile origin
    const int* tile_ent;          // index t of the entry in the column lists bcol_*
    double* zparts;               // [nnz] w_t * theta(site_t), written by the tile kernels
    const T* gT[2];               // G_l(dir) in the path precision, [rows * m]
    int h_rows;                   // H = P^T A_l G_l(forward) on the coarse grid
    const long long* h_site;      // coarse padded offsets
    const T* hT;                  // [rows * m]
    const double* BtG;            // B_l^T G_l(forward), [m * m]
    // general (unfused) path
    double* lrv;                  // [2m] v, then z = B^T theta*_s, of the level's last low-rank step
    T* res;                       // residual f_l - A_l theta on the padded layout (restriction input)
};

// Tile shape of the fused 2D kernels: TX x TY interior sites per CTA.
template <typename T, bool FINE>
struct TileShape {
    static constexpr int TX = FINE ? 64 : 32;
    static constexpr int TY = sizeof(T) == 4 ? 32 : 16;
};

struct DevProblem {
    int m;                     // number of observations
    int gamma_diag;            // Gamma (and its Cholesky factor) is diagonal
    const double* Gamma_inv;   // [m*m]
    const double* LG;          // [m*m] Cholesky factor L_Gamma of Gamma (lower triangular)
    CycleState* cs;
};

__host__ __device__ inline long long site_offset(int dim, int pitch, long long plane, long long base, int i,
                                                 int j, int k)
{
    return base + i + (long long)pitch * j + (dim == 3 ? plane * k : 0);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the
// multiply-xor round with multipliers 0xD2511F53 / 0xCD9E8D57 and the Weyl
// key schedule 0x9E3779B9 / 0xBB67AE85.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, unsigned k0, unsigned k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32 x 32 -> 64-bit product per multiplier (both halves from one wide multiply)
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        const unsigned lo0 = (unsigned)p0, hi0 = (unsigned)(p0 >> 32);
        const unsigned lo1 = (unsigned)p1, hi1 = (unsigned)(p1 >> 32);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Counter words for a draw of `kind` (0 site noise, 1 low-rank noise, 2 coarsest
// sample) on level l and sweep slot; c0 is the pair index.
__device__ __forceinline__ uint4 noise_counter(const CycleState& cs, unsigned pair, unsigned kind, int level,
                                               unsigned slot)
{
    unsigned c1 = (unsigned)cs.cycle;
    unsigned c2 = ((unsigned)(cs.cycle >> 32) & 0xFFFFu) | (cs.chain << 16);
    unsigned c3 = (kind << 24) | ((unsigned)level << 16) | slot;
    return make_uint4(pair, c1, c2, c3);
}

// Box-Muller pair from one Philox block: u = (top 53 bits + 1/2) 2^-53,
// z0 = r cos(2 pi u2), z1 = r sin(2 pi u2), r = sqrt(-2 ln u1).
__device__ __forceinline__ void normal_pair(const uint4 w, double& z0, double& z1)
{
    unsigned long long k1 = (((unsigned long long)w.x << 32) | w.y) >> 11;
    unsigned long long k2 = (((unsigned long long)w.z << 32) | w.w) >> 11;
    double u1 = ((double)k1 + 0.5) * 0x1p-53;
    double u2 = ((double)k2 + 0.5) * 0x1p-53;
    double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// The same draws in FP32: u is the FP32 rounding of (k + 1/2) 2^-53, formed from
// the two 32-bit halves so that the full 53-bit value is used.  The angle is
// reduced to phi = 2 pi (u2 - 1/2) in (-pi, pi], where the hardware sine/cosine
// is accurate to ~4e-7 absolute; cos(2 pi u2) = -cos(phi), sin(2 pi u2) = -sin(phi).
// The logarithm keeps full single precision: near u1 = 1 the radius is small
// and an absolute-error logarithm would be too coarse.  The radius is t / sqrt(t)
// from the reciprocal square root (t = 0 when u1 rounds to 1 is held at 1e-37:
// a radius of ~3e-19 instead of 0).
__device__ __forceinline__ void normal_pair(const uint4 w, float& z0, float& z1)
{
    float u1 = fmaf((float)w.x, 0x1p-32f, fmaf((float)(w.y & 0xFFFFF800u), 0x1p-64f, 0x1p-54f));
    float u2 = fmaf((float)w.z, 0x1p-32f, fmaf((float)(w.w & 0xFFFFF800u), 0x1p-64f, 0x1p-54f));
    const float t = fmaxf(-2.0f * logf(u1), 1e-37f);
    float r = t * rsqrtf(t);
    float s, c;
    __sincosf(6.28318530717958648f * (u2 - 0.5f), &s, &c);
    z0 = -r * c;
    z1 = -r * s;
}

// The four normals of one site-noise block (kind 0, one block per 4-site group of a
// grid row): two Box-Muller pairs from 32-bit uniforms u = (w + 1/2) 2^-32,
// (w.x, w.y) -> z0, z1 for the even columns of the group, (w.z, w.w) -> z2, z3 for
// the odd ones.  FP64: u exact; FP32: the FP32 rounding of u, the same reduced
// angle, accurate logarithm and reciprocal-square-root radius as normal_pair.
__device__ __forceinline__ void normal_quad(const uint4 w, double& z0, double& z1, double& z2, double& z3)
{
    const double r0 = sqrt(-2.0 * log(((double)w.x + 0.5) * 0x1p-32));
    const double r1 = sqrt(-2.0 * log(((double)w.z + 0.5) * 0x1p-32));
    double s, c;
    sincospi(2.0 * (((double)w.y + 0.5) * 0x1p-32), &s, &c);
    z0 = r0 * c;
    z1 = r0 * s;
    sincospi(2.0 * (((double)w.w + 0.5) * 0x1p-32), &s, &c);
    z2 = r1 * c;
    z3 = r1 * s;
}
__device__ __forceinline__ void normal_quad(const uint4 w, float& z0, float& z1, float& z2, float& z3)
{
    const float u1 = fmaf((float)w.x, 0x1p-32f, 0x1p-33f), u2 = fmaf((float)w.y, 0x1p-32f, 0x1p-33f);
    const float u3 = fmaf((float)w.z, 0x1p-32f, 0x1p-33f), u4 = fmaf((float)w.w, 0x1p-32f, 0x1p-33f);
    const float t0 = fmaxf(-2.0f * logf(u1), 1e-37f), t1 = fmaxf(-2.0f * logf(u3), 1e-37f);
    const float r0 = t0 * rsqrtf(t0), r1 = t1 * rsqrtf(t1);
    float s, c;
    __sincosf(6.28318530717958648f * (u2 - 0.5f), &s, &c);
    z0 = -r0 * c;
    z1 = -r0 * s;
    __sincosf(6.28318530717958648f * (u4 - 0.5f), &s, &c);
    z2 = -r1 * c;
    z3 = -r1 * s;
}

// One half of normal_quad: the pair of the even (px = 0) or odd (px = 1) columns,
// transforming only the two words it needs (the same operations as normal_quad)
__device__ __forceinline__ void normal_half(const uint4 w, int px, double& z0, double& z1)
{
    const unsigned wa = px ? w.z : w.x, wb = px ? w.w : w.y;
    const double r = sqrt(-2.0 * log(((double)wa + 0.5) * 0x1p-32));
    double s, c;
    sincospi(2.0 * (((double)wb + 0.5) * 0x1p-32), &s, &c);
    z0 = r * c;
    z1 = r * s;
}
__device__ __forceinline__ void normal_half(const uint4 w, int px, float& z0, float& z1)
{
    const unsigned wa = px ? w.z : w.x, wb = px ? w.w : w.y;
    const float u1 = fmaf((float)wa, 0x1p-32f, 0x1p-33f), u2 = fmaf((float)wb, 0x1p-32f, 0x1p-33f);
    const float t = fmaxf(-2.0f * logf(u1), 1e-37f);
    const float r = t * rsqrtf(t);
    float s, c;
    __sincosf(6.28318530717958648f * (u2 - 0.5f), &s, &c);
    z0 = -r * c;
    z1 = -r * s;
}
template <typename T>
__device__ __forceinline__ void draw_half_ctr(uint4 ctr, unsigned block, int px, unsigned k0, unsigned k1, T& z0,
                                              T& z1)
{
    ctr.x = block;
    normal_half(philox10(ctr, k0, k1), px, z0, z1);
}

// the four site normals of block `block` with the counter words c1..c3 and the key in
// registers (ctr.x is replaced by the block index)
template <typename T>
__device__ __forceinline__ void draw_quad_ctr(uint4 ctr, unsigned block, unsigned k0, unsigned k1, T& z0, T& z1,
                                              T& z2, T& z3)
{
    ctr.x = block;
    normal_quad(philox10(ctr, k0, k1), z0, z1, z2, z3);
}

template <typename T>
__device__ __forceinline__ void draw_pair(const CycleState& cs, unsigned pair, unsigned kind, int level,
                                          unsigned slot, T& z0, T& z1)
{
    uint4 w = philox10(noise_counter(cs, pair, kind, level, slot), (unsigned)cs.seed,
                       (unsigned)(cs.seed >> 32));
    normal_pair(w, z0, z1);
}

// One standard normal of the low-rank noise z'_k (kind 1), evaluated in the
// path precision T (the same draw in both precisions).
template <typename T = double>
__device__ __forceinline__ double lowrank_normal(const CycleState& cs, int level, unsigned slot, int k)
{
    T z0, z1;
    draw_pair<T>(cs, (unsigned)(k >> 1), 1u, level, slot, z0, z1);
    return (double)((k & 1) ? z1 : z0);
}

// Programmatic dependent launch (PTX griddepcontrol): kernels of the captured
// cycle are launched with programmatic stream serialisation, so a kernel's CTAs
// may start while its predecessor drains.  Every such kernel lets its dependents
// launch as soon as its own CTAs are running and calls pdl_wait() in every CTA
// before it touches anything an earlier kernel wrote (the wait returns once the
// predecessor has completed and its memory is visible; since every kernel waits,
// completion is transitive along the chain).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// 1/a and sqrt(a) of a positive FP32 diagonal from one reciprocal square root
// (relative error ~2e-7, below the FP32 rounding of the state update)
__device__ __forceinline__ void inv_and_sqrt(float a, float& inv, float& sq)
{
    float r = rsqrtf(a);
    inv = r * r;
    sq = a * r;
}

// host: launch with programmatic stream serialisation (see pdl_wait)
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace mgmc
