// kernels.cu -- CUDA kernels of one MGMC V-cycle (Alg. 1) for sm_103a.
//
// Per level l (finest first) the host enqueues:
//   k_sweep_colour  x nu1 sweeps x colours : forward random Gibbs sweep (Alg. 3)
//   k_lowrank_v, k_lowrank_apply           : theta' = theta* - G (B^T theta*) (Eq. low_rank_update):
//                                            one CTA forms the m-vector, many CTAs apply G's rows
//   k_residual, k_restrict                 : r = f_l - A_l theta' on the fine grid, then
//                                            f_{l-1} = P^T r and d_{l-1} = d_l - B_l^T theta'
// the grids with n <= coarse_max_n run as one k_coarse_cycle (coarse.cu),
// which ends in the exact coarsest Cholesky sample (Sec. 3.5), and back up:
//   k_prolong                              : theta += P psi_{l-1}
//   k_sweep_colour  (reverse colours), k_lowrank_v + k_lowrank_apply (backward G)
// and k_qoi_advance records F^T theta and advances the cycle counter.
//
// Low-rank bookkeeping: the right-hand side of level l is kept as
// f_l = fdense_l + B_l Gamma^-1 d_l with a dense field fdense_l and an m-vector
// d_l; on the finest level fdense_L = 0 and d_L = y (Eq. f_ell_definition).
// Alg. 3 is evaluated as
//   theta*_s = Gibbs sweep of the dense part fdense_l + D^1/2 z   (k_sweep_colour)
//   theta'   = theta*_s - G (B^T theta*_s - d_l - L_Gamma z')     (k_lowrank_v, k_lowrank_apply)
// which equals theta* - G B^T theta* of Eq. lowrank_gibbs_two_steps with
// theta* = theta*_s + C (Gamma^-1 d_l + xi_LR), because C - G B^T C = G Gamma
// (Eq. Bellstar_definition); no term of size |Gamma^-1 y| is ever formed.
// Restriction: fdense_{l-1} = P^T (fdense_l - A_l theta'), d_{l-1} = d_l - B_l^T theta'
// (P^T B_l = B_{l-1}, Eq. A_ell_1_B_ell_1); B_l^T theta' = z - (B_l^T G) v needs no
// second read of theta'.
#include "kernels.cuh"

#include <type_traits>

namespace mgmc {

// Map a work item of colour `colour` to (row j, k, x parity, x block q).
// Fine 5/7-point levels run the two red-black groups (colour = 0 even, 1 odd);
// Galerkin levels run the 2^d parity classes (colour = px + 2 py + 4 pz).
template <int DIM>
__device__ __forceinline__ bool colour_item(int n, bool redblack, int colour, long long item, int& j, int& k,
                                            int& px, int& q)
{
    int nq = (n + 3) >> 2;
    q = (int)(item % nq);
    long long r = item / nq;
    if (redblack) {
        int nr = DIM == 3 ? n * n : n;
        if (r >= nr) return false;
        j = (int)(r % n);
        k = DIM == 3 ? (int)(r / n) : 0;
        px = (j + k + colour) & 1;
    } else {
        int py = (colour >> 1) & 1, pz = (colour >> 2) & 1;
        int ny = (n - py + 1) >> 1;
        int nz = DIM == 3 ? (n - pz + 1) >> 1 : 1;
        if (r >= (long long)ny * nz) return false;
        j = 2 * (int)(r % ny) + py;
        k = DIM == 3 ? 2 * (int)(r / ny) + pz : 0;
        px = colour & 1;
    }
    return 4 * q + px < n;
}

template <typename T, int DIM>
__device__ __forceinline__ void sweep_item(const DevLevel<T>& L, const DevProblem& P, const CycleState& cs,
                                           bool redblack, int colour, unsigned slot, long long item)
{
    int j, k, px, q;
    if (!colour_item<DIM>(L.n, redblack, colour, item, j, k, px, q)) return;
    int n = L.n;
    int nq = (n + 3) >> 2;
    int i0 = 4 * q + px;
    bool has1 = i0 + 2 < n;
    T z0 = T(0), z1 = T(0);
    if (cs.noise)  // the block of the group's row, this colour's half of it
        draw_half_ctr<T>(noise_counter(cs, 0u, 0u, L.level, slot), (unsigned)(((long long)k * n + j) * nq + q), px,
                         (unsigned)cs.seed, (unsigned)(cs.seed >> 32), z0, z1);
    long long e = site_offset(DIM, L.pitch, L.plane, L.base, i0, j, k);
    if (L.fine) {
        L.x[e] = fine_update<DIM>(L, e, z0);
        if (has1) L.x[e + 2] = fine_update<DIM>(L, e + 2, z1);
    } else {
        L.x[e] = coarse_update<DIM>(L, e, z0);
        if (has1) L.x[e + 2] = coarse_update<DIM>(L, e + 2, z1);
    }
}

template <typename T, int DIM>
__global__ void k_sweep_colour(DevLevel<T> L, DevProblem P, int redblack, int colour, unsigned slot)
{
    const CycleState cs = *P.cs;
    long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    sweep_item<T, DIM>(L, P, cs, redblack != 0, colour, slot, item);
}

// 25-point grids (squared shifted Laplacian, FP64 2D): colour c = cx + 3 cy is the class
// (i mod 3, j mod 3) = (cx, cy); one thread per site of the class.  Site i of row j takes
// the normal of its member of the row's 4-site noise block (the same draw as every
// other sweep kernel: block j nq + (i >> 2), half i & 1, member (i >> 1) & 1).
__device__ __forceinline__ long long colour25_sites(int n, int colour)
{
    const int nx = (n - colour % 3 + 2) / 3, ny = (n - colour / 3 + 2) / 3;
    return nx > 0 && ny > 0 ? (long long)nx * ny : 0;
}

// the t-th site (i, j) of class `colour` = cx + 3 cy
__device__ __forceinline__ void colour25_site(int n, int colour, long long t, int& i, int& j)
{
    const int cx = colour % 3, cy = colour / 3;
    const int nx = (n - cx + 2) / 3;
    i = cx + 3 * (int)(t % nx);
    j = cy + 3 * (int)(t / nx);
}

// the site normals of one sweep of a 25-point grid into zb[j n + i], the draws of
// sweep25_site: item (j, q, px) gives the pair of sites 4q + px and 4q + px + 2 (z0, z1
// of the half block px of row j's block q)
__device__ __forceinline__ void draw25_pair(const DevLevel<double>& L, const CycleState& cs, unsigned slot,
                                            double* zb, long long item)
{
    const int n = L.n, nq = (n + 3) >> 2;
    const int px = (int)(item & 1);
    const long long rq = item >> 1;
    const int q = (int)(rq % nq), j = (int)(rq / nq);
    const int i0 = 4 * q + px;
    if (i0 >= n) return;
    double z0, z1;
    draw_half_ctr<double>(noise_counter(cs, 0u, 0u, L.level, slot), (unsigned)(j * nq + q), px, (unsigned)cs.seed,
                          (unsigned)(cs.seed >> 32), z0, z1);
    zb[(long long)j * n + i0] = z0;
    if (i0 + 2 < n) zb[(long long)j * n + i0 + 2] = z1;
}

__device__ __forceinline__ void sweep25_site(const DevLevel<double>& L, const CycleState& cs, int colour,
                                             unsigned slot, long long t)
{
    const int n = L.n;
    int i, j;
    colour25_site(n, colour, t, i, j);
    double z = 0.0;
    if (cs.noise) {
        double z0, z1;
        const int nq = (n + 3) >> 2;
        draw_half_ctr<double>(noise_counter(cs, 0u, 0u, L.level, slot), (unsigned)(j * nq + (i >> 2)), i & 1,
                              (unsigned)cs.seed, (unsigned)(cs.seed >> 32), z0, z1);
        z = ((i >> 1) & 1) ? z1 : z0;
    }
    const long long e = site_offset(2, L.pitch, L.plane, L.base, i, j, 0);
    L.x[e] = update25(L, e, z);
}

__global__ void k_sweep25(DevLevel<double> L, DevProblem P, int colour, unsigned slot)
{
    const CycleState cs = *P.cs;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= colour25_sites(L.n, colour)) return;
    sweep25_site(L, cs, colour, slot, t);
}

// Exact coarsest sample theta_0 = A~_0^-1 f_0 + L_0^-T z (Sec. 3.5) with the coarsest
// grid's v-th visit slot (W-cycle), one CTA: f_0 = fdense_0 + B_0 Gamma^-1 d_0, the
// forward solve with the Cholesky factor, + z (kind 2, pair s >> 1, member s & 1),
// the backward solve.
template <typename T>
__device__ void coarsest_slot_body(const DevLevel<T>& L, const DevProblem& P, const CycleState& cs,
                                   const double* __restrict__ chol, int n0, unsigned slot, double* r, double* g)
{
    const int n = L.n;
    for (int s = threadIdx.x; s < n0; s += blockDim.x) {
        const int i = s % n, j = (s / n) % n, k = L.dim == 3 ? s / (n * n) : 0;
        r[s] = L.f ? (double)L.f[site_offset(L.dim, L.pitch, L.plane, L.base, i, j, k)] : 0.0;
    }
    for (int kk = threadIdx.x; kk < P.m; kk += blockDim.x) {
        double acc = 0.0;
        for (int t = 0; t < P.m; ++t) acc += P.Gamma_inv[kk * P.m + t] * L.d[t];
        g[kk] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int kk = 0; kk < P.m; ++kk)
            for (int t = L.bcol_ptr[kk]; t < L.bcol_ptr[kk + 1]; ++t) r[L.bcol_dense[t]] += L.bcol_w[t] * g[kk];
    __syncthreads();
    for (int i = 0; i < n0; ++i) {
        if (threadIdx.x == 0) r[i] = r[i] / chol[(long long)i * n0 + i];
        __syncthreads();
        const double yi = r[i];
        for (int t = i + 1 + threadIdx.x; t < n0; t += blockDim.x) r[t] -= chol[(long long)t * n0 + i] * yi;
        __syncthreads();
    }
    if (cs.noise)
        for (int s = threadIdx.x; s < n0; s += blockDim.x) {
            double z0, z1;
            draw_pair<double>(cs, (unsigned)(s >> 1), 2u, 0, slot, z0, z1);
            r[s] += (s & 1) ? z1 : z0;
        }
    __syncthreads();
    for (int i = n0 - 1; i >= 0; --i) {
        if (threadIdx.x == 0) r[i] = r[i] / chol[(long long)i * n0 + i];
        __syncthreads();
        const double xi = r[i];
        for (int t = threadIdx.x; t < i; t += blockDim.x) r[t] -= chol[(long long)i * n0 + t] * xi;
        __syncthreads();
    }
    for (int s = threadIdx.x; s < n0; s += blockDim.x) {
        const int i = s % n, j = (s / n) % n, k = L.dim == 3 ? s / (n * n) : 0;
        L.x[site_offset(L.dim, L.pitch, L.plane, L.base, i, j, k)] = (T)r[s];
    }
}

template <typename T>
__global__ void k_coarsest_slot(DevLevel<T> L, DevProblem P, const double* __restrict__ chol, int n0,
                                unsigned slot)
{
    __shared__ double r[MGMC_MAX_COARSEST];
    __shared__ double g[kMaxObs];
    const CycleState cs = *P.cs;
    coarsest_slot_body<T>(L, P, cs, chol, n0, slot, r, g);
}

template <typename T, int DIM>
__device__ __forceinline__ T prolong_site(const DevLevel<T>& C, int fi, int fj, int fk)
{
    // fine index f: odd -> coarse (f-1)/2 with weight 1; even -> coarse f/2-1 and f/2, weight 1/2
    T acc = T(0);
    int cx[2], cy[2], cz[2];
    T wx[2], wy[2], wz[2];
    int nx, ny, nz;
    auto axis = [](int f, int* c, T* w, int& cnt) {
        if (f & 1) {
            c[0] = (f - 1) >> 1;
            w[0] = T(1);
            cnt = 1;
        } else {
            c[0] = (f >> 1) - 1;
            c[1] = f >> 1;
            w[0] = w[1] = T(0.5);
            cnt = 2;
        }
    };
    axis(fi, cx, wx, nx);
    axis(fj, cy, wy, ny);
    if (DIM == 3) {
        axis(fk, cz, wz, nz);
    } else {
        cz[0] = 0;
        wz[0] = T(1);
        nz = 1;
    }
    for (int c = 0; c < nz; ++c)
        for (int b = 0; b < ny; ++b)
            for (int a = 0; a < nx; ++a) {
                // ghost indices -1 and n read the zero ring
                long long e = site_offset(DIM, C.pitch, C.plane, C.base, cx[a], cy[b], cz[c]);
                acc += wz[c] * wy[b] * wx[a] * C.x[e];
            }
    return acc;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Low-rank step of the unfused path (Alg. 3), two launches.  k_lowrank_v (one CTA):
// z = B^T theta*_s, v = z - d - L_Gamma z' into lrv (dir >= 0); for dir < 0 (no
// smoothing) only d_{l-1} = d_l - z.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void lowrank_v_body(const DevLevel<T>& L, const DevProblem& P, const CycleState& cs,
                                               int dir, unsigned slot, int want_dnext, double* z, double* zp)
{
    const int m = P.m;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        double acc = 0.0;
        for (int t = L.bcol_ptr[k]; t < L.bcol_ptr[k + 1]; ++t) acc += L.bcol_w[t] * (double)L.x[L.bcol_site[t]];
        z[k] = acc;
        zp[k] = (dir >= 0 && cs.noise) ? lowrank_normal<T>(cs, L.level, slot, k) : 0.0;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        if (dir >= 0) {
            double lz = 0.0;
            if (cs.noise) {
                if (P.gamma_diag)
                    lz = P.LG[k * m + k] * zp[k];
                else
                    for (int t = 0; t <= k; ++t) lz += P.LG[k * m + t] * zp[t];
            }
            L.lrv[k] = z[k] - L.d[k] - lz;
            L.lrv[m + k] = z[k];
        } else if (want_dnext) {
            L.dnext[k] = L.d[k] - z[k];
        }
    }
}

template <typename T>
__global__ void k_lowrank_v(DevLevel<T> L, DevProblem P, int dir, unsigned slot, int want_dnext)
{
    __shared__ double z[kMaxObs];
    __shared__ double zp[kMaxObs];
    const CycleState cs = *P.cs;
    lowrank_v_body<T>(L, P, cs, dir, slot, want_dnext, z, zp);
}

// theta' = theta*_s - G v on G's rows r0, r0 + stride, ...
template <typename T>
__device__ __forceinline__ void lowrank_rows(const DevLevel<T>& L, int m, int dir, const double* v, int r0, int stride)
{
    const int rows = L.g_rows[dir];
    const double* G = L.g_val[dir];
    for (int r = r0; r < rows; r += stride) {
        double acc = 0.0;
        for (int kk = 0; kk < m; ++kk) acc += G[(long long)r * m + kk] * v[kk];
        const long long s = L.g_site[dir][r];
        L.x[s] = (T)((double)L.x[s] - acc);
    }
}

// d_{l-1} = d_l - B^T theta' = d_l - z + (B^T G) v
template <typename T>
__device__ __forceinline__ void lowrank_dnext(const DevLevel<T>& L, int m, const double* v)
{
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        double acc = 0.0;
        for (int t = 0; t < m; ++t) acc += L.BtG[k * m + t] * v[t];
        L.dnext[k] = L.d[k] - L.lrv[m + k] + acc;
    }
}

// theta' = theta*_s - G v on G's rows, spread over the grid; with want_dnext block 0
// also forms d_{l-1} = d_l - B^T theta' = d_l - z + (B^T G) v
template <typename T>
__global__ void k_lowrank_apply(DevLevel<T> L, DevProblem P, int dir, int want_dnext)
{
    __shared__ double v[kMaxObs];
    const int m = P.m;
    for (int k = threadIdx.x; k < m; k += blockDim.x) v[k] = L.lrv[k];
    __syncthreads();
    lowrank_rows<T>(L, m, dir, v, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
    if (want_dnext && blockIdx.x == 0) lowrank_dnext<T>(L, m, v);
}

// r = f_l - A_l theta at every interior site of the fine grid (the restriction's input)
template <typename T, int DIM>
__device__ __forceinline__ void residual_site(const DevLevel<T>& F, long long s)
{
    int i = (int)(s % F.n), j = (int)((s / F.n) % F.n), k = DIM == 3 ? (int)(s / ((long long)F.n * F.n)) : 0;
    long long e = site_offset(DIM, F.pitch, F.plane, F.base, i, j, k);
    F.res[e] = (F.f ? F.f[e] : T(0)) - apply_A<DIM>(F, e);
}

template <typename T, int DIM>
__global__ void k_residual(DevLevel<T> F)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long N = (long long)F.n * F.n * (DIM == 3 ? F.n : 1);
    if (s >= N) return;
    residual_site<T, DIM>(F, s);
}

// f_c(I) = sum_p w(p) r(2I + p) over the 3^d fine sites 2I + p, p in {0, 1, 2}^d, from the residual field
template <typename T, int DIM>
__device__ __forceinline__ void restrict_site(const DevLevel<T>& F, const DevLevel<T>& C, long long s)
{
    int I = (int)(s % C.n), J = (int)((s / C.n) % C.n), K = DIM == 3 ? (int)(s / ((long long)C.n * C.n)) : 0;
    T acc = T(0);
    const int nz = DIM == 3 ? 3 : 1;
    for (int pz = 0; pz < nz; ++pz)
        for (int py = 0; py < 3; ++py)
            for (int px = 0; px < 3; ++px) {
                long long e = site_offset(DIM, F.pitch, F.plane, F.base, 2 * I + px, 2 * J + py,
                                          DIM == 3 ? 2 * K + pz : 0);
                T wgt = (T)(pw(px - 1) * pw(py - 1) * (DIM == 3 ? pw(pz - 1) : 1.0));
                acc += wgt * F.res[e];
            }
    C.f[site_offset(DIM, C.pitch, C.plane, C.base, I, J, K)] = acc;
}

template <typename T, int DIM>
__global__ void k_restrict(DevLevel<T> F, DevLevel<T> C)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long N = (long long)C.n * C.n * (DIM == 3 ? C.n : 1);
    if (s >= N) return;
    restrict_site<T, DIM>(F, C, s);
}

template <typename T, int DIM>
__device__ __forceinline__ void prolong_add_site(const DevLevel<T>& C, const DevLevel<T>& F, long long s)
{
    int i = (int)(s % F.n), j = (int)((s / F.n) % F.n), k = DIM == 3 ? (int)(s / ((long long)F.n * F.n)) : 0;
    long long e = site_offset(DIM, F.pitch, F.plane, F.base, i, j, k);
    F.x[e] = F.x[e] + prolong_site<T, DIM>(C, i, j, k);
}

template <typename T, int DIM>
__global__ void k_prolong(DevLevel<T> C, DevLevel<T> F)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long N = (long long)F.n * F.n * (DIM == 3 ? F.n : 1);
    if (s >= N) return;
    prolong_add_site<T, DIM>(C, F, s);
}

// ---------------------------------------------------------------------------
// Grids 0..top of the general path in one CTA (2D).  The host lists the phases of one
// visit of grid `top` -- with the V- or W-cycle recursion below it, in the order and
// with the noise slots of the per-launch path -- and the CTA runs them one after the
// other, a barrier after each phase (and between colours).  Every phase evaluates the
// per-site functions of the per-launch kernels (the two agree to rounding: the compiler
// may contract their multiply-adds differently); one launch replaces the hundreds of
// small launches the coarse visits of a W-cycle need.
// ---------------------------------------------------------------------------
// The descriptors of grids 0..top and (up to kSmallMaxOps) the phase list are staged in
// shared memory first, so that a phase's data loads do not wait on two dependent global
// loads (the phase, then the descriptor fields) each time.
template <typename T>
__global__ void __launch_bounds__(kSmallCycleThreads)
    k_cycle_small(const DevLevel<T>* __restrict__ lv_g, int top, DevProblem P, const double* __restrict__ chol,
                  int n0, const int4* __restrict__ ops_g, int n_ops, double* __restrict__ zb)
{
    __shared__ double r[MGMC_MAX_COARSEST];
    __shared__ double g[kMaxObs];
    __shared__ double z[kMaxObs];
    __shared__ double zp[kMaxObs];
    __shared__ DevLevel<T> lv[kSmallMaxLevels];
    __shared__ int4 ops_s[kSmallMaxOps];
    {
        const int words = (top + 1) * (int)(sizeof(DevLevel<T>) / sizeof(unsigned long long));
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(lv_g);
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(lv);
        for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
        const int ns = n_ops < kSmallMaxOps ? n_ops : kSmallMaxOps;
        for (int q = threadIdx.x; q < ns; q += blockDim.x) ops_s[q] = ops_g[q];
    }
    __syncthreads();
    const CycleState cs = *P.cs;
    const int m = P.m;
    for (int q = 0; q < n_ops; ++q) {
        const int4 op = q < kSmallMaxOps ? ops_s[q] : ops_g[q];
        const DevLevel<T>& L = lv[op.y];
        const long long N = (long long)L.n * L.n;
        switch (op.x) {
        case kOpSweep: {
            const unsigned slot = (unsigned)op.z;
            const int dir = op.w;
            const int nq = (L.n + 3) >> 2;
            bool done = false;
            if constexpr (std::is_same<T, double>::value) {
                if (L.rad == 2) {
                    // the sweep's normals first, for all sites at once (one draw per pair), then
                    // the nine classes read them: the colour phases carry no Box-Muller transform
                    if (cs.noise) {
                        const long long items = (long long)L.n * nq * 2;
                        for (long long it = threadIdx.x; it < items; it += blockDim.x) draw25_pair(L, cs, slot, zb, it);
                        __syncthreads();
                    }
                    for (int ci = 0; ci < 9; ++ci) {
                        const int c = dir == 0 ? ci : 8 - ci;
                        const long long sites = colour25_sites(L.n, c);
                        for (long long t = threadIdx.x; t < sites; t += blockDim.x) {
                            int i, j;
                            colour25_site(L.n, c, t, i, j);
                            const double zz = cs.noise ? zb[(long long)j * L.n + i] : 0.0;
                            const long long e = site_offset(2, L.pitch, L.plane, L.base, i, j, 0);
                            L.x[e] = update25(L, e, zz);
                        }
                        __syncthreads();
                    }
                    done = true;
                }
            }
            if (done) break;
            if (L.fine) {
                for (int g2 = 0; g2 < 2; ++g2) {
                    const int colour = dir == 0 ? g2 : 1 - g2;
                    const long long items = (long long)L.n * nq;
                    for (long long it = threadIdx.x; it < items; it += blockDim.x)
                        sweep_item<T, 2>(L, P, cs, true, colour, slot, it);
                    __syncthreads();
                }
            } else {
                const int seq2[4] = {0, 3, 2, 1};
                for (int ci = 0; ci < 4; ++ci) {
                    const int c = seq2[dir == 0 ? ci : 3 - ci];
                    const int py = (c >> 1) & 1;
                    const long long items = (long long)((L.n - py + 1) / 2) * nq;
                    for (long long it = threadIdx.x; it < items; it += blockDim.x)
                        sweep_item<T, 2>(L, P, cs, false, c, slot, it);
                    __syncthreads();
                }
            }
            break;
        }
        case kOpLowrank: {
            if (m == 0) break;
            const int dir = (op.w & 3) == 2 ? -1 : (op.w & 3);
            const int dn = (op.w >> 2) & 1;
            lowrank_v_body<T>(L, P, cs, dir, (unsigned)op.z, dn, z, zp);
            __syncthreads();
            if (dir >= 0) {
                for (int k = threadIdx.x; k < m; k += blockDim.x) zp[k] = L.lrv[k];
                __syncthreads();
                lowrank_rows<T>(L, m, dir, zp, threadIdx.x, blockDim.x);
                if (dn) lowrank_dnext<T>(L, m, zp);
            }
            break;
        }
        case kOpRestrict: {
            for (long long s2 = threadIdx.x; s2 < N; s2 += blockDim.x) residual_site<T, 2>(L, s2);
            __syncthreads();
            const DevLevel<T>& C = lv[op.y - 1];
            const long long Nc = (long long)C.n * C.n;
            for (long long s2 = threadIdx.x; s2 < Nc; s2 += blockDim.x) restrict_site<T, 2>(L, C, s2);
            break;
        }
        case kOpZero:
            for (long long e = threadIdx.x; e < L.alloc; e += blockDim.x) L.x[e] = T(0);
            break;
        case kOpCoarsest:
            coarsest_slot_body<T>(lv[0], P, cs, chol, n0, (unsigned)op.z, r, g);
            break;
        case kOpProlong: {
            const DevLevel<T>& C = lv[op.y - 1];
            for (long long s2 = threadIdx.x; s2 < N; s2 += blockDim.x) prolong_add_site<T, 2>(C, L, s2);
            break;
        }
        default:
            break;
        }
        __syncthreads();
    }
}

// The whole V-cycle below (and including) level `top`, one CTA.
// levels[0..top] are the device descriptors, index = paper level.
// F^T theta of the finest level into qoi[step]; then step += 1, cycle += 1.
template <typename T>
__global__ void k_qoi_advance(DevLevel<T> L, int n_qoi, const long long* q_site, const double* q_w, DevProblem P)
{
    __shared__ double part[256];
    double acc = 0.0;
    for (int t = threadIdx.x; t < n_qoi; t += blockDim.x) acc += q_w[t] * (double)L.x[q_site[t]];
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        CycleState* cs = P.cs;
        double q = part[0];
        if (cs->qoi) cs->qoi[cs->step] = q;
        if (!isfinite(q)) atomicOr(&cs->status, kStatusNumeric);
        cs->step += 1;
        cs->cycle += 1;
    }
}

__global__ void k_set_cycle(CycleState* cs, unsigned long long seed, unsigned long long cycle, unsigned chain,
                            int noise, double* qoi)
{
    cs->seed = seed;
    cs->cycle = cycle;
    cs->chain = chain;
    cs->noise = noise;
    cs->qoi = qoi;
    cs->step = 0;
}

// dense user field <-> padded finest-level state
template <typename T, int DIM>
__global__ void k_pack(DevLevel<T> L, T* __restrict__ dense, int to_padded)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long N = (long long)L.n * L.n * (DIM == 3 ? L.n : 1);
    if (s >= N) return;
    int i = (int)(s % L.n), j = (int)((s / L.n) % L.n), k = DIM == 3 ? (int)(s / ((long long)L.n * L.n)) : 0;
    long long e = site_offset(DIM, L.pitch, L.plane, L.base, i, j, k);
    if (to_padded)
        L.x[e] = dense[s];
    else
        dense[s] = L.x[e];
}

// Batched 2D form: block (j, c) moves row j of chain c (no divisions).
struct DensePtrs {
    void* p[kPackChunk];
};
template <typename T>
__global__ void k_pack_batch(const PackJob<T>* __restrict__ jobs, DensePtrs dense, int to_padded)
{
    const PackJob<T> J = jobs[blockIdx.y];
    const int j = blockIdx.x;
    if (j >= J.n) return;
    T* d = (T*)dense.p[blockIdx.y] + (long long)j * J.n;
    T* x = J.x + J.base + (long long)J.pitch * j;
    if (to_padded)
        for (int i = threadIdx.x; i < J.n; i += blockDim.x) x[i] = d[i];
    else
        for (int i = threadIdx.x; i < J.n; i += blockDim.x) d[i] = x[i];
}

// ---------------------------------------------------------------------------
// residual norm pieces for the mean solve: u = Gamma^-1 (y - B^T x) (m-vector),
// then r = B u - A x summed as ||r||^2 per block, reduced by one block.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_resid_u(DevLevel<T> L, DevProblem P, double* u)
{
    __shared__ double z[kMaxObs];
    const int m = P.m;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        double acc = 0.0;
        for (int t = L.bcol_ptr[k]; t < L.bcol_ptr[k + 1]; ++t) acc += L.bcol_w[t] * (double)L.x[L.bcol_site[t]];
        z[k] = acc;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < m; k += blockDim.x) z[k] = L.d[k] - z[k];   // d_L - B^T x
    __syncthreads();
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        double acc = 0.0;
        for (int t = 0; t < m; ++t) acc += P.Gamma_inv[k * m + t] * z[t];
        u[k] = acc;
    }
}

template <typename T, int DIM>
__global__ void k_resid_norm(DevLevel<T> L, const double* u, double* partial)
{
    __shared__ double part[256];
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long N = (long long)L.n * L.n * (DIM == 3 ? L.n : 1);
    double v = 0.0;
    if (s < N) {
        int i = (int)(s % L.n), j = (int)((s / L.n) % L.n), k = DIM == 3 ? (int)(s / ((long long)L.n * L.n)) : 0;
        long long e = site_offset(DIM, L.pitch, L.plane, L.base, i, j, k);
        double r = -(double)apply_A<DIM>(L, e);
        if (L.brow_ptr) {
            int row = j + L.n * k;
            for (int t = L.brow_ptr[row]; t < L.brow_ptr[row + 1]; ++t)
                if (L.bent_i[t] == i) r += L.bent_w[t] * u[L.bent_k[t]];
        }
        v = r * r;
    }
    part[threadIdx.x] = v;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) part[threadIdx.x] += part[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = part[0];
}

__global__ void k_sum(const double* partial, int n, double* out)
{
    __shared__ double part[256];
    double acc = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) acc += partial[t];
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) part[threadIdx.x] += part[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0];
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
static inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

template <typename T>
void launch_sweep(const DevLevel<T>& L, const DevProblem& P, int dir, unsigned slot, cudaStream_t st, int& launches)
{
    const int bs = 256;
    int nq = (L.n + 3) / 4;
    if constexpr (std::is_same<T, double>::value) {
        if (L.rad == 2) {
            // the nine classes in code order forward, reversed backward
            for (int ci = 0; ci < 9; ++ci) {
                const int c = dir == 0 ? ci : 8 - ci;
                const long long sites = (long long)((L.n - c % 3 + 2) / 3) * ((L.n - c / 3 + 2) / 3);
                if (sites <= 0) continue;
                k_sweep25<<<blocks_for(sites, bs), bs, 0, st>>>(L, P, c, slot);
                ++launches;
            }
            return;
        }
    }
    if (L.fine) {
        long long rows = L.dim == 3 ? (long long)L.n * L.n : L.n;
        for (int g = 0; g < 2; ++g) {
            int colour = dir == 0 ? g : 1 - g;
            unsigned nb = blocks_for(rows * nq, bs);
            if (L.dim == 2)
                k_sweep_colour<T, 2><<<nb, bs, 0, st>>>(L, P, 1, colour, slot);
            else
                k_sweep_colour<T, 3><<<nb, bs, 0, st>>>(L, P, 1, colour, slot);
            ++launches;
        }
        return;
    }
    const int seq2[4] = {0, 3, 2, 1};
    const int seq3[8] = {0, 6, 5, 3, 4, 2, 1, 7};
    int nc = L.dim == 2 ? 4 : 8;
    for (int ci = 0; ci < nc; ++ci) {
        int c = L.dim == 2 ? seq2[dir == 0 ? ci : nc - 1 - ci] : seq3[dir == 0 ? ci : nc - 1 - ci];
        int py = (c >> 1) & 1, pz = (c >> 2) & 1;
        long long rows = (long long)((L.n - py + 1) / 2) * (L.dim == 3 ? (L.n - pz + 1) / 2 : 1);
        unsigned nb = blocks_for(rows * nq, bs);
        if (L.dim == 2)
            k_sweep_colour<T, 2><<<nb, bs, 0, st>>>(L, P, 0, c, slot);
        else
            k_sweep_colour<T, 3><<<nb, bs, 0, st>>>(L, P, 0, c, slot);
        ++launches;
    }
}

template <typename T>
void launch_lowrank(const DevLevel<T>& L, const DevProblem& P, int dir, unsigned slot, bool dnext, cudaStream_t st,
                    int& launches)
{
    if (P.m == 0) return;
    k_lowrank_v<T><<<1, 256, 0, st>>>(L, P, dir, slot, dnext ? 1 : 0);
    ++launches;
    if (dir < 0) return;
    const int rows = L.g_rows[dir];
    int nb = (rows + 255) / 256;
    nb = nb < 1 ? 1 : (nb > 1024 ? 1024 : nb);
    k_lowrank_apply<T><<<nb, 256, 0, st>>>(L, P, dir, dnext ? 1 : 0);
    ++launches;
}

template <typename T>
void launch_restrict(const DevLevel<T>& F, const DevLevel<T>& C, cudaStream_t st, int& launches)
{
    long long NF = (long long)F.n * F.n * (F.dim == 3 ? F.n : 1);
    long long N = (long long)C.n * C.n * (C.dim == 3 ? C.n : 1);
    if (C.dim == 2) {
        k_residual<T, 2><<<blocks_for(NF, 256), 256, 0, st>>>(F);
        k_restrict<T, 2><<<blocks_for(N, 256), 256, 0, st>>>(F, C);
    } else {
        k_residual<T, 3><<<blocks_for(NF, 256), 256, 0, st>>>(F);
        k_restrict<T, 3><<<blocks_for(N, 256), 256, 0, st>>>(F, C);
    }
    launches += 2;
}

template <typename T>
void launch_prolong(const DevLevel<T>& C, const DevLevel<T>& F, cudaStream_t st, int& launches)
{
    long long N = (long long)F.n * F.n * (F.dim == 3 ? F.n : 1);
    if (F.dim == 2)
        k_prolong<T, 2><<<blocks_for(N, 256), 256, 0, st>>>(C, F);
    else
        k_prolong<T, 3><<<blocks_for(N, 256), 256, 0, st>>>(C, F);
    ++launches;
}

template <typename T>
void launch_coarsest_slot(const DevLevel<T>& L, const DevProblem& P, const double* chol, int n0, unsigned slot,
                          cudaStream_t st, int& launches)
{
    k_coarsest_slot<T><<<1, 256, 0, st>>>(L, P, chol, n0, slot);
    ++launches;
}

template <typename T>
void launch_cycle_small(const DevLevel<T>* levels_dev, int top, const DevProblem& P, const double* chol, int n0,
                        const int4* ops, int n_ops, double* zb, cudaStream_t st, int& launches)
{
    k_cycle_small<T><<<1, kSmallCycleThreads, 0, st>>>(levels_dev, top, P, chol, n0, ops, n_ops, zb);
    ++launches;
}

template <typename T>
void launch_qoi(const DevLevel<T>& L, int n_qoi, const long long* q_site, const double* q_w, const DevProblem& P,
                cudaStream_t st, int& launches)
{
    k_qoi_advance<T><<<1, 256, 0, st>>>(L, n_qoi, q_site, q_w, P);
    ++launches;
}

void launch_set_cycle(CycleState* cs, unsigned long long seed, unsigned long long cycle, unsigned chain, int noise,
                      double* qoi, cudaStream_t st)
{
    k_set_cycle<<<1, 1, 0, st>>>(cs, seed, cycle, chain, noise, qoi);
}

template <typename T>
void launch_pack(const DevLevel<T>& L, T* dense, bool to_padded, cudaStream_t st)
{
    long long N = (long long)L.n * L.n * (L.dim == 3 ? L.n : 1);
    if (L.dim == 2)
        k_pack<T, 2><<<blocks_for(N, 256), 256, 0, st>>>(L, dense, to_padded ? 1 : 0);
    else
        k_pack<T, 3><<<blocks_for(N, 256), 256, 0, st>>>(L, dense, to_padded ? 1 : 0);
}

template <typename T>
void launch_pack_batch(const PackJob<T>* jobs, void* const* dense, int count, int max_n, bool to_padded,
                       cudaStream_t st)
{
    for (int c0 = 0; c0 < count; c0 += kPackChunk) {
        const int k = count - c0 < kPackChunk ? count - c0 : kPackChunk;
        DensePtrs d{};
        for (int c = 0; c < k; ++c) d.p[c] = dense[c0 + c];
        k_pack_batch<T><<<dim3((unsigned)max_n, (unsigned)k), 256, 0, st>>>(jobs + c0, d, to_padded ? 1 : 0);
    }
}

template <typename T>
void launch_resid(const DevLevel<T>& L, const DevProblem& P, double* u, double* partial, int max_partial,
                  double* out, cudaStream_t st)
{
    if (P.m > 0) k_resid_u<T><<<1, 64, 0, st>>>(L, P, u);
    long long N = (long long)L.n * L.n * (L.dim == 3 ? L.n : 1);
    unsigned nb = blocks_for(N, 256);
    (void)max_partial;
    if (L.dim == 2)
        k_resid_norm<T, 2><<<nb, 256, 0, st>>>(L, P.m > 0 ? u : nullptr, partial);
    else
        k_resid_norm<T, 3><<<nb, 256, 0, st>>>(L, P.m > 0 ? u : nullptr, partial);
    k_sum<<<1, 256, 0, st>>>(partial, (int)nb, out);
}

#define MGMC_INSTANTIATE(T)                                                                                       \
    template void launch_sweep<T>(const DevLevel<T>&, const DevProblem&, int, unsigned, cudaStream_t, int&);     \
    template void launch_lowrank<T>(const DevLevel<T>&, const DevProblem&, int, unsigned, bool, cudaStream_t, int&); \
    template void launch_restrict<T>(const DevLevel<T>&, const DevLevel<T>&, cudaStream_t, int&);                \
    template void launch_prolong<T>(const DevLevel<T>&, const DevLevel<T>&, cudaStream_t, int&);                 \
    template void launch_coarsest_slot<T>(const DevLevel<T>&, const DevProblem&, const double*, int, unsigned,     \
                                          cudaStream_t, int&);                                                   \
    template void launch_cycle_small<T>(const DevLevel<T>*, int, const DevProblem&, const double*, int,            \
                                        const int4*, int, double*, cudaStream_t, int&);                          \
    template void launch_qoi<T>(const DevLevel<T>&, int, const long long*, const double*, const DevProblem&,      \
                                cudaStream_t, int&);                                                             \
    template void launch_pack<T>(const DevLevel<T>&, T*, bool, cudaStream_t);                               \
    template void launch_pack_batch<T>(const PackJob<T>*, void* const*, int, int, bool, cudaStream_t);         \
    template void launch_resid<T>(const DevLevel<T>&, const DevProblem&, double*, double*, int, double*,         \
                                  cudaStream_t);

MGMC_INSTANTIATE(float)
MGMC_INSTANTIATE(double)

}  // namespace mgmc
