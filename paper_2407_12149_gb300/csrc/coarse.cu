// coarse.cu -- the V-cycle below and including grid `top` in one CTA (Alg. 1
// recursion for the small grids, ending in the exact coarsest Cholesky sample
// of Sec. 3.5).
//
// The state theta_l, the dense right-hand side fdense_l and the operator
// coefficients of every grid l <= top live in shared memory for the whole
// kernel (padded (n+2)^d blocks with a zero ghost ring), staged once at the
// start.  Each phase (a colour of a sweep, a low-rank step, a restriction, a
// prolongation) is separated by one CTA barrier, so the grids that are too
// small to fill the GPU cost barriers and shared-memory latency rather than
// memory round trips.  The per-site arithmetic is that of stencil.cuh in the
// same order of operations.
#include "kernels.cuh"
#include "tma.cuh"

namespace mgmc {

namespace {

template <int DIM>
__device__ __forceinline__ int sidx(int S, int i, int j, int k)
{
    return DIM == 3 ? ((k + 1) * S + (j + 1)) * S + (i + 1) : (j + 1) * S + (i + 1);
}

template <int DIM>
__device__ __forceinline__ int soff(int o, int S)
{
    int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = DIM == 3 ? o / 9 - 1 : 0;
    return dx + S * (dy + S * dz);
}

// a(l, l + o) from the staged coefficient blocks CS (slot t at CS + t * SZ)
template <int DIM, typename T>
__device__ __forceinline__ T coef_s(const T* CS, int SZ, int ls, int S, int o)
{
    constexpr int C = Offsets<DIM>::C;
    constexpr int NS = Offsets<DIM>::NS;
    if (o > C) return CS[(o - C) * SZ + ls];
    return CS[(NS - 1 - o - C) * SZ + ls + soff<DIM>(o, S)];
}

template <int DIM>
__device__ __forceinline__ double upd_s(const DevLevel<double>& L, const double* X, const double* F,
                                        const double* CS, int SZ, int ls, int S, double z)
{
    if (L.fine) {
        double aii = CS[ls];
        double w = L.woff;
        double acc = 0.0;
        acc += sqrt(aii) * z;
        if (DIM == 3) acc += w * X[ls - S * S];
        acc += w * X[ls - S];
        acc += w * X[ls - 1];
        acc += w * X[ls + 1];
        acc += w * X[ls + S];
        if (DIM == 3) acc += w * X[ls + S * S];
        return acc / aii;
    }
    constexpr int NS = Offsets<DIM>::NS;
    constexpr int C = Offsets<DIM>::C;
    double aii = CS[ls];
    double acc = F[ls];
    acc += sqrt(aii) * z;
#pragma unroll
    for (int o = 0; o < NS; ++o) {
        if (o == C) continue;
        acc -= coef_s<DIM>(CS, SZ, ls, S, o) * X[ls + soff<DIM>(o, S)];
    }
    return acc / aii;
}

template <int DIM>
__device__ __forceinline__ float upd_s(const DevLevel<float>& L, const float* X, const float* F,
                                       const float* CS, int SZ, int ls, int S, float z)
{
    float xi = X[ls];
    if (L.fine) {
        float c = CS[ls];
        float w = L.woff;
        float lap = (xi - X[ls - S]) + (xi - X[ls - 1]) + (xi - X[ls + 1]) + (xi - X[ls + S]);
        if (DIM == 3) lap += (xi - X[ls - S * S]) + (xi - X[ls + S * S]);
        float aii = fmaf(2.0f * DIM, w, c);
        float Ax = fmaf(c, xi, w * lap);
        float ia, sa;
        inv_and_sqrt(aii, ia, sa);
        float rhs = 0.0f + sa * z;
        return xi + (rhs - Ax) * ia;
    }
    constexpr int NS = Offsets<DIM>::NS;
    constexpr int C = Offsets<DIM>::C;
    float s = CS[ls];
    float lap = 0.0f, offsum = 0.0f;
#pragma unroll
    for (int o = 0; o < NS; ++o) {
        if (o == C) continue;
        float a = coef_s<DIM>(CS, SZ, ls, S, o);
        lap = fmaf(a, X[ls + soff<DIM>(o, S)] - xi, lap);
        offsum += a;
    }
    float aii = s - offsum;
    float Ax = fmaf(s, xi, lap);
    float ia, sa;
    inv_and_sqrt(aii, ia, sa);
    float rhs = F[ls] + sa * z;
    return xi + (rhs - Ax) * ia;
}

template <int DIM>
__device__ __forceinline__ double Ax_s(const DevLevel<double>& L, const double* X, const double* CS, int SZ, int ls,
                                       int S)
{
    if (L.fine) {
        double w = -L.woff;
        double acc = 0.0;
        if (DIM == 3) acc += w * X[ls - S * S];
        acc += w * X[ls - S];
        acc += w * X[ls - 1];
        acc += CS[ls] * X[ls];
        acc += w * X[ls + 1];
        acc += w * X[ls + S];
        if (DIM == 3) acc += w * X[ls + S * S];
        return acc;
    }
    constexpr int NS = Offsets<DIM>::NS;
    constexpr int C = Offsets<DIM>::C;
    double acc = 0.0;
#pragma unroll
    for (int o = 0; o < NS; ++o) {
        double a = (o == C) ? CS[ls] : coef_s<DIM>(CS, SZ, ls, S, o);
        acc += a * X[ls + soff<DIM>(o, S)];
    }
    return acc;
}

template <int DIM>
__device__ __forceinline__ float Ax_s(const DevLevel<float>& L, const float* X, const float* CS, int SZ, int ls,
                                      int S)
{
    float xi = X[ls];
    if (L.fine) {
        float lap = (xi - X[ls - S]) + (xi - X[ls - 1]) + (xi - X[ls + 1]) + (xi - X[ls + S]);
        if (DIM == 3) lap += (xi - X[ls - S * S]) + (xi - X[ls + S * S]);
        return fmaf(CS[ls], xi, L.woff * lap);
    }
    constexpr int NS = Offsets<DIM>::NS;
    constexpr int C = Offsets<DIM>::C;
    float lap = 0.0f;
#pragma unroll
    for (int o = 0; o < NS; ++o) {
        if (o == C) continue;
        lap = fmaf(coef_s<DIM>(CS, SZ, ls, S, o), X[ls + soff<DIM>(o, S)] - xi, lap);
    }
    return fmaf(CS[ls], xi, lap);
}

// One sweep: first every normal of the sweep is drawn in one parallel phase
// into Z (index 2 * pair + member, pair = the Philox counter word c0), then the
// colours run as short stencil phases.
template <typename T, int DIM>
__device__ void s_sweep(const DevLevel<T>& L, const CycleState& cs, T* X, const T* F, const T* CS, T* Z, int dir,
                        unsigned slot)
{
    // colour orders (0, 3, 2, 1) and (0, 6, 5, 3, 4, 2, 1, 7) as packed nibbles (no local-memory table)
    auto seq = [](int i) { return (int)(((DIM == 2 ? 0x1230u : 0x71243560u) >> (4 * i)) & 0xFu); };
    constexpr int NCOL = DIM == 2 ? 4 : 8;
    const int n = L.n, S = n + 2;
    const int SZ = DIM == 3 ? S * S * S : S * S;
    const int nq = (n + 3) >> 2;
    const int nblocks = nq * n * (DIM == 3 ? n : 1);
    if (cs.noise) {
        // one block per 4-site group of a row: Z[4 b .. 4 b + 3] = the even columns' pair,
        // then the odd columns' pair
        const uint4 ctr = noise_counter(cs, 0u, 0u, L.level, slot);
        const unsigned k0 = (unsigned)cs.seed, k1 = (unsigned)(cs.seed >> 32);
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
            T a0, a1, b0, b1;
            draw_quad_ctr<T>(ctr, (unsigned)b, k0, k1, a0, a1, b0, b1);
            Z[4 * b] = a0;
            Z[4 * b + 1] = a1;
            Z[4 * b + 2] = b0;
            Z[4 * b + 3] = b1;
        }
        __syncthreads();
    }
    for (int ci = 0; ci < NCOL; ++ci) {
        const int c = seq(dir == 0 ? ci : NCOL - 1 - ci);
        const int px = c & 1, py = (c >> 1) & 1, pz = (c >> 2) & 1;
        const int ny = (n - py + 1) >> 1;
        const int nz = DIM == 3 ? (n - pz + 1) >> 1 : 1;
        const int items = nq * ny * nz;
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int q = it % nq;
            const int r = it / nq;
            const int j = 2 * (r % ny) + py;
            const int k = DIM == 3 ? 2 * (r / ny) + pz : 0;
            const int i0 = 4 * q + px;
            if (i0 >= n) continue;
            const bool has1 = i0 + 2 < n;
            T z0 = T(0), z1 = T(0);
            if (cs.noise) {
                const int blk = (int)(((long long)k * n + j) * nq + q);
                z0 = Z[4 * blk + 2 * px];
                z1 = Z[4 * blk + 2 * px + 1];
            }
            const int ls = sidx<DIM>(S, i0, j, k);
            X[ls] = upd_s<DIM>(L, X, F, CS, SZ, ls, S, z0);
            if (has1) X[ls + 2] = upd_s<DIM>(L, X, F, CS, SZ, ls + 2, S, z1);
        }
        __syncthreads();
    }
}

// theta' = theta*_s - G (B^T theta*_s - d - L_Gamma z') (dir >= 0); with want_dnext
// also d_{l-1} = d_l - B^T theta' = d_l - z + (B^T G) v.  Sites are shared-memory
// indices; G is applied in the path precision.
template <typename T>
__device__ void s_lowrank(const DevLevel<T>& L, const DevProblem& P, const CycleState& cs, T* X, int dir,
                          unsigned slot, bool want_dnext)
{
    __shared__ double z[kMaxObs];
    __shared__ double zp[kMaxObs];
    __shared__ double v[kMaxObs];
    const int m = P.m;
    if (m == 0) return;
    const bool noise = dir >= 0 && cs.noise;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        double acc = 0.0;
        for (int t = L.bcol_ptr[k]; t < L.bcol_ptr[k + 1]; ++t) acc += L.bcol_w[t] * (double)X[L.bcol_ss[t]];
        z[k] = acc;
        zp[k] = noise ? lowrank_normal<T>(cs, L.level, slot, k) : 0.0;
        if (P.gamma_diag) v[k] = acc - L.d[k] - (noise ? P.LG[k * m + k] * zp[k] : 0.0);
    }
    __syncthreads();
    if (!P.gamma_diag) {
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            double lz = 0.0;
            if (noise)
                for (int t = 0; t <= k; ++t) lz += P.LG[k * m + t] * zp[t];
            v[k] = z[k] - L.d[k] - lz;
        }
        __syncthreads();
    }
    if (dir >= 0) {
        const int rows = L.g_rows[dir];
        const T* G = L.gT[dir];
        for (int r = threadIdx.x; r < rows; r += blockDim.x) {
            T acc = T(0);
            for (int kk = 0; kk < m; ++kk) acc += G[(long long)r * m + kk] * (T)v[kk];
            const int s = L.g_ss[dir][r];
            X[s] = X[s] - acc;
        }
    }
    if (want_dnext) {
        // forward direction only (the restriction step after the pre-smoothing)
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            double acc = 0.0;
            if (dir >= 0)
                for (int t = 0; t < m; ++t) acc += L.BtG[k * m + t] * v[t];
            L.dnext[k] = L.d[k] - z[k] + acc;
        }
    }
    __syncthreads();
}

template <typename T, int DIM>
__device__ void s_restrict(const DevLevel<T>& Fl, const T* XF, const T* FF, const T* CSF, const DevLevel<T>& Cl,
                           T* FC)
{
    const int nf = Fl.n, Sf = nf + 2, nc = Cl.n, Sc = nc + 2;
    const int SZ = DIM == 3 ? Sf * Sf * Sf : Sf * Sf;
    const int N = nc * nc * (DIM == 3 ? nc : 1);
    for (int s = threadIdx.x; s < N; s += blockDim.x) {
        const int I = s % nc, J = (s / nc) % nc, K = DIM == 3 ? s / (nc * nc) : 0;
        T acc = T(0);
        for (int pz = 0; pz < (DIM == 3 ? 3 : 1); ++pz)
            for (int py = 0; py < 3; ++py)
                for (int px = 0; px < 3; ++px) {
                    const int fi = 2 * I + px, fj = 2 * J + py, fk = DIM == 3 ? 2 * K + pz : 0;
                    const int ls = sidx<DIM>(Sf, fi, fj, fk);
                    const T wgt = (T)(pw(px - 1) * pw(py - 1) * (DIM == 3 ? pw(pz - 1) : 1.0));
                    const T r = FF[ls] - Ax_s<DIM>(Fl, XF, CSF, SZ, ls, Sf);
                    acc += wgt * r;
                }
        FC[sidx<DIM>(Sc, I, J, K)] = acc;
    }
    __syncthreads();
}

template <typename T, int DIM>
__device__ void s_prolong(const DevLevel<T>& Cl, const T* XC, const DevLevel<T>& Fl, T* XF)
{
    const int nf = Fl.n, Sf = nf + 2, Sc = Cl.n + 2;
    const int N = nf * nf * (DIM == 3 ? nf : 1);
    for (int s = threadIdx.x; s < N; s += blockDim.x) {
        const int fi = s % nf, fj = (s / nf) % nf, fk = DIM == 3 ? s / (nf * nf) : 0;
        int cx[2], cy[2], cz[2], nx, ny, nz;
        T wx[2], wy[2], wz[2];
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
        T acc = T(0);
        for (int c = 0; c < nz; ++c)
            for (int b = 0; b < ny; ++b)
                for (int a = 0; a < nx; ++a)
                    acc += wz[c] * wy[b] * wx[a] * XC[sidx<DIM>(Sc, cx[a], cy[b], DIM == 3 ? cz[c] : 0)];
        const int ls = sidx<DIM>(Sf, fi, fj, fk);
        XF[ls] = XF[ls] + acc;
    }
    __syncthreads();
}

template <typename T, int DIM>
__device__ void s_coarsest(const DevLevel<T>& L, const DevProblem& P, const CycleState& cs, T* X, const T* F,
                           const double* chol, const double* Ls, int n0)
{
    __shared__ double r[MGMC_MAX_COARSEST];
    const int n = L.n, S = n + 2;
    for (int s = threadIdx.x; s < n0; s += blockDim.x) {
        const int i = s % n, j = (s / n) % n, k = DIM == 3 ? s / (n * n) : 0;
        r[s] = (double)F[sidx<DIM>(S, i, j, k)];
    }
    __syncthreads();
    __shared__ double g[kMaxObs];   // Gamma^-1 d_0
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
    if (n0 <= kCoarsestWarp) {
        // one warp, lane t holding r_t, the factor staged in shared memory (Ls): the same
        // operations in the same order as the CTA-wide solves below, without CTA barriers
        if (threadIdx.x < 32) {
            const int t = threadIdx.x;
            double rt = t < n0 ? r[t] : 0.0;
            for (int i = 0; i < n0; ++i) {
                const double ri = __shfl_sync(0xffffffffu, rt, i) / Ls[i * n0 + i];
                if (t == i)
                    rt = ri;
                else if (t > i && t < n0)
                    rt -= Ls[t * n0 + i] * ri;
            }
            if (cs.noise && t < n0) {
                double z0, z1;
                draw_pair<double>(cs, (unsigned)(t >> 1), 2u, 0, 0u, z0, z1);
                rt += (t & 1) ? z1 : z0;
            }
            for (int i = n0 - 1; i >= 0; --i) {
                const double xi = __shfl_sync(0xffffffffu, rt, i) / Ls[i * n0 + i];
                if (t == i)
                    rt = xi;
                else if (t < i)
                    rt -= Ls[i * n0 + t] * xi;
            }
            if (t < n0) r[t] = rt;
        }
        __syncthreads();
    } else {
        for (int i = 0; i < n0; ++i) {
            if (threadIdx.x == 0) r[i] = r[i] / chol[(long long)i * n0 + i];
            __syncthreads();
            const double yi = r[i];
            for (int t = i + 1 + threadIdx.x; t < n0; t += blockDim.x) r[t] -= chol[(long long)t * n0 + i] * yi;
            __syncthreads();
        }
        if (cs.noise) {
            for (int s = threadIdx.x; s < n0; s += blockDim.x) {
                double z0, z1;
                draw_pair<double>(cs, (unsigned)(s >> 1), 2u, 0, 0u, z0, z1);
                r[s] += (s & 1) ? z1 : z0;
            }
        }
        __syncthreads();
        for (int i = n0 - 1; i >= 0; --i) {
            if (threadIdx.x == 0) r[i] = r[i] / chol[(long long)i * n0 + i];
            __syncthreads();
            const double xi = r[i];
            for (int t = threadIdx.x; t < i; t += blockDim.x) r[t] -= chol[(long long)i * n0 + t] * xi;
            __syncthreads();
        }
    }
    for (int s = threadIdx.x; s < n0; s += blockDim.x) {
        const int i = s % n, j = (s / n) % n, k = DIM == 3 ? s / (n * n) : 0;
        X[sidx<DIM>(S, i, j, k)] = (T)r[s];
    }
    __syncthreads();
}

template <int DIM>
constexpr int coarse_threads()
{
    return DIM == 2 ? 1024 : 512;
}

}  // namespace

// Shared-memory elements of grids 0..top: state, right-hand side and
// coefficient blocks (1 coefficient block for the 5/7-point finest grid,
// (3^d + 1)/2 for a Galerkin grid), plus the normals of one sweep of grid top.
long long coarse_smem_elems(int dim, const int* n_of_level, int top, bool top_is_fd_finest)
{
    long long tot = 0;
    for (int l = 0; l <= top; ++l) {
        long long S = n_of_level[l] + 2;
        int ncoef = (l == top && top_is_fd_finest) ? 1 : (dim == 2 ? 5 : 14);
        tot += (2 + ncoef) * (dim == 3 ? S * S * S : S * S);
    }
    // normals of one sweep of the largest grid: 2 per Philox pair
    long long n = n_of_level[top], nq = (n + 3) / 4;
    tot += 4 * nq * n * (dim == 3 ? n : 1);
    // the coarsest grid's Cholesky factor when one warp solves with it (doubles, at
    // most two elements each, plus alignment)
    long long n0 = n_of_level[0];
    n0 = dim == 3 ? n0 * n0 * n0 : n0 * n0;
    if (n0 <= kCoarsestWarp) tot += 2 * n0 * n0 + 2;
    return tot;
}

// 8-byte words of a trivially copyable descriptor, all threads of the CTA
template <typename D>
__device__ __forceinline__ void copy_words(D* dst, const D* src)
{
    static_assert(sizeof(D) % 8 == 0, "descriptors are copied as 8-byte words");
    const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
    unsigned long long* d = reinterpret_cast<unsigned long long*>(dst);
    for (int w = threadIdx.x; w < (int)(sizeof(D) / 8); w += blockDim.x) d[w] = s[w];
}

template <typename T, int DIM>
__device__ __forceinline__ void coarse_body(const DevLevel<T>* __restrict__ levels, int top, int is_finest,
                                            const DevProblem& Pg, const double* chol, int n0, int nu1, int nu2,
                                            unsigned char* smem_raw)
{
    // the grids' descriptors and the problem in shared memory, and the offset of every
    // grid's block: the phases below read them at shared-memory latency
    __shared__ __align__(16) DevLevel<T> lv[kCoarseMaxLevels];
    __shared__ __align__(16) DevProblem P;
    __shared__ int blk_off[kCoarseMaxLevels];
    for (int l = 0; l <= top; ++l) copy_words(&lv[l], &levels[l]);
    copy_words(&P, &Pg);
    __syncthreads();
    auto grid_sz = [&](int l) {
        const int S = lv[l].n + 2;
        return DIM == 3 ? S * S * S : S * S;
    };
    auto nblocks = [&](int l) { return 2 + (lv[l].fine ? 1 : (DIM == 2 ? 5 : 14)); };
    if (threadIdx.x == 0) {
        int o = 0;
        for (int l = 0; l <= top; ++l) {
            blk_off[l] = o;
            o += nblocks(l) * grid_sz(l);
        }
    }
    __syncthreads();
    // the layout must fit the launch's dynamic shared memory: a mismatch between the
    // host's sizing and this layout is reported (status bit), never run
    {
        unsigned dsz;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsz));
        const long long nt = lv[top].n;
        long long need = (long long)blk_off[top] + (long long)nblocks(top) * grid_sz(top) +
                         4LL * ((nt + 3) / 4) * nt * (DIM == 3 ? nt : 1);
        if (n0 <= kCoarsestWarp) need += 2LL * n0 * n0 + 2;
        if (need * (long long)sizeof(T) > (long long)dsz) {
            if (threadIdx.x == 0) atomicOr(&Pg.cs->status, kStatusLayout);
            return;
        }
    }
    T* base = reinterpret_cast<T*>(smem_raw);
    // block layout per grid: X, F, coefficient slots (in that order)
    auto blk = [&](int l, int which) -> T* { return base + blk_off[l] + which * grid_sz(l); };
    // zero everything, then stage the coefficients of every grid and the top grid's
    // right-hand side (and the chain state when the top grid is the finest)
    T* Z = blk(top, nblocks(top));   // normals of one sweep
    {
        const long long tot = (long long)(Z - base);
        for (long long i = threadIdx.x; i < tot; i += blockDim.x) base[i] = T(0);
    }
    __syncthreads();
    for (int l = 0; l <= top; ++l) {
        const DevLevel<T>& L = lv[l];
        const int n = L.n, S = n + 2;
        const int sz = DIM == 3 ? S * S * S : S * S;
        const int nco = L.fine ? 1 : (DIM == 2 ? 5 : 14);
        T* CS = blk(l, 2);
        for (int s = threadIdx.x; s < sz; s += blockDim.x) {
            const int i = s % S - 1, j = (s / S) % S - 1, k = DIM == 3 ? s / (S * S) - 1 : 0;
            const long long e = site_offset(DIM, L.pitch, L.plane, L.base, i, j, k);
            if (L.fine) {
                CS[s] = L.diag[e];
            } else {
                for (int t = 0; t < nco; ++t) CS[t * sz + s] = L.coef[(long long)t * L.alloc + e];
            }
        }
    }
    // the coarsest grid's Cholesky factor, for the one-warp solves
    double* Ls = nullptr;
    if (n0 <= kCoarsestWarp) {
        const int nt = lv[top].n;
        const int zsz = 4 * ((nt + 3) / 4) * nt * (DIM == 3 ? nt : 1);
        Ls = reinterpret_cast<double*>(smem_align_up<8>(reinterpret_cast<unsigned char*>(Z + zsz)));
        for (int i = threadIdx.x; i < n0 * n0; i += blockDim.x) Ls[i] = chol[i];
    }
    // the descriptors and operators above never change after set-up; the top grid's
    // right-hand side and state (and the cycle state) come from the preceding launches
    pdl_wait();
    {
        const DevLevel<T>& L = lv[top];
        const int n = L.n, S = n + 2;
        const int N = n * n * (DIM == 3 ? n : 1);
        for (int s = threadIdx.x; s < N; s += blockDim.x) {
            const int i = s % n, j = (s / n) % n, k = DIM == 3 ? s / (n * n) : 0;
            const long long e = site_offset(DIM, L.pitch, L.plane, L.base, i, j, k);
            const int ls = sidx<DIM>(S, i, j, k);
            if (is_finest) blk(top, 0)[ls] = L.x[e];
            if (L.f) blk(top, 1)[ls] = L.f[e];
        }
    }
    __syncthreads();
    const CycleState cs = *P.cs;
    for (int l = top; l >= 1; --l) {
        const DevLevel<T>& L = lv[l];
        T* X = blk(l, 0);
        T* F = blk(l, 1);
        const T* CS = blk(l, 2);
        for (int s = 0; s < nu1; ++s) {
            s_sweep<T, DIM>(L, cs, X, F, CS, Z, 0, (unsigned)(2 * s));
            s_lowrank<T>(L, P, cs, X, 0, (unsigned)(2 * s), s == nu1 - 1);
        }
        if (nu1 == 0) s_lowrank<T>(L, P, cs, X, -1, 0u, true);
        s_restrict<T, DIM>(L, X, F, CS, lv[l - 1], blk(l - 1, 1));
    }
    s_coarsest<T, DIM>(lv[0], P, cs, blk(0, 0), blk(0, 1), chol, Ls, n0);
    for (int l = 1; l <= top; ++l) {
        const DevLevel<T>& L = lv[l];
        T* X = blk(l, 0);
        const T* F = blk(l, 1);
        const T* CS = blk(l, 2);
        s_prolong<T, DIM>(lv[l - 1], blk(l - 1, 0), L, X);
        for (int s = 0; s < nu2; ++s) {
            s_sweep<T, DIM>(L, cs, X, F, CS, Z, 1, (unsigned)(2 * s + 1));
            s_lowrank<T>(L, P, cs, X, 1, (unsigned)(2 * s + 1), false);
        }
    }
    // the top grid's final state goes back to global memory
    {
        const DevLevel<T>& L = lv[top];
        const T* X = blk(top, 0);
        const int n = L.n, S = n + 2;
        const int N = n * n * (DIM == 3 ? n : 1);
        for (int s = threadIdx.x; s < N; s += blockDim.x) {
            const int i = s % n, j = (s / n) % n, k = DIM == 3 ? s / (n * n) : 0;
            L.x[site_offset(DIM, L.pitch, L.plane, L.base, i, j, k)] = X[sidx<DIM>(S, i, j, k)];
        }
    }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(coarse_threads<DIM>())
    k_coarse_cycle(const DevLevel<T>* __restrict__ levels, int top, int is_finest, DevProblem P, const double* chol,
                   int n0, int nu1, int nu2)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    coarse_body<T, DIM>(levels, top, is_finest, P, chol, n0, nu1, nu2, smem_raw);
}

// Batched: one CTA per chain (2D).  The same instantiation serves few chains
// (1024 threads, latency) and many chains (256 threads, several chains per SM);
// the thread count never changes the arithmetic.
constexpr int kCoarseBatchMaxThreads = 1024;

template <typename T>
__global__ void __launch_bounds__(kCoarseBatchMaxThreads) k_coarse_cycle_batch(const CoarseJob<T>* __restrict__ jobs)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_launch_dependents();
    const CoarseJob<T>& J = jobs[blockIdx.x];   // static table; coarse_body waits for the predecessor
    coarse_body<T, 2>(J.levels, J.top, J.is_finest, *J.P, J.chol, J.n0, 1, 1, smem_raw);
}

// F^T theta of every chain's finest grid, then step += 1, cycle += 1 (one CTA per chain)
template <typename T>
__global__ void k_qoi_batch(const QoiJob<T>* __restrict__ jobs)
{
    __shared__ double part[256];
    pdl_launch_dependents();
    // the QoI sites and weights never change: the first kQoiPre of each thread are loaded
    // before the wait on the preceding launch, the state after it (same summation order)
    constexpr int kQoiPre = 8;
    const QoiJob<T> J = jobs[blockIdx.x];
    long long site[kQoiPre];
    double w[kQoiPre];
#pragma unroll
    for (int r = 0; r < kQoiPre; ++r) {
        const int t = threadIdx.x + r * blockDim.x;
        site[r] = t < J.n_qoi ? J.q_site[t] : 0;
        w[r] = t < J.n_qoi ? J.q_w[t] : 0.0;
    }
    pdl_wait();
    double acc = 0.0;
#pragma unroll
    for (int r = 0; r < kQoiPre; ++r)
        if (threadIdx.x + r * blockDim.x < J.n_qoi) acc += w[r] * (double)J.x[site[r]];
    for (int t = threadIdx.x + kQoiPre * blockDim.x; t < J.n_qoi; t += blockDim.x)
        acc += J.q_w[t] * (double)J.x[J.q_site[t]];
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) part[threadIdx.x] += part[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        CycleState* cs = J.cs;
        double q = part[0];
        if (cs->qoi) cs->qoi[cs->step] = q;
        if (!isfinite(q)) atomicOr(&cs->status, kStatusNumeric);
        cs->step += 1;
        cs->cycle += 1;
    }
}

__global__ void k_set_cycle_batch(CycleState* const* cs, int n, unsigned long long seed, unsigned long long cycle,
                                  int noise, double* qoi, long long n_steps)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    CycleState* s = cs[c];
    s->seed = seed;
    s->cycle = cycle;
    s->chain = (unsigned)c;
    s->noise = noise;
    s->qoi = qoi ? qoi + (long long)c * n_steps : nullptr;
    s->step = 0;
}

template <typename T>
cudaError_t coarse_prepare_batch(size_t smem_bytes)
{
    return cudaFuncSetAttribute(k_coarse_cycle_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

template <typename T>
void launch_coarse_batch(const CoarseJob<T>* jobs, int n, int threads, size_t smem_bytes, cudaStream_t st,
                         int& launches)
{
    launch_pdl(k_coarse_cycle_batch<T>, dim3((unsigned)n), dim3((unsigned)threads), smem_bytes, st, jobs);
    ++launches;
}

template <typename T>
void launch_qoi_batch(const QoiJob<T>* jobs, int n, cudaStream_t st, int& launches)
{
    launch_pdl(k_qoi_batch<T>, dim3((unsigned)n), dim3(256), 0, st, jobs);
    ++launches;
}

void launch_set_cycle_batch(CycleState* const* cs, int n, unsigned long long seed, unsigned long long cycle, int noise,
                            double* qoi, long long n_steps, cudaStream_t st)
{
    k_set_cycle_batch<<<(n + 127) / 128, 128, 0, st>>>(cs, n, seed, cycle, noise, qoi, n_steps);
}

template cudaError_t coarse_prepare_batch<float>(size_t);
template cudaError_t coarse_prepare_batch<double>(size_t);
template void launch_coarse_batch<float>(const CoarseJob<float>*, int, int, size_t, cudaStream_t, int&);
template void launch_coarse_batch<double>(const CoarseJob<double>*, int, int, size_t, cudaStream_t, int&);
template void launch_qoi_batch<float>(const QoiJob<float>*, int, cudaStream_t, int&);
template void launch_qoi_batch<double>(const QoiJob<double>*, int, cudaStream_t, int&);

template <typename T>
cudaError_t coarse_prepare(int dim, size_t smem_bytes)
{
    if (dim == 2)
        return cudaFuncSetAttribute(k_coarse_cycle<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    return cudaFuncSetAttribute(k_coarse_cycle<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

template <typename T>
void launch_coarse(const DevLevel<T>* levels_dev, int dim, int top, bool is_finest, const DevProblem& P,
                   const double* chol, int n0, int nu1, int nu2, size_t smem_bytes, cudaStream_t st, int& launches)
{
    if (dim == 2)
        k_coarse_cycle<T, 2><<<1, coarse_threads<2>(), smem_bytes, st>>>(levels_dev, top, is_finest ? 1 : 0, P, chol,
                                                                          n0, nu1, nu2);
    else
        k_coarse_cycle<T, 3><<<1, coarse_threads<3>(), smem_bytes, st>>>(levels_dev, top, is_finest ? 1 : 0, P, chol,
                                                                          n0, nu1, nu2);
    ++launches;
}

template cudaError_t coarse_prepare<float>(int, size_t);
template cudaError_t coarse_prepare<double>(int, size_t);
template void launch_coarse<float>(const DevLevel<float>*, int, int, bool, const DevProblem&, const double*, int, int,
                                   int, size_t, cudaStream_t, int&);
template void launch_coarse<double>(const DevLevel<double>*, int, int, bool, const DevProblem&, const double*, int,
                                    int, int, size_t, cudaStream_t, int&);

}  // namespace mgmc
