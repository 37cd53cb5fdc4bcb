// tile2d.cu -- fused shared-memory tile kernels of the 2D V-cycle (nu1 = nu2 = 1).
//
// One CTA owns a TX x TY tile of a grid level and stages the state, the
// operator and the dense right-hand side of the tile plus a halo in shared
// memory (16-byte vector loads of whole padded rows).
//
// Forward kernel (Alg. 1 pre-smoothing + restriction):
//   all colours of one forward Gibbs sweep in shared memory -- colour p is
//   updated on the tile grown by NC + 1 - p rings, so the sites near the tile edge
//   see exactly the values a global sweep would give them (the counter-based
//   Philox noise makes the recomputed halo bitwise identical to the
//   neighbour's own update) -- then the residual r = fdense - A theta*_s on
//   the tile plus one ring and its restriction P^T r onto the coarse sites of
//   the tile.  theta*_s goes to the second state buffer; the products
//   w_t theta*_s(site_t) of the observation entries inside the tile go to
//   zparts for the low-rank kernel.
// Backward kernel (prolongation + post-smoothing):
//   theta' + P psi_{l-1} on the tile plus NC rings, then the colours in
//   reverse order, shrinking by one ring per colour.
//
// 5-point finest grid: NC = 2 (red, black); 9-point Galerkin grids: NC = 4
// parity colours in the order (0,0), (1,1), (0,1), (1,0).  The per-site
// arithmetic is the same as in stencil.cuh (FP64 plain form, FP32 correction
// form) in the same order of operations.
#include "kernels.cuh"
#include "tile2d.cuh"

namespace mgmc {

namespace {

template <typename T>
struct Vec;
template <>
struct Vec<float> {
    using type = float4;
    static constexpr int N = 4;
};
template <>
struct Vec<double> {
    using type = double2;
    static constexpr int N = 2;
};

constexpr int kTileThreads = 256;

}  // namespace

template <typename T, bool FINE, bool BWD>
struct TileGeom {
    static constexpr int TX = TileShape<T, FINE>::TX;
    static constexpr int TY = TileShape<T, FINE>::TY;
    static constexpr int VEC = Vec<T>::N;
    static constexpr int NC = FINE ? 2 : 4;
    // rings of state staged around the tile: backward NC (the last colour ends on
    // the tile); forward NC + 2 (the last colour must also cover ring 2 because the
    // residual on ring 1 -- the coarse patches reach one site past the tile -- reads it)
    static constexpr int R = BWD ? NC : NC + 2;
    static constexpr int RX = (R + VEC - 1) / VEC * VEC;  // the same along x, in whole vectors
    static constexpr int SX = TX + 2 * RX;
    static constexpr int SY = TY + 2 * R;
    static constexpr int NCOEF = FINE ? 1 : 5;
    static constexpr int NFLD = 1 + NCOEF + (FINE ? 0 : 1);  // x, coefficients, fdense
    static constexpr int RES = (TX + 1) * (TY + 1);         // residual on tile + high ring
    static constexpr int PX = SX / 2 + 2;                   // coarse psi tile (backward)
    static constexpr int PY = SY / 2 + 2;
    static constexpr size_t smem_bytes()
    {
        return sizeof(T) * ((size_t)NFLD * SX * SY + (BWD ? (size_t)PX * PY : (size_t)RES));
    }
};

namespace {

// dst[ly * SX + lx] = src at interior (gx0 + lx, gy0 + ly); zero outside the padded array
template <typename T, int SX, int SY>
__device__ __forceinline__ void stage(T* dst, const T* src, const DevLevel<T>& L, int gx0, int gy0)
{
    using V = typename Vec<T>::type;
    constexpr int VN = Vec<T>::N;
    constexpr int NV = SX / VN;
    for (int idx = threadIdx.x; idx < NV * SY; idx += blockDim.x) {
        int vx = idx % NV, ly = idx / NV;
        int i = gx0 + vx * VN, j = gy0 + ly;
        V v;
        if (src && j >= -1 && j <= L.n && i + 4 >= 0 && i + 4 + VN <= L.pitch) {
            long long e = (long long)L.pitch * (j + 1) + (i + 4);
            v = *reinterpret_cast<const V*>(src + e);
        } else {
            v = V{};
        }
        *reinterpret_cast<V*>(dst + ly * SX + vx * VN) = v;
    }
}

// --- per-site arithmetic on the staged tile (same operations as stencil.cuh) ---
template <int SX>
__device__ __forceinline__ double upd_fine(const double* X, const double* C0, int l, double w, double z)
{
    double aii = C0[l];
    double acc = 0.0;
    acc += sqrt(aii) * z;
    acc += w * X[l - SX];
    acc += w * X[l - 1];
    acc += w * X[l + 1];
    acc += w * X[l + SX];
    return acc / aii;
}

template <int SX>
__device__ __forceinline__ float upd_fine(const float* X, const float* C0, int l, float w, float z)
{
    float xi = X[l];
    float c = C0[l];
    float lap = (xi - X[l - SX]) + (xi - X[l - 1]) + (xi - X[l + 1]) + (xi - X[l + SX]);
    float aii = fmaf(4.0f, w, c);
    float Ax = fmaf(c, xi, w * lap);
    float ia, sa;
    inv_and_sqrt(aii, ia, sa);
    float rhs = 0.0f + sa * z;
    return xi + (rhs - Ax) * ia;
}

// 9-point offsets o = (dx+1) + 3 (dy+1); a(l, l+o) for o > 4 is coefficient slot o-4 of
// site l, for o < 4 it is slot 4-o of the neighbour l + off(o)
template <int SX>
__device__ __forceinline__ int noff(int o)
{
    return (o % 3 - 1) + (o / 3 - 1) * SX;
}

template <int SX, int SXY>
__device__ __forceinline__ double coef9(const double* Cf, int l, int o)
{
    return o > 4 ? Cf[(o - 4) * SXY + l] : Cf[(4 - o) * SXY + l + noff<SX>(o)];
}
template <int SX, int SXY>
__device__ __forceinline__ float coef9(const float* Cf, int l, int o)
{
    return o > 4 ? Cf[(o - 4) * SXY + l] : Cf[(4 - o) * SXY + l + noff<SX>(o)];
}

template <int SX, int SXY>
__device__ __forceinline__ double upd_9(const double* X, const double* Cf, const double* F, int l, double z)
{
    double aii = Cf[l];
    double acc = F[l];
    acc += sqrt(aii) * z;
#pragma unroll
    for (int o = 0; o < 9; ++o) {
        if (o == 4) continue;
        acc -= coef9<SX, SXY>(Cf, l, o) * X[l + noff<SX>(o)];
    }
    return acc / aii;
}

template <int SX, int SXY>
__device__ __forceinline__ float upd_9(const float* X, const float* Cf, const float* F, int l, float z)
{
    float xi = X[l];
    float s = Cf[l];
    float lap = 0.0f, offsum = 0.0f;
#pragma unroll
    for (int o = 0; o < 9; ++o) {
        if (o == 4) continue;
        float a = coef9<SX, SXY>(Cf, l, o);
        lap = fmaf(a, X[l + noff<SX>(o)] - xi, lap);
        offsum += a;
    }
    float aii = s - offsum;
    float Ax = fmaf(s, xi, lap);
    float ia, sa;
    inv_and_sqrt(aii, ia, sa);
    float rhs = F[l] + sa * z;
    return xi + (rhs - Ax) * ia;
}

template <int SX>
__device__ __forceinline__ double Ax_fine(const double* X, const double* C0, int l, double woff)
{
    double w = -woff;
    double acc = 0.0;
    acc += w * X[l - SX];
    acc += w * X[l - 1];
    acc += C0[l] * X[l];
    acc += w * X[l + 1];
    acc += w * X[l + SX];
    return acc;
}
template <int SX>
__device__ __forceinline__ float Ax_fine(const float* X, const float* C0, int l, float woff)
{
    float xi = X[l];
    float lap = (xi - X[l - SX]) + (xi - X[l - 1]) + (xi - X[l + 1]) + (xi - X[l + SX]);
    return fmaf(C0[l], xi, woff * lap);
}
template <int SX, int SXY>
__device__ __forceinline__ double Ax_9(const double* X, const double* Cf, int l)
{
    double acc = 0.0;
#pragma unroll
    for (int o = 0; o < 9; ++o) {
        double a = o == 4 ? Cf[l] : coef9<SX, SXY>(Cf, l, o);
        acc += a * X[l + noff<SX>(o)];
    }
    return acc;
}
template <int SX, int SXY>
__device__ __forceinline__ float Ax_9(const float* X, const float* Cf, int l)
{
    float xi = X[l];
    float lap = 0.0f;
#pragma unroll
    for (int o = 0; o < 9; ++o) {
        if (o == 4) continue;
        lap = fmaf(coef9<SX, SXY>(Cf, l, o), X[l + noff<SX>(o)] - xi, lap);
    }
    return fmaf(Cf[l], xi, lap);
}

__host__ __device__ constexpr int colour_seq4(int p) { return p == 0 ? 0 : p == 1 ? 3 : p == 2 ? 2 : 1; }

// One colour of a sweep on the staged tile.  Work items are (4-site group, row)
// pairs of a fixed, compile-time count, so that index arithmetic uses constant
// divisors; items outside the grid or the phase's ring are predicated off.
// Site (i, j) lives at l = (j - gy0) * SX + (i - gx0).
template <typename T, bool FINE, bool BWD, typename G, int P>
__device__ __forceinline__ void tile_phase(const DevLevel<T>& L, const CycleState& cs, T* X, const T* Cf,
                                           const T* F, int x0, int y0, unsigned slot)
{
    constexpr int SX = G::SX;
    constexpr int SXY = G::SX * G::SY;
    constexpr int colour = FINE ? (BWD ? 1 - P : P) : (BWD ? colour_seq4(G::NC - 1 - P) : colour_seq4(P));
    constexpr int rp = BWD ? G::NC - 1 - P : G::NC + 1 - P;
    // groups gq = GQ0 .. (TX + rp - 1) / 4 relative to x0 / 4, GQ0 = floor(-rp / 4)
    constexpr int GQ0 = -((rp + 3) / 4);
    constexpr int NQ = (G::TX + rp - 1) / 4 - GQ0 + 1;
    // rows dy = dy0 + step * t, t < NR
    constexpr int PY = (colour >> 1) & 1;
    constexpr int DY0 = FINE ? -rp : -rp + ((PY + rp) & 1);
    constexpr int STEP = FINE ? 1 : 2;
    constexpr int NR = (G::TY + rp - DY0 + STEP - 1) / STEP;
    const int n = L.n;
    const int nq = (n + 3) >> 2;
    const int q0 = x0 >> 2;
    for (int it = threadIdx.x; it < NQ * NR; it += kTileThreads) {
        const int gq = it % NQ + GQ0;
        const int dy = DY0 + STEP * (it / NQ);
        const int j = y0 + dy;
        const int px = FINE ? ((j + colour) & 1) : (colour & 1);
        const int dx0 = 4 * gq + px, dx1 = dx0 + 2;
        const int i0 = x0 + dx0, i1 = x0 + dx1;
        const bool rowok = j >= 0 && j < n && dy < G::TY + rp;
        const bool v0 = rowok && dx0 >= -rp && dx0 < G::TX + rp && i0 >= 0 && i0 < n;
        const bool v1 = rowok && dx1 >= -rp && dx1 < G::TX + rp && i1 >= 0 && i1 < n;
        if (!v0 && !v1) continue;
        T z0 = T(0), z1 = T(0);
        if (cs.noise) {
            unsigned pair = (unsigned)(((long long)j * nq + (q0 + gq)) * 2 + px);
            draw_pair<T>(cs, pair, 0u, L.level, slot, z0, z1);
        }
        const int l0 = (dy + G::R) * SX + (dx0 + G::RX);
        if (FINE) {
            if (v0) X[l0] = upd_fine<SX>(X, Cf, l0, L.woff, z0);
            if (v1) X[l0 + 2] = upd_fine<SX>(X, Cf, l0 + 2, L.woff, z1);
        } else {
            if (v0) X[l0] = upd_9<SX, SXY>(X, Cf, F, l0, z0);
            if (v1) X[l0 + 2] = upd_9<SX, SXY>(X, Cf, F, l0 + 2, z1);
        }
    }
}

// All colours of one sweep, one CTA barrier after each.
template <typename T, bool FINE, bool BWD, typename G, int P = 0>
__device__ __forceinline__ void tile_sweep(const DevLevel<T>& L, const CycleState& cs, T* X, const T* Cf,
                                           const T* F, int x0, int y0, unsigned slot)
{
    if constexpr (P < G::NC) {
        tile_phase<T, FINE, BWD, G, P>(L, cs, X, Cf, F, x0, y0, slot);
        __syncthreads();
        tile_sweep<T, FINE, BWD, G, P + 1>(L, cs, X, Cf, F, x0, y0, slot);
    }
}

// w_t * theta(site_t) of the observation entries inside the tile
template <typename T, typename G>
__device__ __forceinline__ void tile_zparts(const DevLevel<T>& L, const T* X, int tile)
{
    if (!L.tile_ptr) return;
    const int t0 = L.tile_ptr[tile], t1 = L.tile_ptr[tile + 1];
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
        int loc = L.tile_loc[t];
        int lx = (loc & 0xFFFF) + G::RX, ly = (loc >> 16) + G::R;
        int ent = L.tile_ent[t];
        L.zparts[ent] = L.bcol_w[ent] * (double)X[ly * G::SX + lx];
    }
}

template <typename T, typename G>
__device__ __forceinline__ void tile_store(const DevLevel<T>& L, T* dst, const T* X, int x0, int y0)
{
    using V = typename Vec<T>::type;
    constexpr int VN = Vec<T>::N;
    constexpr int NV = G::TX / VN;
    for (int idx = threadIdx.x; idx < NV * G::TY; idx += blockDim.x) {
        int vx = idx % NV, ty = idx / NV;
        int i = x0 + vx * VN, j = y0 + ty;
        if (j >= L.n || i + 4 + VN > L.pitch) continue;
        long long e = (long long)L.pitch * (j + 1) + (i + 4);
        *reinterpret_cast<V*>(dst + e) = *reinterpret_cast<const V*>(X + (ty + G::R) * G::SX + vx * VN + G::RX);
    }
}

}  // namespace

template <typename T, bool FINE>
__device__ __forceinline__ void tile_fwd_body(const DevLevel<T>& L, const DevLevel<T>& C, const DevProblem& P,
                                              int x_zero, int bx, int by, unsigned char* smem_raw)
{
    using G = TileGeom<T, FINE, false>;
    T* X = reinterpret_cast<T*>(smem_raw);
    T* Cf = X + G::SX * G::SY;
    T* F = Cf + G::NCOEF * G::SX * G::SY;
    T* Rr = F + (FINE ? 0 : G::SX * G::SY);
    const CycleState cs = *P.cs;
    const int x0 = bx * G::TX, y0 = by * G::TY;
    const int gx0 = x0 - G::RX, gy0 = y0 - G::R;
    stage<T, G::SX, G::SY>(X, x_zero ? nullptr : L.x, L, gx0, gy0);
    if (FINE) {
        stage<T, G::SX, G::SY>(Cf, L.diag, L, gx0, gy0);
    } else {
        for (int t = 0; t < G::NCOEF; ++t)
            stage<T, G::SX, G::SY>(Cf + t * G::SX * G::SY, L.coef + (long long)t * L.alloc, L, gx0, gy0);
        stage<T, G::SX, G::SY>(F, L.f, L, gx0, gy0);
    }
    __syncthreads();
    tile_sweep<T, FINE, false, G>(L, cs, X, Cf, F, x0, y0, 0u);
    const int tile = by * L.ntx + bx;
    tile_zparts<T, G>(L, X, tile);
    // residual r = fdense - A theta*_s on [x0, x0+TX] x [y0, y0+TY] (inside the grid)
    constexpr int RW = G::TX + 1;
    for (int idx = threadIdx.x; idx < G::RES; idx += blockDim.x) {
        int rx = idx % RW, ry = idx / RW;
        int i = x0 + rx, j = y0 + ry;
        T r = T(0);
        if (i < L.n && j < L.n) {
            int l = (j - gy0) * G::SX + (i - gx0);
            if (FINE)
                r = T(0) - Ax_fine<G::SX>(X, Cf, l, L.woff);
            else
                r = F[l] - Ax_9<G::SX, G::SX * G::SY>(X, Cf, l);
        }
        Rr[idx] = r;
    }
    __syncthreads();
    // restriction onto the coarse sites of the tile: f_c = sum_p w(p) r(2I + p)
    const int I0 = x0 >> 1, J0 = y0 >> 1;
    for (int idx = threadIdx.x; idx < (G::TX / 2) * (G::TY / 2); idx += blockDim.x) {
        int I = I0 + idx % (G::TX / 2), J = J0 + idx / (G::TX / 2);
        if (I >= C.n || J >= C.n) continue;
        T acc = T(0);
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) {
                T wgt = (T)(pw(a - 1) * pw(b - 1));
                acc += wgt * Rr[(2 * J + b - y0) * RW + (2 * I + a - x0)];
            }
        C.f[site_offset(2, C.pitch, C.plane, C.base, I, J, 0)] = acc;
    }
    tile_store<T, G>(L, L.x2, X, x0, y0);
}

template <typename T, bool FINE>
__device__ __forceinline__ void tile_bwd_body(const DevLevel<T>& L, const DevLevel<T>& C, const DevProblem& P, int bx,
                                              int by, unsigned char* smem_raw)
{
    using G = TileGeom<T, FINE, true>;
    T* X = reinterpret_cast<T*>(smem_raw);
    T* Cf = X + G::SX * G::SY;
    T* F = Cf + G::NCOEF * G::SX * G::SY;
    T* Ps = F + (FINE ? 0 : G::SX * G::SY);
    const CycleState cs = *P.cs;
    const int x0 = bx * G::TX, y0 = by * G::TY;
    const int gx0 = x0 - G::RX, gy0 = y0 - G::R;
    stage<T, G::SX, G::SY>(X, L.x2, L, gx0, gy0);
    if (FINE) {
        stage<T, G::SX, G::SY>(Cf, L.diag, L, gx0, gy0);
    } else {
        for (int t = 0; t < G::NCOEF; ++t)
            stage<T, G::SX, G::SY>(Cf + t * G::SX * G::SY, L.coef + (long long)t * L.alloc, L, gx0, gy0);
        stage<T, G::SX, G::SY>(F, L.f, L, gx0, gy0);
    }
    // coarse psi around the tile (ghost indices -1 and n_c read the zero ring)
    const int Ilo = (gx0 >> 1) - 1, Jlo = (gy0 >> 1) - 1;
    for (int idx = threadIdx.x; idx < G::PX * G::PY; idx += blockDim.x) {
        int I = Ilo + idx % G::PX, J = Jlo + idx / G::PX;
        T v = T(0);
        if (J >= -1 && J <= C.n && I + 4 >= 0 && I + 4 < C.pitch) v = C.x[(long long)C.pitch * (J + 1) + (I + 4)];
        Ps[idx] = v;
    }
    __syncthreads();
    // theta' + P psi on the staged region (interior sites only)
    for (int idx = threadIdx.x; idx < G::SX * G::SY; idx += blockDim.x) {
        int lx = idx % G::SX, ly = idx / G::SX;
        int i = gx0 + lx, j = gy0 + ly;
        if (i < 0 || i >= L.n || j < 0 || j >= L.n) continue;
        int cx[2], cy[2], nx, ny;
        T wx[2], wy[2];
        if (i & 1) { cx[0] = (i - 1) >> 1; wx[0] = T(1); nx = 1; }
        else { cx[0] = (i >> 1) - 1; cx[1] = i >> 1; wx[0] = wx[1] = T(0.5); nx = 2; }
        if (j & 1) { cy[0] = (j - 1) >> 1; wy[0] = T(1); ny = 1; }
        else { cy[0] = (j >> 1) - 1; cy[1] = j >> 1; wy[0] = wy[1] = T(0.5); ny = 2; }
        T acc = T(0);
        for (int b = 0; b < ny; ++b)
            for (int a = 0; a < nx; ++a)
                acc += T(1) * wy[b] * wx[a] * Ps[(cy[b] - Jlo) * G::PX + (cx[a] - Ilo)];
        X[idx] = X[idx] + acc;
    }
    __syncthreads();
    tile_sweep<T, FINE, true, G>(L, cs, X, Cf, F, x0, y0, 1u);
    tile_zparts<T, G>(L, X, by * L.ntx + bx);
    tile_store<T, G>(L, L.x, X, x0, y0);
}

template <typename T, bool FINE>
__global__ void __launch_bounds__(kTileThreads) k_tile_fwd(DevLevel<T> L, DevLevel<T> C, DevProblem P, int x_zero)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile_fwd_body<T, FINE>(L, C, P, x_zero, blockIdx.x, blockIdx.y, smem_raw);
}

template <typename T, bool FINE>
__global__ void __launch_bounds__(kTileThreads) k_tile_bwd(DevLevel<T> L, DevLevel<T> C, DevProblem P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile_bwd_body<T, FINE>(L, C, P, blockIdx.x, blockIdx.y, smem_raw);
}

// Batched forms: one launch covers the same grid depth of many chains.  Block b
// belongs to the job whose tile range [tile0, tile0 + ntiles) contains b.
template <typename T>
__device__ __forceinline__ int find_job(const TileJob<T>* jobs, int njobs, int b)
{
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].tile0 <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <typename T, bool FINE>
__global__ void __launch_bounds__(kTileThreads) k_tile_fwd_batch(const TileJob<T>* __restrict__ jobs, int njobs,
                                                                 int x_zero)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TileJob<T>& J = jobs[find_job(jobs, njobs, blockIdx.x)];
    const int t = blockIdx.x - J.tile0;
    tile_fwd_body<T, FINE>(*J.L, *J.C, *J.P, x_zero, t % J.L->ntx, t / J.L->ntx, smem_raw);
}

template <typename T, bool FINE>
__global__ void __launch_bounds__(kTileThreads) k_tile_bwd_batch(const TileJob<T>* __restrict__ jobs, int njobs)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TileJob<T>& J = jobs[find_job(jobs, njobs, blockIdx.x)];
    const int t = blockIdx.x - J.tile0;
    tile_bwd_body<T, FINE>(*J.L, *J.C, *J.P, t % J.L->ntx, t / J.L->ntx, smem_raw);
}

// Low-rank step after a fused sweep (Alg. 3 last line, see kernels.cu):
//   z = B^T theta*_s from zparts, v = z - d - L_Gamma z',
//   theta' = theta*_s - G v on the support of G;
// on the way down also f_{l-1} += H v (H = P^T A G) and
// d_{l-1} = d_l - B^T theta' = d_l - z + (B^T G) v.
template <typename T>
__device__ __forceinline__ void lowrank_fused_body(const DevLevel<T>& L, const DevLevel<T>& C, const DevProblem& P,
                                                   int down, int blk, int nblk)
{
    __shared__ double z[kMaxObs];
    __shared__ double zp[kMaxObs];
    __shared__ double v[kMaxObs];
    const CycleState cs = *P.cs;
    const int m = P.m;
    const int dir = down ? 0 : 1;
    const unsigned slot = down ? 0u : 1u;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        double acc = 0.0;
        for (int t = L.bcol_ptr[k]; t < L.bcol_ptr[k + 1]; ++t) acc += L.zparts[t];
        z[k] = acc;
        zp[k] = cs.noise ? lowrank_normal<T>(cs, L.level, slot, k) : 0.0;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        double lz = 0.0;
        if (cs.noise) {
            if (P.gamma_diag)
                lz = P.LG[k * m + k] * zp[k];
            else
                for (int t = 0; t <= k; ++t) lz += P.LG[k * m + t] * zp[t];
        }
        v[k] = z[k] - L.d[k] - lz;
    }
    __syncthreads();
    T* x = down ? L.x2 : L.x;
    const int stride = nblk * blockDim.x;
    const T* Gm = L.gT[dir];
    for (int r = blk * blockDim.x + threadIdx.x; r < L.g_rows[dir]; r += stride) {
        T acc = T(0);
        for (int k = 0; k < m; ++k) acc += Gm[(long long)r * m + k] * (T)v[k];
        long long s = L.g_site[dir][r];
        x[s] = x[s] - acc;
    }
    if (!down) return;
    for (int r = blk * blockDim.x + threadIdx.x; r < L.h_rows; r += stride) {
        T acc = T(0);
        for (int k = 0; k < m; ++k) acc += L.hT[(long long)r * m + k] * (T)v[k];
        long long s = L.h_site[r];
        C.f[s] = C.f[s] + acc;
    }
    if (blk == 0)
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            double acc = 0.0;
            for (int t = 0; t < m; ++t) acc += L.BtG[k * m + t] * v[t];
            L.dnext[k] = L.d[k] - z[k] + acc;
        }
}

template <typename T>
__global__ void k_lowrank_fused(DevLevel<T> L, DevLevel<T> C, DevProblem P, int down)
{
    lowrank_fused_body<T>(L, C, P, down, blockIdx.x, gridDim.x);
}

// batched: job j owns blocks [block0, block0 + nblocks)
template <typename T>
__global__ void k_lowrank_fused_batch(const LowrankJob<T>* __restrict__ jobs, int njobs, int down)
{
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].block0 <= (int)blockIdx.x)
            lo = mid;
        else
            hi = mid - 1;
    }
    const LowrankJob<T>& J = jobs[lo];
    lowrank_fused_body<T>(*J.L, *J.C, *J.P, down, blockIdx.x - J.block0, J.nblocks);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int lowrank_blocks(int rows)
{
    int blocks = (rows + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 64) blocks = 64;
    return blocks;
}
template <typename T, bool FINE>
static void tile_dims(const DevLevel<T>& L, dim3& grid)
{
    grid = dim3((unsigned)((L.n + TileShape<T, FINE>::TX - 1) / TileShape<T, FINE>::TX),
                (unsigned)((L.n + TileShape<T, FINE>::TY - 1) / TileShape<T, FINE>::TY));
}

template <typename T>
cudaError_t tile_prepare()
{
    cudaError_t e = cudaSuccess;
    e = cudaFuncSetAttribute(k_tile_fwd<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TileGeom<T, true, false>::smem_bytes());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tile_fwd<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TileGeom<T, false, false>::smem_bytes());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tile_bwd<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TileGeom<T, true, true>::smem_bytes());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_tile_bwd<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TileGeom<T, false, true>::smem_bytes());
}

template <typename T>
void launch_tile_fwd(const DevLevel<T>& L, const DevLevel<T>& C, const DevProblem& P, bool x_zero, cudaStream_t st,
                     int& launches)
{
    dim3 grid;
    if (L.fine) {
        tile_dims<T, true>(L, grid);
        k_tile_fwd<T, true><<<grid, kTileThreads, TileGeom<T, true, false>::smem_bytes(), st>>>(L, C, P, x_zero);
    } else {
        tile_dims<T, false>(L, grid);
        k_tile_fwd<T, false><<<grid, kTileThreads, TileGeom<T, false, false>::smem_bytes(), st>>>(L, C, P, x_zero);
    }
    ++launches;
}

template <typename T>
void launch_tile_bwd(const DevLevel<T>& L, const DevLevel<T>& C, const DevProblem& P, cudaStream_t st, int& launches)
{
    dim3 grid;
    if (L.fine) {
        tile_dims<T, true>(L, grid);
        k_tile_bwd<T, true><<<grid, kTileThreads, TileGeom<T, true, true>::smem_bytes(), st>>>(L, C, P);
    } else {
        tile_dims<T, false>(L, grid);
        k_tile_bwd<T, false><<<grid, kTileThreads, TileGeom<T, false, true>::smem_bytes(), st>>>(L, C, P);
    }
    ++launches;
}

template <typename T>
void launch_lowrank_fused(const DevLevel<T>& L, const DevLevel<T>& C, const DevProblem& P, bool down, cudaStream_t st,
                          int& launches)
{
    if (P.m == 0) return;
    int rows = L.g_rows[down ? 0 : 1];
    if (down && L.h_rows > rows) rows = L.h_rows;
    k_lowrank_fused<T><<<lowrank_blocks(rows), 256, 0, st>>>(L, C, P, down ? 1 : 0);
    ++launches;
}

template <typename T>
cudaError_t tile_prepare_batch()
{
    cudaError_t e = cudaFuncSetAttribute(k_tile_fwd_batch<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TileGeom<T, true, false>::smem_bytes());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tile_fwd_batch<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TileGeom<T, false, false>::smem_bytes());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tile_bwd_batch<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TileGeom<T, true, true>::smem_bytes());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_tile_bwd_batch<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TileGeom<T, false, true>::smem_bytes());
}

template <typename T>
void launch_tile_batch(const TileJob<T>* jobs, int njobs, int nblocks, bool fine, bool bwd, bool x_zero,
                       cudaStream_t st, int& launches)
{
    if (nblocks <= 0) return;
    if (!bwd) {
        if (fine)
            k_tile_fwd_batch<T, true><<<nblocks, kTileThreads, TileGeom<T, true, false>::smem_bytes(), st>>>(
                jobs, njobs, x_zero ? 1 : 0);
        else
            k_tile_fwd_batch<T, false><<<nblocks, kTileThreads, TileGeom<T, false, false>::smem_bytes(), st>>>(
                jobs, njobs, x_zero ? 1 : 0);
    } else {
        if (fine)
            k_tile_bwd_batch<T, true><<<nblocks, kTileThreads, TileGeom<T, true, true>::smem_bytes(), st>>>(jobs,
                                                                                                             njobs);
        else
            k_tile_bwd_batch<T, false><<<nblocks, kTileThreads, TileGeom<T, false, true>::smem_bytes(), st>>>(jobs,
                                                                                                               njobs);
    }
    ++launches;
}

template <typename T>
void launch_lowrank_batch(const LowrankJob<T>* jobs, int njobs, int nblocks, bool down, cudaStream_t st,
                          int& launches)
{
    if (nblocks <= 0) return;
    k_lowrank_fused_batch<T><<<nblocks, 256, 0, st>>>(jobs, njobs, down ? 1 : 0);
    ++launches;
}

#define MGMC_TILE_INST(T)                                                                                        \
    template cudaError_t tile_prepare<T>();                                                                       \
    template void launch_tile_fwd<T>(const DevLevel<T>&, const DevLevel<T>&, const DevProblem&, bool, cudaStream_t, \
                                     int&);                                                                       \
    template void launch_tile_bwd<T>(const DevLevel<T>&, const DevLevel<T>&, const DevProblem&, cudaStream_t, int&); \
    template void launch_lowrank_fused<T>(const DevLevel<T>&, const DevLevel<T>&, const DevProblem&, bool,         \
                                          cudaStream_t, int&);                                                     \
    template cudaError_t tile_prepare_batch<T>();                                                                 \
    template void launch_tile_batch<T>(const TileJob<T>*, int, int, bool, bool, bool, cudaStream_t, int&);         \
    template void launch_lowrank_batch<T>(const LowrankJob<T>*, int, int, bool, cudaStream_t, int&);

MGMC_TILE_INST(float)
MGMC_TILE_INST(double)

}  // namespace mgmc
