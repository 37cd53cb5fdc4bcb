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
#include <cstring>
#include <mutex>

#include "kernels.cuh"
#include "tile2d.cuh"
#include "tma.cuh"

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

}  // namespace

template <typename T, bool FINE, bool BWD>
struct TileGeom {
    static constexpr int TX = TileShape<T, FINE>::TX;
    static constexpr int TY = TileShape<T, FINE>::TY;
    static constexpr int VEC = Vec<T>::N;
    static constexpr int NC = FINE ? 2 : 4;
    // threads per CTA (256 measured faster than 384 on the 5-point grid, whose two
    // colour phases have ~650 work items per tile; ~250 per phase on 9-point grids)
    static constexpr int NT = 256;
    // rings of state staged around the tile: backward NC (the last colour ends on
    // the tile); forward NC + 2 (the last colour must also cover ring 2 because the
    // residual on ring 1 -- the coarse patches reach one site past the tile -- reads it)
    static constexpr int R = BWD ? NC : NC + 2;
    static constexpr int RX = (R + VEC - 1) / VEC * VEC;  // the same along x, in whole 16-byte vectors
    static constexpr int SW = TX + 2 * RX;                  // staged columns
    // row pitch in shared memory (= the TMA box width): the FP32 9-point tiles get 4
    // or 12 extra columns so that the float4 rows of neighbouring work items (two
    // grid rows apart) fall on different bank groups
    static constexpr int PAD = (sizeof(T) == 4 && !FINE) ? (BWD ? 12 : 4) : 0;
    static constexpr int SX = SW + PAD;
    static constexpr int SY = TY + 2 * R;
    static constexpr int NCOEF = FINE ? 1 : 5;
    static constexpr int NFLD = 1 + NCOEF + (FINE ? 0 : 1);  // x, coefficients, fdense
    // field stride in elements: every field (a TMA destination) starts on 128 bytes
    static constexpr int FS = (SX * SY * (int)sizeof(T) + 127) / 128 * 128 / (int)sizeof(T);
    static constexpr int RW4 = TX + 4;                      // FP32 residual row: whole 4-site groups
    static constexpr int RES = sizeof(T) == 4 ? RW4 * (TY + 1) : (TX + 1) * (TY + 1);  // residual on tile + high ring
    // backward: coarse psi around the tile, columns cx0 .. cx0 + PX - 1 with
    // cx0 = (gx0 >> 1) - 1; the box starts POFF columns earlier, on a 16-byte boundary
    // (cx0 + 4 = x0 / 2 + 3 - RX / 2 and x0 / 2 is a multiple of the vector width)
    static constexpr int PX = SW / 2 + 2;
    static constexpr int PY = SY / 2 + 2;
    static constexpr int POFF = ((3 - RX / 2) % VEC + VEC) % VEC;
    static constexpr int PXA = (PX + POFF + VEC - 1) / VEC * VEC;
    static constexpr int PSZ = (PXA * PY * (int)sizeof(T) + 127) / 128 * 128 / (int)sizeof(T);
    // tensor maps: x source, coefficient fields, fdense (9-point), psi (backward)
    static constexpr int NMAP = NFLD + (BWD ? 1 : 0);
    // stage buffers: two on the 5-point grid (tile k + 1 is copied while tile k is
    // computed), one on the 9-point grids (7 fields; three CTAs per SM overlap instead)
    static constexpr int NSTAGE = FINE ? 2 : 1;
    static constexpr int STAGE = NFLD * FS + (BWD ? PSZ : 0);  // elements per stage buffer
    // single-stage backward kernels keep a second state buffer: the next tile's state
    // is copied into it while the current tile still stores its own
    static constexpr int XALT = (NSTAGE == 1 && BWD) ? FS : 0;
    static constexpr unsigned BOX_BYTES = (unsigned)(SX * SY * sizeof(T));
    static constexpr unsigned PSI_BYTES = (unsigned)(PXA * PY * sizeof(T));
    // TMA: box corners x0 - RX + 4 and (psi) x0 / 2 - RX / 2 + 3 - POFF must be multiples of
    // 16 bytes, box rows (SX, PXA) whole 16-byte vectors, boxes at most 256 per side
    static_assert(RX % VEC == 0 && TX % (2 * VEC) == 0 && SX % VEC == 0 && PXA % VEC == 0, "TMA alignment");
    static_assert(SX <= 256 && SY <= 256 && PXA <= 256 && PY <= 256, "TMA box size");
};

namespace {

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

// --- FP32 group updates: the two same-colour sites (components q = px, px + 2) of
// the 4-site group whose first site is at the 16-byte aligned index lb.  Whole
// float4 rows are read; the one column outside the group (lb - 1 for px = 0,
// lb + 4 for px = 1) is read as a scalar.  The group's float4 is written back
// whole: its other two sites have the other colour and are not written by any
// thread in this phase.  Same operations, in the same order, as upd_fine / upd_9.
__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void sts4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
template <int SX>
__device__ __forceinline__ void pair_fine(float* X, const float* C0, int lb, int px, float w, float z0, float z1,
                                          bool v0, bool v1)
{
    const float4 r0 = lds4(X + lb), ru = lds4(X + lb - SX), rd = lds4(X + lb + SX), c = lds4(C0 + lb);
    const float e = X[px ? lb + 4 : lb - 1];
    const bool o = px != 0;
    // site a: component px; site b: component px + 2
    const float xa = o ? r0.y : r0.x, xb = o ? r0.w : r0.z;
    const float na = fine_site(xa, o ? ru.y : ru.x, o ? r0.x : e, o ? r0.z : r0.y, o ? rd.y : rd.x,
                               o ? c.y : c.x, w, z0);
    const float nb = fine_site(xb, o ? ru.w : ru.z, o ? r0.z : r0.y, o ? e : r0.w, o ? rd.w : rd.z,
                               o ? c.w : c.z, w, z1);
    float4 r = r0;
    if (o) {
        if (v0) r.y = na;
        if (v1) r.w = nb;
    } else {
        if (v0) r.x = na;
        if (v1) r.z = nb;
    }
    sts4(X + lb, r);
}

template <int PX, int SX, int SXY>
__device__ __forceinline__ void pair_9(float* X, const float* Cf, const float* F, int lb, float z0, float z1, bool v0,
                                       bool v1)
{
    Rows9 r;
    r.xm = lds4(X + lb - SX);
    r.x0 = lds4(X + lb);
    r.xp = lds4(X + lb + SX);
    r.s0 = lds4(Cf + lb);
    r.c1 = lds4(Cf + SXY + lb);
    r.c2 = lds4(Cf + 2 * SXY + lb);
    r.c3 = lds4(Cf + 3 * SXY + lb);
    r.c4 = lds4(Cf + 4 * SXY + lb);
    r.c2m = lds4(Cf + 2 * SXY + lb - SX);
    r.c3m = lds4(Cf + 3 * SXY + lb - SX);
    r.c4m = lds4(Cf + 4 * SXY + lb - SX);
    r.f = lds4(F + lb);
    if (PX == 0) {
        r.exm = X[lb - SX - 1];
        r.ex0 = X[lb - 1];
        r.exp = X[lb + SX - 1];
        r.c1e = Cf[SXY + lb - 1];
        r.c4me = Cf[4 * SXY + lb - SX - 1];
        r.c2me = 0.f;
    } else {
        r.exm = X[lb - SX + 4];
        r.ex0 = X[lb + 4];
        r.exp = X[lb + SX + 4];
        r.c1e = 0.f;
        r.c4me = 0.f;
        r.c2me = Cf[2 * SXY + lb - SX + 4];
    }
    const float na = site9<PX>(r, z0);
    const float nb = site9<PX + 2>(r, z1);
    float4 o = r.x0;
    if (PX == 0) {
        if (v0) o.x = na;
        if (v1) o.z = nb;
    } else {
        if (v0) o.y = na;
        if (v1) o.w = nb;
    }
    sts4(X + lb, o);
}

// --- FP32 residual of 4 consecutive sites (components 0..3 of the group at lb):
// A theta in the same order of operations as Ax_fine / Ax_9.
template <int SX>
__device__ __forceinline__ float4 ax4_fine(const float* X, const float* C0, int lb, float w)
{
    const float4 r0 = lds4(X + lb), ru = lds4(X + lb - SX), rd = lds4(X + lb + SX), c = lds4(C0 + lb);
    const float el = X[lb - 1], er = X[lb + 4];
    auto one = [&](float xi, float up, float lf, float rt, float dn, float cc) {
        float lap = (xi - up) + (xi - lf) + (xi - rt) + (xi - dn);
        return fmaf(cc, xi, w * lap);
    };
    return make_float4(one(r0.x, ru.x, el, r0.y, rd.x, c.x), one(r0.y, ru.y, r0.x, r0.z, rd.y, c.y),
                       one(r0.z, ru.z, r0.y, r0.w, rd.z, c.z), one(r0.w, ru.w, r0.z, er, rd.w, c.w));
}

template <int SX, int SXY>
__device__ __forceinline__ float4 res4_9(const float* X, const float* Cf, const float* F, int lb)
{
    Rows9R R;
    Rows9& r = R.r;
    r.xm = lds4(X + lb - SX);
    r.x0 = lds4(X + lb);
    r.xp = lds4(X + lb + SX);
    r.s0 = lds4(Cf + lb);
    r.c1 = lds4(Cf + SXY + lb);
    r.c2 = lds4(Cf + 2 * SXY + lb);
    r.c3 = lds4(Cf + 3 * SXY + lb);
    r.c4 = lds4(Cf + 4 * SXY + lb);
    r.c2m = lds4(Cf + 2 * SXY + lb - SX);
    r.c3m = lds4(Cf + 3 * SXY + lb - SX);
    r.c4m = lds4(Cf + 4 * SXY + lb - SX);
    r.f = lds4(F + lb);
    r.exm = X[lb - SX - 1];
    r.ex0 = X[lb - 1];
    r.exp = X[lb + SX - 1];
    r.c1e = Cf[SXY + lb - 1];
    r.c4me = Cf[4 * SXY + lb - SX - 1];
    r.c2me = 0.f;
    R.xmr = X[lb - SX + 4];
    R.x0r = X[lb + 4];
    R.xpr = X[lb + SX + 4];
    R.c2mr = Cf[2 * SXY + lb - SX + 4];
    return make_float4(r.f.x - ax9q<0>(R), r.f.y - ax9q<1>(R), r.f.z - ax9q<2>(R), r.f.w - ax9q<3>(R));
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
    constexpr int SXY = G::FS;  // stride between the staged fields
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
    // counter words and key of this sweep's site noise, out of the item loop
    const uint4 ctr = noise_counter(cs, 0u, 0u, L.level, slot);
    const unsigned k0 = (unsigned)cs.seed, k1 = (unsigned)(cs.seed >> 32);
    const bool noise = cs.noise != 0;
    for (int it = threadIdx.x; it < NQ * NR; it += G::NT) {
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
        if (noise)  // the block of the group's row, this colour's half of it
            draw_half_ctr<T>(ctr, (unsigned)((long long)j * nq + (q0 + gq)), px, k0, k1, z0, z1);
        if constexpr (sizeof(T) == 4) {
            // FP32: whole 4-site groups as float4 rows of the staged tile
            const int lb = (dy + G::R) * SX + (4 * gq + G::RX);
            if constexpr (FINE)
                pair_fine<SX>((float*)X, (const float*)Cf, lb, px, (float)L.woff, (float)z0, (float)z1, v0, v1);
            else
                pair_9<colour & 1, SX, SXY>((float*)X, (const float*)Cf, (const float*)F, lb, (float)z0, (float)z1,
                                            v0, v1);
        } else {
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
// [first, last) of the tile's observation entries; loaded at the start of a tile so
// that the round trip overlaps the sweep
template <typename T>
__device__ __forceinline__ int2 tile_entries(const DevLevel<T>& L, int tile)
{
    return L.tile_ptr ? make_int2(L.tile_ptr[tile], L.tile_ptr[tile + 1]) : make_int2(0, 0);
}

template <typename T, typename G>
__device__ __forceinline__ void tile_zparts(const DevLevel<T>& L, const T* X, int2 range)
{
    for (int t = range.x + threadIdx.x; t < range.y; t += blockDim.x) {
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

// Forward tile (Alg. 1 pre-smoothing + restriction) on a staged stage buffer:
// X (state, zero-filled here when the sweep starts from psi = 0), Cf (operator
// fields), F (dense right-hand side, 9-point grids), Rr (residual scratch).
// fields_free() is called by every thread once Cf and F are no longer read (after the
// residual), so the next tile's copies can start while the restriction runs.
template <typename T, bool FINE, typename Hook>
__device__ __forceinline__ void tile_fwd_compute(const DevLevel<T>& L, const DevLevel<T>& C, const CycleState& cs,
                                                 int x_zero, int bx, int by, T* X, const T* Cf, const T* F, T* Rr,
                                                 Hook&& fields_free)
{
    using G = TileGeom<T, FINE, false>;
    const int x0 = bx * G::TX, y0 = by * G::TY;
    const int gx0 = x0 - G::RX, gy0 = y0 - G::R;
    const int2 zr = tile_entries(L, by * L.ntx + bx);
    if (x_zero) {
        for (int idx = threadIdx.x; idx < G::SX * G::SY; idx += G::NT) X[idx] = T(0);
        __syncthreads();
    }
    tile_sweep<T, FINE, false, G>(L, cs, X, Cf, F, x0, y0, 0u);
    // residual r = fdense - A theta*_s on [x0, x0+TX] x [y0, y0+TY] (inside the grid)
    const int I0 = x0 >> 1, J0 = y0 >> 1;
    if constexpr (sizeof(T) == 4) {
        // FP32: 4-site groups over [x0, x0 + TX + 3]; the columns past x0 + TX are not used
        constexpr int RW = G::RW4;
        constexpr int NGX = RW / 4;
        float* R4 = (float*)Rr;
        for (int idx = threadIdx.x; idx < NGX * (G::TY + 1); idx += G::NT) {
            const int gx = idx % NGX, ry = idx / NGX;
            const int i = x0 + 4 * gx, j = y0 + ry;
            const int lb = (ry + G::R) * G::SX + (4 * gx + G::RX);
            float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j < L.n && i < L.n) {
                if (FINE) {
                    const float4 a = ax4_fine<G::SX>((const float*)X, (const float*)Cf, lb, (float)L.woff);
                    r = make_float4(0.0f - a.x, 0.0f - a.y, 0.0f - a.z, 0.0f - a.w);
                } else {
                    r = res4_9<G::SX, G::FS>((const float*)X, (const float*)Cf, (const float*)F, lb);
                }
                if (i + 1 >= L.n) r.y = 0.f;
                if (i + 2 >= L.n) r.z = 0.f;
                if (i + 3 >= L.n) r.w = 0.f;
            }
            sts4(R4 + ry * RW + 4 * gx, r);
        }
        __syncthreads();
        fields_free();
        // restriction of two coarse sites per item: f_c = sum_p w(p) r(2I + p),
        // fine columns 2I .. 2I + 4 of three rows
        for (int idx = threadIdx.x; idx < (G::TX / 4) * (G::TY / 2); idx += G::NT) {
            const int I = I0 + 2 * (idx % (G::TX / 4)), J = J0 + idx / (G::TX / 4);
            if (I >= C.n || J >= C.n) continue;
            const int cb = (2 * J - y0) * RW + (2 * I - x0);
            float4 v[3];
            float e[3];
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                v[b] = lds4(R4 + cb + b * RW);
                e[b] = R4[cb + b * RW + 4];
            }
            float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const float wb = b == 1 ? 1.0f : 0.5f;
                acc0 += (0.5f * wb) * v[b].x;
                acc0 += (1.0f * wb) * v[b].y;
                acc0 += (0.5f * wb) * v[b].z;
                acc1 += (0.5f * wb) * v[b].z;
                acc1 += (1.0f * wb) * v[b].w;
                acc1 += (0.5f * wb) * e[b];
            }
            long long o = site_offset(2, C.pitch, C.plane, C.base, I, J, 0);
            // o is even (I, the padded base and the pitch are): both sites in one 8-byte store
            if (I + 1 < C.n)
                *reinterpret_cast<float2*>(C.f + o) = make_float2(acc0, acc1);
            else
                C.f[o] = (T)acc0;
        }
    } else {
        constexpr int RW = G::TX + 1;
        for (int idx = threadIdx.x; idx < G::RES; idx += G::NT) {
            int rx = idx % RW, ry = idx / RW;
            int i = x0 + rx, j = y0 + ry;
            T r = T(0);
            if (i < L.n && j < L.n) {
                int l = (j - gy0) * G::SX + (i - gx0);
                if (FINE)
                    r = T(0) - Ax_fine<G::SX>(X, Cf, l, L.woff);
                else
                    r = F[l] - Ax_9<G::SX, G::FS>(X, Cf, l);
            }
            Rr[idx] = r;
        }
        __syncthreads();
        fields_free();
        // restriction onto the coarse sites of the tile: f_c = sum_p w(p) r(2I + p)
        for (int idx = threadIdx.x; idx < (G::TX / 2) * (G::TY / 2); idx += G::NT) {
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
    }
    // w_t theta*_s at the tile's observation entries (theta*_s is still in X: the
    // residual and the restriction do not write it, and the next tile's copies that may
    // already be in flight do not target it)
    tile_zparts<T, G>(L, X, zr);
    tile_store<T, G>(L, L.x2, X, x0, y0);
}

// Backward tile (prolongation + Alg. 1 post-smoothing) on a staged stage buffer:
// X (theta*' of the forward pass), Cf, F, Ps (coarse psi box, origin POFF columns
// before cx0 = (gx0 >> 1) - 1, row cy0 = (gy0 >> 1) - 1).
// fields_free() is called by every thread once Cf, F and Ps are no longer read
// (after the sweep).
template <typename T, bool FINE, typename Hook>
__device__ __forceinline__ void tile_bwd_compute(const DevLevel<T>& L, const CycleState& cs, int bx, int by, T* X,
                                                 const T* Cf, const T* F, const T* Ps, Hook&& fields_free)
{
    using G = TileGeom<T, FINE, true>;
    const int x0 = bx * G::TX, y0 = by * G::TY;
    const int gx0 = x0 - G::RX, gy0 = y0 - G::R;
    const int Ilo = (gx0 >> 1) - 1 - G::POFF, Jlo = (gy0 >> 1) - 1;
    const int2 zr = tile_entries(L, by * L.ntx + bx);
    // theta' + P psi on the staged region (interior sites only)
    if constexpr (sizeof(T) == 4) {
        // FP32: one 4-site group (i = gx0 + 4v even) per item; fine site i + c takes
        // the coarse columns a - 1, a (c = 0), a (c = 1), a, a + 1 (c = 2), a + 1 (c = 3),
        // a = i / 2, i.e. Ps columns 2v, 2v + 1, 2v + 2; the same sums as below
        constexpr int NV = G::SW / 4;
        float* Xf = (float*)X;
        const float* Pf = (const float*)Ps;
        for (int idx = threadIdx.x; idx < NV * G::SY; idx += G::NT) {
            const int v = idx % NV, ly = idx / NV;
            const int i = gx0 + 4 * v, j = gy0 + ly;
            if (j < 0 || j >= L.n || i + 3 < 0 || i >= L.n) continue;
            // coarse rows: j odd -> (j - 1) / 2 (weight 1); j even -> j / 2 - 1, j / 2 (1/2 each)
            const int odd = j & 1;
            const int pr0 = odd ? ((ly - 1) >> 1) + 1 : (ly >> 1);
            const float wy = odd ? 1.0f : 0.5f;
            float p0[3], p1[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                p0[c] = Pf[pr0 * G::PXA + G::POFF + 2 * v + c];
                p1[c] = odd ? 0.f : Pf[(pr0 + 1) * G::PXA + G::POFF + 2 * v + c];
            }
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            a0 += 1.0f * wy * 0.5f * p0[0];
            a0 += 1.0f * wy * 0.5f * p0[1];
            a1 += 1.0f * wy * 1.0f * p0[1];
            a2 += 1.0f * wy * 0.5f * p0[1];
            a2 += 1.0f * wy * 0.5f * p0[2];
            a3 += 1.0f * wy * 1.0f * p0[2];
            if (!odd) {
                a0 += 1.0f * wy * 0.5f * p1[0];
                a0 += 1.0f * wy * 0.5f * p1[1];
                a1 += 1.0f * wy * 1.0f * p1[1];
                a2 += 1.0f * wy * 0.5f * p1[1];
                a2 += 1.0f * wy * 0.5f * p1[2];
                a3 += 1.0f * wy * 1.0f * p1[2];
            }
            float4 x = lds4(Xf + ly * G::SX + 4 * v);
            if (i >= 0) x.x = x.x + a0;
            if (i + 1 >= 0 && i + 1 < L.n) x.y = x.y + a1;
            if (i + 2 >= 0 && i + 2 < L.n) x.z = x.z + a2;
            if (i + 3 < L.n) x.w = x.w + a3;
            sts4(Xf + ly * G::SX + 4 * v, x);
        }
    } else {
        for (int idx = threadIdx.x; idx < G::SW * G::SY; idx += G::NT) {
            int lx = idx % G::SW, ly = idx / G::SW;
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
                    acc += T(1) * wy[b] * wx[a] * Ps[(cy[b] - Jlo) * G::PXA + (cx[a] - Ilo)];
            X[ly * G::SX + lx] = X[ly * G::SX + lx] + acc;
        }
    }
    __syncthreads();
    tile_sweep<T, FINE, true, G>(L, cs, X, Cf, F, x0, y0, 1u);
    fields_free();
    tile_zparts<T, G>(L, X, zr);
    tile_store<T, G>(L, L.x, X, x0, y0);
}


// TMA staging: each field of a stage is one 2D tiled bulk tensor copy of the
// padded array (tma.cuh), the box anchored at the staged region's corner in
// padded coordinates; the parts of a box outside the array are filled with
// zeros -- the ghost ring's value.  The copies of a stage complete on one mbarrier.

template <typename T>
__device__ __forceinline__ int job_first(const TileJob<T>& j) { return j.tile0; }
template <typename T>
__device__ __forceinline__ int job_first(const LowrankJob<T>& j) { return j.block0; }

// Batched launches cover the same grid depth of many chains.  Item b (a tile or a
// block) belongs to the job whose range [first, first + count) contains it: found
// by division when every job has `per` items, else by binary search.
template <typename Job>
__device__ __forceinline__ int find_job(const Job* jobs, int njobs, int per, int b)
{
    if (per > 0) return b / per;
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (job_first(jobs[mid]) <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// the job descriptor into shared memory, 8-byte words in parallel (one round trip)
template <typename Job>
__device__ __forceinline__ void load_job(Job& dst, const Job* src)
{
    static_assert(sizeof(Job) % 8 == 0, "job descriptors are copied as 8-byte words");
    const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
    unsigned long long* d = reinterpret_cast<unsigned long long*>(&dst);
    for (int w = threadIdx.x; w < (int)(sizeof(Job) / 8); w += blockDim.x) d[w] = s[w];
    __syncthreads();
}

constexpr int kHdrBytes = (int)((sizeof(TileJob<double>) + 127) / 128 * 128);
static_assert(sizeof(TileJob<float>) <= (size_t)kHdrBytes, "tile job header slot");

template <typename T, bool FINE, bool BWD>
constexpr size_t tile_smem_bytes()
{
    using G = TileGeom<T, FINE, BWD>;
    return 2 * (size_t)kHdrBytes + 128 +
           sizeof(T) * ((size_t)G::NSTAGE * G::STAGE + G::XALT + (BWD ? 0 : (size_t)G::RES));
}

// Persistent tile kernel of one grid depth of every chain.  Tile order: with
// cpj > 0 every chain owns cpj consecutive CTAs, which stride through its tiles
// in row order (the CTAs of a chain work on neighbouring tiles at the same time,
// so halo rows are read from L2, and each CTA loads one job descriptor); with
// cpj = 0 (more chains than CTAs) all CTAs stride through all tiles.  With two
// stage buffers the copies of tile k + 1 are issued before tile k is computed.
// A stage that does not arrive within 1 s sets the chain's status to 2
// (MGMC_ERR_TIMEOUT), waits (bounded) for the copies in flight and ends the CTA.
template <typename T, bool FINE, bool BWD>
__global__ void __launch_bounds__(TileGeom<T, FINE, BWD>::NT, 3)
    k_tile_batch(const TileJob<T>* __restrict__ jobs, const TileMaps* __restrict__ maps, int njobs, int per,
                 int ntiles, int cpj, int x_zero)
{
    using G = TileGeom<T, FINE, BWD>;
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    // TMA destinations start on 128-byte boundaries (the launch adds 128 bytes of slack)
    unsigned char* smem_raw = smem_align_up<128>(smem_dyn);
    // header slot s (computed, not an indexed array: that would live in local memory)
    auto hdr = [smem_raw](int s) { return reinterpret_cast<TileJob<T>*>(smem_raw + s * kHdrBytes); };
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + 2 * kHdrBytes);
    T* buf = reinterpret_cast<T*>(smem_raw + 2 * kHdrBytes + 128);
    T* Rr = buf + G::NSTAGE * G::STAGE + G::XALT;
    __shared__ CycleState cs_s[2];
    __shared__ int jid[2];

    pdl_launch_dependents();
    // tiles tb, tb + step, ... < te
    int tb, te, step;
    if (cpj > 0) {
        const int j = blockIdx.x / cpj;
        const int first = per > 0 ? j * per : jobs[j].tile0;
        tb = first + (int)(blockIdx.x % cpj);
        te = first + (per > 0 ? per : jobs[j].ntiles);
        step = cpj;
    } else {
        tb = blockIdx.x;
        te = ntiles;
        step = gridDim.x;
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar[0]);
        mbar_init(&bar[1]);
        fence_mbar_init();
        jid[0] = jid[1] = -1;
    }
    __syncthreads();
    // the TMA copies of tile t (header in slot hs) into stage buffer ds, its state into xd
    // (thread 0).  part 0: all fields; 1: the expected bytes of all and the operator
    // coefficients alone (they never change after set-up); 2: the rest (state, dense
    // right-hand side, coarse psi), which the preceding launches write.
    auto issue = [&](int t, int hs, int ds, T* xd, int part) {
        const TileJob<T>& J = *hdr(hs);
        const int lt = t - J.tile0;
        const int x0 = (lt % J.L.ntx) * G::TX, y0 = (lt / J.L.ntx) * G::TY;
        const int cx = x0 - G::RX + 4, cy = y0 - G::R + 1;  // padded coordinates of the box corner
        const CUtensorMap* M = maps[jid[hs]].m;
        T* b = buf + ds * G::STAGE;
        const bool loadx = BWD || !x_zero;
        if (part != 2) {
            const unsigned bytes =
                (unsigned)(G::NFLD - (loadx ? 0 : 1)) * G::BOX_BYTES + (BWD ? G::PSI_BYTES : 0u);
            mbar_expect_tx(&bar[ds], bytes);
            for (int f = 1; f <= G::NCOEF; ++f) tma_load_2d(b + f * G::FS, &M[f], cx, cy, &bar[ds]);
        }
        if (part == 1) return;
        if (loadx) tma_load_2d(xd, &M[0], cx, cy, &bar[ds]);
        for (int f = G::NCOEF + 1; f < G::NFLD; ++f) tma_load_2d(b + f * G::FS, &M[f], cx, cy, &bar[ds]);
        if (BWD) {
            const int gx0 = x0 - G::RX, gy0 = y0 - G::R;
            tma_load_2d(b + G::NFLD * G::FS, &M[G::NFLD], ((gx0 >> 1) - 1 - G::POFF) + 4, ((gy0 >> 1) - 1) + 1,
                        &bar[ds]);
        }
    };
    // a CTA of a per-chain group loads its job descriptor (static) and starts the copies
    // of its first tile's operator coefficients before the wait on the preceding launch;
    // the cycle state and the other fields follow it
    const int pre = (cpj > 0 && tb < te) ? (int)(blockIdx.x / cpj) : -1;
    if (pre >= 0) {
        load_job(*hdr(0), jobs + pre);
        if (threadIdx.x == 0) {
            jid[0] = pre;
            issue(tb, 0, 0, buf, 1);
        }
    }
    pdl_wait();
    if (tb >= te) return;
    if (pre >= 0) {
        if (threadIdx.x == 0) cs_s[0] = *hdr(0)->P.cs;
        __syncthreads();
    }

    // header and cycle state of tile t's chain into slot hs
    auto fetch = [&](int t, int hs) {
        const int j = find_job(jobs, njobs, per, t);
        if (jid[hs] == j) return;
        const bool other = jid[hs ^ 1] == j;
        __syncthreads();  // every thread has read jid[]
        if (other) {
            const unsigned long long* s = reinterpret_cast<const unsigned long long*>(hdr(hs ^ 1));
            unsigned long long* d = reinterpret_cast<unsigned long long*>(hdr(hs));
            for (int w = threadIdx.x; w < (int)(sizeof(TileJob<T>) / 8); w += G::NT) d[w] = s[w];
            if (threadIdx.x == 0) cs_s[hs] = cs_s[hs ^ 1];
            __syncthreads();
        } else {
            load_job(*hdr(hs), jobs + j);
            if (threadIdx.x == 0) cs_s[hs] = *hdr(hs)->P.cs;
        }
        if (threadIdx.x == 0) jid[hs] = j;
        __syncthreads();
    };
    // state buffer of the k-th tile: field 0 of its stage, or the second state buffer
    // for odd k of a single-stage backward kernel
    auto xbuf = [&](int k, int ds) { return (G::XALT && (k & 1)) ? buf + G::STAGE : buf + ds * G::STAGE; };
    // single-stage kernels issue the next tile's copies as soon as the current tile no
    // longer reads its operator fields (the state is not copied forward from psi = 0,
    // and has its own second buffer backward)
    const bool early = G::NSTAGE == 1 && (BWD || x_zero);
    fetch(tb, 0);
    if (threadIdx.x == 0) issue(tb, 0, 0, xbuf(0, 0), pre >= 0 ? 2 : 0);
    for (int t = tb, k = 0; t < te; t += step, ++k) {
        const int hs = k & 1;
        const int ds = G::NSTAGE == 2 ? (k & 1) : 0;
        const unsigned parity = (unsigned)((G::NSTAGE == 2 ? (k >> 1) : k) & 1);
        const bool more = t + step < te;
        if (G::NSTAGE == 2 && more) {
            fetch(t + step, hs ^ 1);
            if (threadIdx.x == 0) issue(t + step, hs ^ 1, ds ^ 1, xbuf(k + 1, ds ^ 1), 0);
        }
        const bool ok = mbar_wait(&bar[ds], parity, cs_s[hs].wait_ns);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(&hdr(hs)->P.cs->status, kStatusTimeout);
                __threadfence();
                mbar_wait(&bar[ds], parity);
                if (G::NSTAGE == 2 && more) mbar_wait(&bar[ds ^ 1], (unsigned)(((k + 1) >> 1) & 1));
            }
            __syncthreads();
            return;
        }
        const TileJob<T>& J = *hdr(hs);
        const int lt = t - J.tile0;
        const int bx = lt % J.L.ntx, by = lt / J.L.ntx;
        T* b = buf + ds * G::STAGE;
        auto fields_free = [&]() {
            if (!(early && more)) return;
            fence_proxy_async();
            fetch(t + step, hs ^ 1);
            __syncthreads();
            if (threadIdx.x == 0) issue(t + step, hs ^ 1, 0, xbuf(k + 1, 0), 0);
        };
        if constexpr (BWD)
            tile_bwd_compute<T, FINE>(J.L, cs_s[hs], bx, by, xbuf(k, ds), b + G::FS, b + (1 + G::NCOEF) * G::FS,
                                      b + G::NFLD * G::FS, fields_free);
        else
            tile_fwd_compute<T, FINE>(J.L, J.C, cs_s[hs], x_zero, bx, by, xbuf(k, ds), b + G::FS,
                                      b + (1 + G::NCOEF) * G::FS, Rr, fields_free);
        fence_proxy_async();
        __syncthreads();
        if (G::NSTAGE == 1 && !early && more) {
            fetch(t + step, hs ^ 1);
            if (threadIdx.x == 0) issue(t + step, hs ^ 1, 0, xbuf(k + 1, 0), 0);
        }
    }
}

// Low-rank step after a fused sweep (Alg. 3 last line, see kernels.cu):
//   z = B^T theta*_s from zparts, v = z - d - L_Gamma z',
//   theta' = theta*_s - G v on the support of G;
// on the way down also f_{l-1} += H v (H = P^T A G) and
// d_{l-1} = d_l - B^T theta' = d_l - z + (B^T G) v.
// The same step when m <= kLrReg and every thread holds at most one row of G
// (and of H): all loads that do not depend on v -- the thread's G/H row, its
// site and the value there, B^T G, d, the Cholesky diagonal -- are issued before
// z and v are formed.  The static ones (G/H rows, sites, B^T G, column pointers,
// L_Gamma) are issued before the wait on the preceding launch (pdl_wait), so
// after it only the state, f, d and the z partials are fetched: one round trip.
// The sums run in the same order as the general path.  Both forms call
// pdl_wait themselves.
constexpr int kLrReg = 16;
// entries of a column of B whose sites are loaded before the wait (point observations have 4)
constexpr int kLrEnt = 4;

// z_k = (B^T theta)_k from the z partials of the tile kernels, or (streamed finest
// grid, no partials) from the state itself: the same products w_t theta(site_t),
// rounded before they are summed, in the same order
template <typename T>
__device__ __forceinline__ double lowrank_z(const DevLevel<T>& L, const T* x, int k)
{
    double acc = 0.0;
    if (L.zparts)
        for (int t = L.bcol_ptr[k]; t < L.bcol_ptr[k + 1]; ++t) acc += L.zparts[t];
    else
        for (int t = L.bcol_ptr[k]; t < L.bcol_ptr[k + 1]; ++t) acc += __dmul_rn(L.bcol_w[t], (double)x[L.bcol_site[t]]);
    return acc;
}

template <typename T>
__device__ __forceinline__ void lowrank_fused_short(const DevLevel<T>& L, const DevLevel<T>& C, const DevProblem& P,
                                                    int down, int blk, double* z, double* zp, double* v)
{
    const int m = P.m;
    const int dir = down ? 0 : 1;
    const unsigned slot = down ? 0u : 1u;
    T* x = down ? L.x2 : L.x;
    const int r0 = blk * blockDim.x + threadIdx.x;
    const int k0 = threadIdx.x;
    const bool hg = r0 < L.g_rows[dir];
    const bool hh = down && r0 < L.h_rows;
    const bool hk = k0 < m;
    const bool hb = down && blk == 0 && hk;
    T gr[kLrReg], hr[kLrReg];
    double bg[kLrReg];
#pragma unroll
    for (int k = 0; k < kLrReg; ++k) {
        gr[k] = (hg && k < m) ? L.gT[dir][(long long)r0 * m + k] : T(0);
        hr[k] = (hh && k < m) ? L.hT[(long long)r0 * m + k] : T(0);
        bg[k] = (hb && k < m) ? L.BtG[k0 * m + k] : 0.0;
    }
    const long long gs = hg ? L.g_site[dir][r0] : 0;
    const long long hs = hh ? L.h_site[r0] : 0;
    int t0 = 0, t1 = 0;
    double lgk = 0.0;
    if (hk) {
        t0 = L.bcol_ptr[k0];
        t1 = L.bcol_ptr[k0 + 1];
        if (P.gamma_diag) lgk = P.LG[k0 * m + k0];
    }
    // without z partials (streamed finest grid) the state is read at the entries of
    // column k0 of B: their sites and weights are static
    const bool zst = L.zparts == nullptr;
    long long es[kLrEnt];
    double ew[kLrEnt];
#pragma unroll
    for (int u = 0; u < kLrEnt; ++u) {
        const bool has = hk && zst && t0 + u < t1;
        es[u] = has ? L.bcol_site[t0 + u] : 0;
        ew[u] = has ? L.bcol_w[t0 + u] : 0.0;
    }
    // everything below depends on the preceding launches
    pdl_wait();
    const CycleState cs = *P.cs;
    const double dk = hk ? L.d[k0] : 0.0;
    const T xv = hg ? x[gs] : T(0);
    const T fv = hh ? C.f[hs] : T(0);
    if (hk) {
        double acc = 0.0;
        if (zst) {
#pragma unroll
            for (int u = 0; u < kLrEnt; ++u)
                if (t0 + u < t1) acc += __dmul_rn(ew[u], (double)x[es[u]]);
            for (int t = t0 + kLrEnt; t < t1; ++t) acc += __dmul_rn(L.bcol_w[t], (double)x[L.bcol_site[t]]);
        } else {
            for (int t = t0; t < t1; ++t) acc += L.zparts[t];
        }
        z[k0] = acc;
        zp[k0] = cs.noise ? lowrank_normal<T>(cs, L.level, slot, k0) : 0.0;
    }
    __syncthreads();
    if (hk) {
        double lz = 0.0;
        if (cs.noise) {
            if (P.gamma_diag)
                lz = lgk * zp[k0];
            else
                for (int t = 0; t <= k0; ++t) lz += P.LG[k0 * m + t] * zp[t];
        }
        v[k0] = z[k0] - dk - lz;
    }
    __syncthreads();
    if (hg) {
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < kLrReg; ++k)
            if (k < m) acc += gr[k] * (T)v[k];
        x[gs] = xv - acc;
    }
    if (hh) {
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < kLrReg; ++k)
            if (k < m) acc += hr[k] * (T)v[k];
        C.f[hs] = fv + acc;
    }
    if (hb) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < kLrReg; ++k)
            if (k < m) acc += bg[k] * v[k];
        L.dnext[k0] = dk - z[k0] + acc;
    }
}

template <typename T>
__device__ __forceinline__ void lowrank_fused_body(const DevLevel<T>& L, const DevLevel<T>& C, const DevProblem& P,
                                                   int down, int blk, int nblk)
{
    __shared__ double z[kMaxObs];
    __shared__ double zp[kMaxObs];
    __shared__ double v[kMaxObs];
    const int m = P.m;
    const int dir = down ? 0 : 1;
    const unsigned slot = down ? 0u : 1u;
    const int stride = nblk * blockDim.x;
    if (m <= kLrReg && L.g_rows[dir] <= stride && (!down || L.h_rows <= stride)) {
        lowrank_fused_short<T>(L, C, P, down, blk, z, zp, v);
        return;
    }
    pdl_wait();
    const CycleState cs = *P.cs;
    T* x = down ? L.x2 : L.x;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        z[k] = lowrank_z<T>(L, x, k);
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

// batched: job j owns blocks [block0, block0 + nblocks)
template <typename T>
__global__ void k_lowrank_fused_batch(const LowrankJob<T>* __restrict__ jobs, int njobs, int per, int down)
{
    __shared__ __align__(16) LowrankJob<T> J;
    pdl_launch_dependents();
    load_job(J, jobs + find_job(jobs, njobs, per, blockIdx.x));   // static table
    lowrank_fused_body<T>(J.L, J.C, J.P, down, blockIdx.x - J.block0, J.nblocks);   // waits inside
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
namespace {

// 2D tiled map of a padded field: pitch x rows elements, box bw x bh, zero fill outside
template <typename T>
bool encode_field(CUtensorMap* m, const T* base, int pitch, int rows, int bw, int bh)
{
    EncodeTiled fn = tensor_map_encoder();
    if (!fn || !base) return false;
    cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(T)};
    cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
    cuuint32_t es[2] = {1, 1};
    return fn(m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, (void*)base,
              dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T, bool FINE, bool BWD>
bool make_maps(const DevLevel<T>& L, const DevLevel<T>& C, TileMaps* out)
{
    using G = TileGeom<T, FINE, BWD>;
    static_assert(G::NMAP <= kTileMaxMaps, "tensor maps per tile job");
    const int rows = L.n + 2;
    bool ok = encode_field<T>(&out->m[0], BWD ? L.x2 : L.x, L.pitch, rows, G::SX, G::SY);
    if (FINE) {
        ok = ok && encode_field<T>(&out->m[1], L.diag, L.pitch, rows, G::SX, G::SY);
    } else {
        for (int t = 0; t < G::NCOEF; ++t)
            ok = ok && encode_field<T>(&out->m[1 + t], L.coef + (long long)t * L.alloc, L.pitch, rows, G::SX, G::SY);
        ok = ok && encode_field<T>(&out->m[1 + G::NCOEF], L.f, L.pitch, rows, G::SX, G::SY);
    }
    if (BWD) ok = ok && encode_field<T>(&out->m[G::NFLD], C.x, C.pitch, C.n + 2, G::PXA, G::PY);
    return ok;
}

// resident CTAs per SM of each tile kernel (filled by tile_prepare_batch) and the SM count
int g_tile_ctas[2][2][2];  // [fp64][fine][bwd]
int g_sms = 0;

template <typename T, bool FINE, bool BWD>
cudaError_t prepare_one()
{
    const size_t smem = tile_smem_bytes<T, FINE, BWD>() + 128;
    cudaError_t e = cudaFuncSetAttribute(k_tile_batch<T, FINE, BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_tile_batch<T, FINE, BWD>, TileGeom<T, FINE, BWD>::NT,
                                                      smem);
    if (e != cudaSuccess) return e;
    g_tile_ctas[sizeof(T) == 8][FINE][BWD] = nb > 0 ? nb : 1;
    return cudaSuccess;
}

template <typename T, bool FINE, bool BWD>
void launch_one(const TileJob<T>* jobs, const TileMaps* maps, int njobs, int per, int ntiles, bool x_zero,
                cudaStream_t st)
{
    long long grid = (long long)g_tile_ctas[sizeof(T) == 8][FINE][BWD] * (g_sms > 0 ? g_sms : 1);
    // chains with a common tile count and no more chains than resident CTAs: cpj CTAs per chain
    int cpj = 0;
    if (per > 0 && njobs <= grid) {
        cpj = (int)(grid / njobs);
        if (cpj > per) cpj = per;
        grid = (long long)cpj * njobs;
    } else if (grid > ntiles) {
        grid = ntiles;
    }
    launch_pdl(k_tile_batch<T, FINE, BWD>, dim3((unsigned)grid), dim3(TileGeom<T, FINE, BWD>::NT),
               tile_smem_bytes<T, FINE, BWD>() + 128, st, jobs, maps, njobs, per, ntiles, cpj, x_zero ? 1 : 0);
}

}  // namespace

template <typename T>
bool make_tile_maps(const DevLevel<T>& L, const DevLevel<T>& C, bool bwd, TileMaps* out)
{
    std::memset(out, 0, sizeof(*out));
    if (L.fine)
        return bwd ? make_maps<T, true, true>(L, C, out) : make_maps<T, true, false>(L, C, out);
    return bwd ? make_maps<T, false, true>(L, C, out) : make_maps<T, false, false>(L, C, out);
}

template <typename T>
cudaError_t tile_prepare_batch()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = prepare_one<T, true, false>();
    if (e == cudaSuccess) e = prepare_one<T, true, true>();
    if (e == cudaSuccess) e = prepare_one<T, false, false>();
    if (e == cudaSuccess) e = prepare_one<T, false, true>();
    if (e == cudaSuccess && !tensor_map_encoder()) e = cudaErrorNotSupported;
    return e;
}

template <typename T>
void launch_tile_batch(const TileJob<T>* jobs, const TileMaps* maps, int njobs, int per, int ntiles, bool fine,
                       bool bwd, bool x_zero, cudaStream_t st, int& launches)
{
    if (ntiles <= 0) return;
    if (fine)
        bwd ? launch_one<T, true, true>(jobs, maps, njobs, per, ntiles, x_zero, st)
            : launch_one<T, true, false>(jobs, maps, njobs, per, ntiles, x_zero, st);
    else
        bwd ? launch_one<T, false, true>(jobs, maps, njobs, per, ntiles, x_zero, st)
            : launch_one<T, false, false>(jobs, maps, njobs, per, ntiles, x_zero, st);
    ++launches;
}

template <typename T>
void launch_lowrank_batch(const LowrankJob<T>* jobs, int njobs, int per, int nblocks, bool down, cudaStream_t st,
                          int& launches)
{
    if (nblocks <= 0) return;
    launch_pdl(k_lowrank_fused_batch<T>, dim3((unsigned)nblocks), dim3(256), 0, st, jobs, njobs, per, down ? 1 : 0);
    ++launches;
}

#define MGMC_TILE_INST(T)                                                                                        \
    template bool make_tile_maps<T>(const DevLevel<T>&, const DevLevel<T>&, bool, TileMaps*);                    \
    template cudaError_t tile_prepare_batch<T>();                                                                 \
    template void launch_tile_batch<T>(const TileJob<T>*, const TileMaps*, int, int, int, bool, bool, bool,       \
                                       cudaStream_t, int&);                                                       \
    template void launch_lowrank_batch<T>(const LowrankJob<T>*, int, int, int, bool, cudaStream_t, int&);

MGMC_TILE_INST(float)
MGMC_TILE_INST(double)

}  // namespace mgmc
