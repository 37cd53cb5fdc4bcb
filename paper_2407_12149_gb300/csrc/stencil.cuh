// stencil.cuh -- per-site arithmetic of the random Gibbs smoother, the
// residual and the grid transfers, shared by all sweep kernels.
//
// FP64 uses the plain form x_i <- (f_i + xi_i - sum_{j != i} a_ij x_j) / a_ii
// (Alg. 3 as a colour-ordered Gauss-Seidel sweep).  FP32 uses the algebraically
// identical correction form x_i <- x_i + (f_i + xi_i - (A x)_i) / a_ii (1/a_ii and
// sqrt(a_ii) from one reciprocal square root) with
// (A x)_i = rowsum_i x_i + sum_{j != i} a_ij (x_j - x_i): in single precision
// this keeps the small kappa^2 part of the operator (and so the smooth modes
// of the field) accurate, which the plain form would round away.
#pragma once
#include "common.cuh"

namespace mgmc {

// stencil offsets in lexicographic order of (dx, dy, dz), dx fastest
template <int DIM>
struct Offsets {
    static constexpr int NS = DIM == 2 ? 9 : 27;
    static constexpr int C = (NS - 1) / 2;
};

template <int DIM>
__device__ __forceinline__ long long off_of(int o, int pitch, long long plane)
{
    int dx = o % 3 - 1;
    int dy = (o / 3) % 3 - 1;
    int dz = DIM == 3 ? o / 9 - 1 : 0;
    return (long long)dx + (long long)pitch * dy + plane * dz;
}

// a(i, i + o) of a coarse level, read from the symmetric half storage
template <int DIM, typename T>
__device__ __forceinline__ T coef_at(const DevLevel<T>& L, long long e, int o)
{
    constexpr int C = Offsets<DIM>::C;
    constexpr int NS = Offsets<DIM>::NS;
    if (o > C) return L.coef[(long long)(o - C) * L.alloc + e];
    long long en = e + off_of<DIM>(o, L.pitch, L.plane);
    return L.coef[(long long)(NS - 1 - o - C) * L.alloc + en];
}

// radius-2 (25-point) 2D stencils: offset o = (dx+2) + 5 (dy+2), centre 12
__device__ __forceinline__ long long off25(int o, int pitch)
{
    return (long long)(o % 5 - 2) + (long long)pitch * (o / 5 - 2);
}

// a(i, i + o) of a 25-point grid from the symmetric half storage (a(i, i + o) for
// o < 12 is a(i + o, i), slot 12 - o at the neighbour)
__device__ __forceinline__ double coef25_at(const DevLevel<double>& L, long long e, int o)
{
    if (o > 12) return L.coef[(long long)(o - 12) * L.alloc + e];
    return L.coef[(long long)(12 - o) * L.alloc + e + off25(o, L.pitch)];
}

// one Gibbs update of a 25-point site, x_i <- (f_i + sqrt(a_ii) z - sum_{j != i} a_ij x_j) / a_ii
// with the neighbours in lexicographic offset order; 1 / a_ii and sqrt(a_ii) come from the
// host (FP64 division and square root are long instruction sequences on this GPU)
__device__ __forceinline__ double update25(const DevLevel<double>& L, long long e, double z)
{
    double acc = L.f ? L.f[e] : 0.0;
    acc += L.inv_sqrt25[L.alloc + e] * z;
#pragma unroll
    for (int o = 0; o < 25; ++o) {
        if (o == 12) continue;
        acc -= coef25_at(L, e, o) * L.x[e + off25(o, L.pitch)];
    }
    return acc * L.inv_sqrt25[e];
}

// ---------------------------------------------------------------------------
// one site update of the Gibbs sweep with right-hand side fdense_i + sqrt(a_ii) z
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ double fine_update(const DevLevel<double>& L, long long e, double z)
{
    const double* x = L.x;
    double aii = L.diag[e];
    double w = L.woff;
    double acc = L.f ? L.f[e] : 0.0;
    acc += sqrt(aii) * z;
    // neighbours in the order (0,0,-1), (0,-1,0), (-1,0,0), (1,0,0), (0,1,0), (0,0,1)
    if (DIM == 3) acc += w * x[e - L.plane];
    acc += w * x[e - L.pitch];
    acc += w * x[e - 1];
    acc += w * x[e + 1];
    acc += w * x[e + L.pitch];
    if (DIM == 3) acc += w * x[e + L.plane];
    return acc / aii;
}

template <int DIM>
__device__ __forceinline__ float fine_update(const DevLevel<float>& L, long long e, float z)
{
    const float* x = L.x;
    float xi = x[e];
    float c = L.diag[e];
    float w = L.woff;
    float lap = (xi - x[e - L.pitch]) + (xi - x[e - 1]) + (xi - x[e + 1]) + (xi - x[e + L.pitch]);
    if (DIM == 3) lap += (xi - x[e - L.plane]) + (xi - x[e + L.plane]);
    float aii = fmaf(2.0f * DIM, w, c);
    float Ax = fmaf(c, xi, w * lap);
    float ia, sa;
    inv_and_sqrt(aii, ia, sa);
    float rhs = (L.f ? L.f[e] : 0.0f) + sa * z;
    return xi + (rhs - Ax) * ia;
}

template <int DIM>
__device__ __forceinline__ double coarse_update(const DevLevel<double>& L, long long e, double z)
{
    constexpr int NS = Offsets<DIM>::NS;
    constexpr int C = Offsets<DIM>::C;
    double aii = L.coef[e];
    double acc = L.f ? L.f[e] : 0.0;
    acc += sqrt(aii) * z;
#pragma unroll
    for (int o = 0; o < NS; ++o) {
        if (o == C) continue;
        acc -= coef_at<DIM>(L, e, o) * L.x[e + off_of<DIM>(o, L.pitch, L.plane)];
    }
    return acc / aii;
}

template <int DIM>
__device__ __forceinline__ float coarse_update(const DevLevel<float>& L, long long e, float z)
{
    constexpr int NS = Offsets<DIM>::NS;
    constexpr int C = Offsets<DIM>::C;
    float xi = L.x[e];
    float s = L.coef[e];
    float lap = 0.0f, offsum = 0.0f;
#pragma unroll
    for (int o = 0; o < NS; ++o) {
        if (o == C) continue;
        float a = coef_at<DIM>(L, e, o);
        lap = fmaf(a, L.x[e + off_of<DIM>(o, L.pitch, L.plane)] - xi, lap);
        offsum += a;
    }
    float aii = s - offsum;
    float Ax = fmaf(s, xi, lap);
    float ia, sa;
    inv_and_sqrt(aii, ia, sa);
    float rhs = (L.f ? L.f[e] : 0.0f) + sa * z;
    return xi + (rhs - Ax) * ia;
}

// One FP32 Gibbs update of a 5-point site from its value xi, its four neighbours,
// the row-sum part c = s kappa^2_i and the off-diagonal magnitude w (dense
// right-hand side 0: the finest grid), the same operations as fine_update.
__device__ __forceinline__ float fine_site(float xi, float up, float lf, float rt, float dn, float c, float w, float z)
{
    float lap = (xi - up) + (xi - lf) + (xi - rt) + (xi - dn);
    float aii = fmaf(4.0f, w, c);
    float Ax = fmaf(c, xi, w * lap);
    float ia, sa;
    inv_and_sqrt(aii, ia, sa);
    float rhs = 0.0f + sa * z;
    return xi + (rhs - Ax) * ia;
}

// (A x)_i of a 5-point FP32 site (dense part), the same operations as apply_A
__device__ __forceinline__ float fine_ax(float xi, float up, float lf, float rt, float dn, float c, float w)
{
    float lap = (xi - up) + (xi - lf) + (xi - rt) + (xi - dn);
    return fmaf(c, xi, w * lap);
}

// (A x)_e of the level (dense part of the operator)
template <int DIM>
__device__ __forceinline__ double apply_A(const DevLevel<double>& L, long long e)
{
    const double* x = L.x;
    if (L.fine) {
        double w = -L.woff;
        // oracle order: offsets lexicographic, centre in place
        double acc = 0.0;
        if (DIM == 3) acc += w * x[e - L.plane];
        acc += w * x[e - L.pitch];
        acc += w * x[e - 1];
        acc += L.diag[e] * x[e];
        acc += w * x[e + 1];
        acc += w * x[e + L.pitch];
        if (DIM == 3) acc += w * x[e + L.plane];
        return acc;
    }
    if (DIM == 2 && L.rad == 2) {
        double acc = 0.0;
#pragma unroll
        for (int o = 0; o < 25; ++o) {
            double a = (o == 12) ? L.coef[e] : coef25_at(L, e, o);
            acc += a * x[e + off25(o, L.pitch)];
        }
        return acc;
    }
    constexpr int NS = Offsets<DIM>::NS;
    constexpr int C = Offsets<DIM>::C;
    double acc = 0.0;
#pragma unroll
    for (int o = 0; o < NS; ++o) {
        double a = (o == C) ? L.coef[e] : coef_at<DIM>(L, e, o);
        acc += a * x[e + off_of<DIM>(o, L.pitch, L.plane)];
    }
    return acc;
}

template <int DIM>
__device__ __forceinline__ float apply_A(const DevLevel<float>& L, long long e)
{
    const float* x = L.x;
    float xi = x[e];
    if (L.fine) {
        float lap = (xi - x[e - L.pitch]) + (xi - x[e - 1]) + (xi - x[e + 1]) + (xi - x[e + L.pitch]);
        if (DIM == 3) lap += (xi - x[e - L.plane]) + (xi - x[e + L.plane]);
        return fmaf(L.diag[e], xi, L.woff * lap);
    }
    constexpr int NS = Offsets<DIM>::NS;
    constexpr int C = Offsets<DIM>::C;
    float lap = 0.0f;
#pragma unroll
    for (int o = 0; o < NS; ++o) {
        if (o == C) continue;
        lap = fmaf(coef_at<DIM>(L, e, o), x[e + off_of<DIM>(o, L.pitch, L.plane)] - xi, lap);
    }
    return fmaf(L.coef[e], xi, lap);
}

// --- FP32 9-point sites of a 4-site group (components 0..3), shared by the tile
// and the streaming kernels so that both evaluate the same operations in the
// same order (coarse_update / apply_A of the Galerkin grids).
// component k of the row (k = -1 and k = 4 are the scalar e outside the group)
__device__ __forceinline__ float cmp(const float4& v, float e, int k)
{
    return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : k == 3 ? v.w : e;
}

// rows of one 9-point group item: X rows -1, 0, +1; coefficient slot 0 and slots
// 1..4 on row 0; slots 2..4 on row -1; the dense right-hand side
struct Rows9 {
    float4 xm, x0, xp, s0, c1, c2, c3, c4, c2m, c3m, c4m, f;
    float exm, ex0, exp, c1e, c4me, c2me;  // the column outside the group (left or right, see cmp)
};

template <int Q>
__device__ __forceinline__ float site9(const Rows9& r, float z)
{
    const float xi = cmp(r.x0, 0.f, Q);
    float lap = 0.0f, offsum = 0.0f, a;
    // o = 0: (-1,-1)
    a = cmp(r.c4m, r.c4me, Q - 1);
    lap = fmaf(a, cmp(r.xm, r.exm, Q - 1) - xi, lap);
    offsum += a;
    // o = 1: (0,-1)
    a = cmp(r.c3m, 0.f, Q);
    lap = fmaf(a, cmp(r.xm, r.exm, Q) - xi, lap);
    offsum += a;
    // o = 2: (+1,-1)
    a = cmp(r.c2m, r.c2me, Q + 1);
    lap = fmaf(a, cmp(r.xm, r.exm, Q + 1) - xi, lap);
    offsum += a;
    // o = 3: (-1,0)
    a = cmp(r.c1, r.c1e, Q - 1);
    lap = fmaf(a, cmp(r.x0, r.ex0, Q - 1) - xi, lap);
    offsum += a;
    // o = 5: (+1,0)
    a = cmp(r.c1, 0.f, Q);
    lap = fmaf(a, cmp(r.x0, r.ex0, Q + 1) - xi, lap);
    offsum += a;
    // o = 6: (-1,+1)
    a = cmp(r.c2, 0.f, Q);
    lap = fmaf(a, cmp(r.xp, r.exp, Q - 1) - xi, lap);
    offsum += a;
    // o = 7: (0,+1)
    a = cmp(r.c3, 0.f, Q);
    lap = fmaf(a, cmp(r.xp, r.exp, Q) - xi, lap);
    offsum += a;
    // o = 8: (+1,+1)
    a = cmp(r.c4, 0.f, Q);
    lap = fmaf(a, cmp(r.xp, r.exp, Q + 1) - xi, lap);
    offsum += a;
    const float s = cmp(r.s0, 0.f, Q);
    const float aii = s - offsum;
    const float Ax = fmaf(s, xi, lap);
    float ia, sa;
    inv_and_sqrt(aii, ia, sa);
    const float rhs = cmp(r.f, 0.f, Q) + sa * z;
    return xi + (rhs - Ax) * ia;
}

// rows for the 4-site residual: extras on both sides
struct Rows9R {
    Rows9 r;      // extras of r on the left (exm, ex0, exp, c1e, c4me)
    float xmr, x0r, xpr, c2mr;  // right extras
};

template <int Q>
__device__ __forceinline__ float ax9q(const Rows9R& R)
{
    const Rows9& r = R.r;
    auto X = [&](const float4& v, float el, float er, int k) { return k < 0 ? el : k > 3 ? er : cmp(v, 0.f, k); };
    const float xi = cmp(r.x0, 0.f, Q);
    float lap = 0.0f;
    lap = fmaf(cmp(r.c4m, r.c4me, Q - 1), X(r.xm, r.exm, R.xmr, Q - 1) - xi, lap);
    lap = fmaf(cmp(r.c3m, 0.f, Q), X(r.xm, r.exm, R.xmr, Q) - xi, lap);
    lap = fmaf(Q + 1 > 3 ? R.c2mr : cmp(r.c2m, 0.f, Q + 1), X(r.xm, r.exm, R.xmr, Q + 1) - xi, lap);
    lap = fmaf(cmp(r.c1, r.c1e, Q - 1), X(r.x0, r.ex0, R.x0r, Q - 1) - xi, lap);
    lap = fmaf(cmp(r.c1, 0.f, Q), X(r.x0, r.ex0, R.x0r, Q + 1) - xi, lap);
    lap = fmaf(cmp(r.c2, 0.f, Q), X(r.xp, r.exp, R.xpr, Q - 1) - xi, lap);
    lap = fmaf(cmp(r.c3, 0.f, Q), X(r.xp, r.exp, R.xpr, Q) - xi, lap);
    lap = fmaf(cmp(r.c4, 0.f, Q), X(r.xp, r.exp, R.xpr, Q + 1) - xi, lap);
    return fmaf(cmp(r.s0, 0.f, Q), xi, lap);
}

// 1D weight of the canonical prolongation for offset p in {-1, 0, 1}
__device__ __forceinline__ double pw(int p) { return p == 0 ? 1.0 : 0.5; }

}  // namespace mgmc
