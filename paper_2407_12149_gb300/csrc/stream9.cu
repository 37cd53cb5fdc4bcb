// stream9.cu -- the 9-point Galerkin grids (FP32) streamed in bands.
//
// The grid of every chain at one depth of the V-cycle is cut into bands of 64
// columns and each band into strips of 16 rows.  A CTA owns a contiguous range
// of strips and streams down each band it meets, one strip per pipeline step,
// through a ring of five 8-row blocks of the five operator fields, the dense
// right-hand side and (backward) the state in shared memory; each block is one
// TMA box of 80 x 8 per field (the band plus an 8-column halo on each side),
// issued one step before it is needed.  The four parity colours of a sweep form
// a wavefront: colour phases on rows of one parity lag each other by one row, so
// every value a phase reads is the one a global colour sweep gives (only the
// first step of a run and a band halo that shrinks by one column per phase are
// recomputed).  With R the first row of step s:
//   forward (from psi = 0: the state starts at zero; Alg. 1 pre-smoothing,
//   residual and restriction)
//     P0 colour (0,0) on the even rows of [R, R+16), P1 (1,1) and P2 (0,1) on the
//     odd rows of [R-1, R+15), P3 (1,0) on the even rows of [R-2, R+14), residual
//     r = fd - A theta*_s on [R-3, R+13), restriction of the coarse rows whose
//     three fine rows are complete;
//   backward (prolongation and post-smoothing, colours in reverse order)
//     theta += P psi on [R, R+16), P0 colour (1,0) on the even rows of
//     [R-1, R+15), P1 (0,1) and P2 (1,1) on the odd rows of [R-2, R+14), P3
//     (0,0) on the even rows of [R-3, R+13); P3 of a step runs in the next
//     step's first barrier interval, beside its prolongation (disjoint rows).
// Thread (g, rp) owns the 4-site group g on the even row a = R + 2 rp (P0), the
// odd row a - 1 (P1, P2) and the even row a - 2 (P3), and the residual rows
// a - 3 and a - 2; it stores the final rows a - 1 and a - 2.
//
// The per-site arithmetic (site9 / ax9q of stencil.cuh), the noise draws and the
// sums of the residual, restriction and prolongation are those of the tile
// kernels (tile2d.cu) in the same order: both paths give bitwise identical
// states.  The products w_t theta(site_t) of Alg. 3's z = B^T theta are left to
// the low-rank kernel, which reads the state at the observation entries.
#include <algorithm>
#include <cstring>

#include "stencil.cuh"
#include "stream9.cuh"
#include "stream_core.cuh"
#include "tma.cuh"

namespace mgmc {

namespace {

using namespace sc;

constexpr int kBW = kStream9Band;
constexpr int kK = kStream9Rows;
constexpr int kNG = kBW / 4 + 3;    // groups of columns x0 - 4 .. x0 + kBW + 7
constexpr int kNT = kNG * kK / 2;   // threads: one group of two rows per step
constexpr int kSX = kBW + 16;       // staged row: columns x0 - 8 .. x0 + kBW + 7
constexpr int kBK = 8;              // rows per TMA block (two per step)
constexpr int kNB = 5;              // ring slots: three blocks read by a step, two in flight
constexpr int kRing = kNB * kBK;    // rows of each field ring
constexpr int kFS = kRing * kSX;    // floats of one field ring
constexpr int kRW = 4 * (kNG - 1);  // residual row: the groups of columns x0 .. x0 + kBW + 7
constexpr int kRRing = 64;          // rows of the residual ring (a step writes rows R-3 .. R+12 while the
                                    // restriction of the previous step reads rows R-20 .. R-4)
constexpr int kPX = kBW / 2 + 8;    // staged coarse columns x0/2 - 4 .. x0/2 + kBW/2 + 3
constexpr int kPK = kBK / 2;        // coarse rows per block
constexpr int kPRing = kNB * kPK;   // rows of the psi ring
constexpr int kNF = 7;              // staged fields: state, five operator fields, right-hand side
// TMA boxes (columns x rows) and the bytes each delivers: the tensor maps and the
// mbarrier's expected transaction bytes both use these
constexpr int kBoxW = kSX, kBoxH = kBK, kPBoxW = kPX, kPBoxH = kPK;
constexpr unsigned kBox = kBoxW * kBoxH * 4;
constexpr unsigned kPBox = kPBoxW * kPBoxH * 4;
constexpr size_t kHead = 256;  // mbarriers; also keeps the reads one float left of the rings inside shared memory
constexpr int kTail = 8;       // floats after the last ring (the right-edge read of the last group)
// hand-off of site normals between the threads of consecutive rows: [step parity][rp][g][2]
constexpr int kZx = 2 * (kK / 2) * kNG * 2;
constexpr size_t kFwdSmem = 128 + kHead + 4 * ((size_t)kNF * kFS + (size_t)kRRing * kRW + kZx + kTail);
constexpr size_t kBwdSmem = 128 + kHead + 4 * ((size_t)kNF * kFS + (size_t)kPRing * kPX + kZx + kTail);
static_assert(kNT >= 8 * 16, "thread layout: the restriction needs 8 x 16 threads");
static_assert(kBox % 128 == 0 && kPBox % 128 == 0 && (kFS * 4) % 128 == 0, "TMA destinations on 128-byte boundaries");
static_assert(kSX <= 256 && kPX <= 256 && (kSX * 4) % 16 == 0 && (kPX * 4) % 16 == 0, "TMA box");
static_assert(kNB * 8 <= (int)kHead && kNB <= 32, "mbarriers and phase bits");
static_assert(kRRing >= 2 * kK + 1 && (kRRing & (kRRing - 1)) == 0, "residual ring");

__device__ __forceinline__ int wrap(int v, int m) { return v >= m ? v - m : v; }

// the 9-point rows of a group: x rows m (j - 1), o (j), p (j + 1), the operator rows
// j and j - 1, the right-hand side row j; edge columns left (PX = 0) or right (PX = 1)
template <int PX>
__device__ __forceinline__ void load9(Rows9& r, const float* X, const float* Cf, const float* F, int om, int oo, int op)
{
    r.xm = ld4(X + om);
    r.x0 = ld4(X + oo);
    r.xp = ld4(X + op);
    r.s0 = ld4(Cf + oo);
    r.c1 = ld4(Cf + kFS + oo);
    r.c2 = ld4(Cf + 2 * kFS + oo);
    r.c3 = ld4(Cf + 3 * kFS + oo);
    r.c4 = ld4(Cf + 4 * kFS + oo);
    r.c2m = ld4(Cf + 2 * kFS + om);
    r.c3m = ld4(Cf + 3 * kFS + om);
    r.c4m = ld4(Cf + 4 * kFS + om);
    r.f = ld4(F + oo);
    if (PX == 0) {
        r.exm = X[om - 1];
        r.ex0 = X[oo - 1];
        r.exp = X[op - 1];
        r.c1e = Cf[kFS + oo - 1];
        r.c4me = Cf[4 * kFS + om - 1];
        r.c2me = 0.f;
    } else {
        r.exm = X[om + 4];
        r.ex0 = X[oo + 4];
        r.exp = X[op + 4];
        r.c1e = 0.f;
        r.c4me = 0.f;
        r.c2me = Cf[2 * kFS + om + 4];
    }
}

// the same-colour sites PX and PX + 2 of the group row r.x0 (v0, v1: which are updated)
template <int PX>
__device__ __forceinline__ float4 upd9(const Rows9& r, float z0, float z1, bool v0, bool v1)
{
    const float na = site9<PX>(r, z0);
    const float nb = site9<PX + 2>(r, z1);
    float4 o = r.x0;
    if (PX == 0) {
        o.x = v0 ? na : o.x;
        o.z = v1 ? nb : o.z;
    } else {
        o.y = v0 ? na : o.y;
        o.w = v1 ? nb : o.w;
    }
    return o;
}

// r = fd - A theta of the 4 sites of the group row oo (x rows om, oo, op)
__device__ __forceinline__ float4 res9(const float* X, const float* Cf, const float* F, int om, int oo, int op)
{
    Rows9R R;
    load9<0>(R.r, X, Cf, F, om, oo, op);
    R.xmr = X[om + 4];
    R.x0r = X[oo + 4];
    R.xpr = X[op + 4];
    R.c2mr = Cf[2 * kFS + om + 4];
    const Rows9& r = R.r;
    return make_float4(r.f.x - ax9q<0>(R), r.f.y - ax9q<1>(R), r.f.z - ax9q<2>(R), r.f.w - ax9q<3>(R));
}

// Forward pass of the 9-point grids of one depth, from psi = 0: one launch over all
// strips of all chains.
__global__ void __launch_bounds__(kNT, 2)
    k_stream9_fwd(const StreamJob* __restrict__ jobs, const Stream9Maps* __restrict__ maps, int njobs,
                  long long total)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* sm = smem_align_up<128>(smem_dyn);
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm);
    float* const Xr = reinterpret_cast<float*>(sm + kHead);
    float* const Cr = Xr + kFS;  // operator slot t at Cr + t kFS
    float* const Fr = Cr + 5 * kFS;
    float* const Rr = Fr + kFS;
    float* const Zx = Rr + kRRing * kRW;
    const int tid = threadIdx.x;
    const int g = tid % kNG, rp = tid / kNG;
    pdl_launch_dependents();
    if (tid == 0) {
        for (int q = 0; q < kNB; ++q) mbar_init(&bar[q]);
        fence_mbar_init();
    }
    __syncthreads();
    pdl_wait();
    const long long s_beg = total * blockIdx.x / gridDim.x, s_end = total * (blockIdx.x + 1) / gridDim.x;
    unsigned ph = 0;
    for (long long gs = s_beg; gs < s_end;) {
        const Run run = next_run<kK, kBW>(jobs, njobs, gs, s_end);
        const StreamJob* J = jobs + run.jb;
        const int n = run.n, nc = run.nc, x0 = run.x0, ya = run.ya, yb = run.yb;
        const int jend = yb >> 1;  // coarse rows J with centre row 2J + 1 in [ya, yb)
        // step s: R = ya - 2 + 16 s; it stores rows [R - 2, R + 14) and completes the
        // residual rows up to R + 12, so the coarse rows [ya/2 - 3 + 8 s, ya/2 + 5 + 8 s)
        const int S =
            max(max(cdiv_pos(yb - ya - (kK - 4), kK), cdiv_pos(jend - (ya >> 1) - (kK / 2 - 3), kK / 2)) + 1, 1);
        const int KB = 2 * S;  // last block; block k holds rows [ya - 6 + 8 k, ya + 2 + 8 k)
        const int base = ya - 6;
        const CycleState cs = *J->cs;
        const uint4 ctr = noise_counter(cs, 0u, 0u, J->L.level, 0u);
        const RoundKeys K = round_keys((unsigned)cs.seed, (unsigned)(cs.seed >> 32));
        const float zs = cs.noise ? 1.0f : 0.0f;
        const int nq = (n + 3) >> 2;
        const int gx = x0 - 4 + 4 * g;  // first column of the thread's group
        auto col = [&](int i, int lo, int hi) { return i >= lo && i <= hi && i >= 0 && i < n; };
        // columns each phase must update (the residual needs [x0, x0 + kBW])
        const bool c00 = col(gx, x0 - 4, x0 + kBW + 4), c02 = col(gx + 2, x0 - 4, x0 + kBW + 4);
        const bool c11 = col(gx + 1, x0 - 3, x0 + kBW + 3), c13 = col(gx + 3, x0 - 3, x0 + kBW + 3);
        const bool c20 = col(gx, x0 - 2, x0 + kBW + 2), c22 = col(gx + 2, x0 - 2, x0 + kBW + 2);
        const bool c31 = col(gx + 1, x0 - 1, x0 + kBW + 1), c33 = col(gx + 3, x0 - 1, x0 + kBW + 1);
        // site-noise block of the thread's row a in step 0 (row ya - 2 + 2 rp, group gx / 4);
        // the row above is nq back.  P0 takes the even columns' pair of row a, P1 and P2 the
        // odd and even pairs of row a - 1, P3 the odd pair of row a - 2, which the thread
        // above (rp - 1, or rp = 7 of the previous step) drew as its row a and hands over in Zx
unsigned blk = (unsigned)((long long)(ya - 2 + 2 * rp) * nq + (gx >> 2));
        const unsigned dstep = (unsigned)(kK * nq), drow = (unsigned)nq;
        auto zx = [&](int par, int r) { return Zx + ((par * (kK / 2) + r) * kNG + g) * 2; };
        const bool hasR = g >= 1;
        const bool rin = gx < n, r1 = gx + 1 < n, r2 = gx + 2 < n, r3 = gx + 3 < n;
        const bool hasS = g >= 1 && g <= kBW / 4 && gx < n;  // the band's own columns
        const int ci = tid & 15, cj = tid >> 4;  // restriction: coarse columns I, I + 1, row ya/2 - 3 + 8 t + cj
        const int I = (x0 >> 1) + 2 * ci;
        const bool hasC = tid < 8 * 16 && I < nc;
        const bool pairC = I + 1 < nc;
        float* const xout = J->L.x2 + J->L.base + gx;
        const long long pitch = J->L.pitch;
        float* const fc = J->C.f + J->C.base + I;
        const long long cpitch = J->C.pitch;
        auto rrow = [&](int j) { return ((j - ya + 8) & (kRRing - 1)) * kRW; };
        // restriction of the coarse rows of step t: f_c = sum_p w(p) r(2I + p), fine columns 2I .. 2I + 4
        auto restrict_step = [&](int t) {
            const int Jc = (ya >> 1) - 3 + (kK / 2) * t + cj;
            if (!hasC || Jc < (ya >> 1) || Jc >= jend) return;
            float4 v[3];
            float e[3];
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const float* rq = Rr + rrow(2 * Jc + b) + 4 * ci;
                v[b] = ld4(rq);
                e[b] = rq[4];
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
            float* o = fc + cpitch * Jc;
            // o is 8-byte aligned (I, the padded base and the pitch are even): both sites in one store
            if (pairC)
                *reinterpret_cast<float2*>(o) = make_float2(acc0, acc1);
            else
                *o = acc0;
        };
        const Stream9Maps* M = maps + run.jb;
        // block k: the operator fields and the right-hand side of its rows (the state
        // starts at zero and is cleared by the threads)
        auto issue = [&](int k) {
            const int q = k % kNB;
            mbar_expect_tx(&bar[q], 6 * kBox);
            const int prow = base + kBK * k + 1;
#pragma unroll
            for (int t = 0; t < 5; ++t) tma_load_2d(Cr + t * kFS + q * kBK * kSX, &M->c[t], x0 - 4, prow, &bar[q]);
            tma_load_2d(Fr + q * kBK * kSX, &M->f, x0 - 4, prow, &bar[q]);
        };
        auto clear_x = [&](int k) {
            float4* p = reinterpret_cast<float4*>(Xr + (k % kNB) * kBK * kSX);
            for (int i = tid; i < kBK * kSX / 4; i += kNT) p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        };
        // the rings are free: every thread is done with the previous run
        fence_proxy_async();
        __syncthreads();
        int issued = min(KB, kNB - 1), waited = -1;
        if (tid == 0)
            for (int k = 0; k <= issued; ++k) issue(k);
        for (int k = 0; k <= issued; ++k) clear_x(k);
        // ring row of a - 4 for the thread's even row a of step 0 (rows only grow)
        int r4 = 2 * rp;  // (ya - 2 + 2 rp) - 4 - base
        for (int s = 0; s < S; ++s) {
            const int R = ya - 2 + kK * s;
            // blocks up to 2s + 2 (rows up to R + 16) are in shared memory
            const bool ok = wait_blocks<kNB>(bar, ph, waited, min(2 * s + 2, KB), cs.wait_ns);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) give_up<kNB>(J->cs, bar, ph, waited, issued);
                __syncthreads();
                return;
            }
            // blocks 2s - 2 and 2s - 1 were last read in step s - 1: blocks 2s + 3, 2s + 4 take their slots
            if (s > 0) {
                const int hi = min(2 * s + 4, KB);
                if (tid == 0)
                    for (int k = 2 * s + 3; k <= hi; ++k) issue(k);
                for (int k = 2 * s + 3; k <= hi; ++k) clear_x(k);
                issued = max(issued, hi);
            }
            const int a = R + 2 * rp;  // even row of the thread
            const int o4 = r4 * kSX + 4 + 4 * g;
            const int o3 = wrap(r4 + 1, kRing) * kSX + 4 + 4 * g, o2 = wrap(r4 + 2, kRing) * kSX + 4 + 4 * g;
            const int o1 = wrap(r4 + 3, kRing) * kSX + 4 + 4 * g, o0 = wrap(r4 + 4, kRing) * kSX + 4 + 4 * g;
            const int op = wrap(r4 + 5, kRing) * kSX + 4 + 4 * g;
            const bool v0 = (unsigned)a < (unsigned)n, v1 = (unsigned)(a - 1) < (unsigned)n,
                       v2 = (unsigned)(a - 2) < (unsigned)n, v3 = (unsigned)(a - 3) < (unsigned)n;
            // P0, colour (0,0), row a
            {
                const Quad qa = draw_q(ctr, blk, K);
                float* z = zx(s & 1, rp);
                z[0] = qa.b0;
                z[1] = qa.b1;
                const float z00 = qa.a0, z01 = qa.a1;
                Rows9 r;
                load9<0>(r, Xr, Cr, Fr, o1, o0, op);
                st4(Xr + o0, upd9<0>(r, z00 * zs, z01 * zs, v0 && c00, v0 && c02));
            }
            __syncthreads();
            // P1, colour (1,1), and P2, colour (0,1), on row a - 1
            const Quad qm = draw_q(ctr, blk - drow, K);
            const float z10 = qm.b0, z11 = qm.b1, z20 = qm.a0, z21 = qm.a1;
            Rows9 r;
            load9<1>(r, Xr, Cr, Fr, o2, o1, o0);
            r.x0 = upd9<1>(r, z10 * zs, z11 * zs, v1 && c11, v1 && c13);
            st4(Xr + o1, r.x0);
            __syncthreads();
            {
                // rows a - 2 and a are unchanged since P1; the left column of row a - 1 is the
                // left group's P1 result
                r.exm = Xr[o2 - 1];
                r.ex0 = Xr[o1 - 1];
                r.exp = Xr[o0 - 1];
                r.c1e = Cr[kFS + o1 - 1];
                r.c4me = Cr[4 * kFS + o2 - 1];
                r.c2me = 0.f;
                const float4 o = upd9<0>(r, z20 * zs, z21 * zs, v1 && c20, v1 && c22);
                st4(Xr + o1, o);
                if (hasS && a - 1 >= ya && a - 1 < yb) st4(xout + pitch * (a - 1), o);
            }
            __syncthreads();
            // P3, colour (1,0), row a - 2; then its final state
            {
                float z30, z31;
                if (rp > 0 || s > 0) {
                    const float* z = rp > 0 ? zx(s & 1, rp - 1) : zx((s + 1) & 1, kK / 2 - 1);
                    z30 = z[0];
                    z31 = z[1];
                } else {
                    const Quad qu = draw_q(ctr, blk - 2 * drow, K);
                    z30 = qu.b0;
                    z31 = qu.b1;
                }
                Rows9 q;
                load9<1>(q, Xr, Cr, Fr, o3, o2, o1);
                const float4 o = upd9<1>(q, z30 * zs, z31 * zs, v2 && c31, v2 && c33);
                st4(Xr + o2, o);
                if (hasS && a - 2 >= ya && a - 2 < yb) st4(xout + pitch * (a - 2), o);
            }
            __syncthreads();
            // residual on rows a - 3 and a - 2 (0 outside the grid)
            if (hasR) {
                float4 rz = make_float4(0.f, 0.f, 0.f, 0.f), ra = rz;
                if (rin && v3) rz = res9(Xr, Cr, Fr, o4, o3, o2);
                if (rin && v2) ra = res9(Xr, Cr, Fr, o3, o2, o1);
                rz.y = r1 ? rz.y : 0.f;
                rz.z = r2 ? rz.z : 0.f;
                rz.w = r3 ? rz.w : 0.f;
                ra.y = r1 ? ra.y : 0.f;
                ra.z = r2 ? ra.z : 0.f;
                ra.w = r3 ? ra.w : 0.f;
                st4(Rr + rrow(a - 3) + 4 * (g - 1), rz);
                st4(Rr + rrow(a - 2) + 4 * (g - 1), ra);
            }
            // the coarse rows of the previous step (its residual rows are complete)
            if (s > 0) restrict_step(s - 1);
            fence_proxy_async();
            blk += dstep;
            r4 = wrap(r4 + kK, kRing);
        }
        __syncthreads();
        restrict_step(S - 1);
    }
}

// Backward pass of the 9-point grids of one depth: one launch over all strips of all
// chains.
__global__ void __launch_bounds__(kNT, 2)
    k_stream9_bwd(const StreamJob* __restrict__ jobs, const Stream9Maps* __restrict__ maps, int njobs,
                  long long total)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* sm = smem_align_up<128>(smem_dyn);
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm);
    float* const Xr = reinterpret_cast<float*>(sm + kHead);
    float* const Cr = Xr + kFS;
    float* const Fr = Cr + 5 * kFS;
    float* const Pr = Fr + kFS;
    float* const Zx = Pr + kPRing * kPX;
    const int tid = threadIdx.x;
    const int g = tid % kNG, rp = tid / kNG;
    pdl_launch_dependents();
    if (tid == 0) {
        for (int q = 0; q < kNB; ++q) mbar_init(&bar[q]);
        fence_mbar_init();
    }
    __syncthreads();
    pdl_wait();
    const long long s_beg = total * blockIdx.x / gridDim.x, s_end = total * (blockIdx.x + 1) / gridDim.x;
    unsigned ph = 0;
    for (long long gs = s_beg; gs < s_end;) {
        const Run run = next_run<kK, kBW>(jobs, njobs, gs, s_end);
        const StreamJob* J = jobs + run.jb;
        const int n = run.n, x0 = run.x0, ya = run.ya, yb = run.yb;
        // step s: R = ya - 4 + 16 s; it stores rows [R - 2, R + 14)
        const int S = cdiv_pos(yb - ya - (kK - 6), kK) + 1;
        const int KB = 2 * S;  // last block; block k holds rows [ya - 7 + 8 k, ya + 1 + 8 k) and
                               // coarse rows [ya/2 - 3 + 4 k, ya/2 + 1 + 4 k) of psi
        const int base = ya - 7;
        const int jcb = (ya >> 1) - 3;
        const CycleState cs = *J->cs;
        const uint4 ctr = noise_counter(cs, 0u, 0u, J->L.level, 1u);
        const RoundKeys K = round_keys((unsigned)cs.seed, (unsigned)(cs.seed >> 32));
        const float zs = cs.noise ? 1.0f : 0.0f;
        const int nq = (n + 3) >> 2;
        const int gx = x0 - 4 + 4 * g;
        auto col = [&](int i, int lo, int hi) { return i >= lo && i <= hi && i >= 0 && i < n; };
        // columns each phase must update (the band's own columns [x0, x0 + kBW) end final)
        const bool c01 = col(gx + 1, x0 - 3, x0 + kBW + 2), c03 = col(gx + 3, x0 - 3, x0 + kBW + 2);
        const bool c10 = col(gx, x0 - 2, x0 + kBW + 1), c12 = col(gx + 2, x0 - 2, x0 + kBW + 1);
        const bool c21 = col(gx + 1, x0 - 1, x0 + kBW), c23 = col(gx + 3, x0 - 1, x0 + kBW);
        const bool c30 = col(gx, x0, x0 + kBW - 1), c32 = col(gx + 2, x0, x0 + kBW - 1);
        // site-noise block of the thread's row a in step 0 (row ya - 4 + 2 rp, group gx / 4);
        // the row above is nq back.  P0 takes the odd columns' pair of row a, P1 and P2 the
        // even and odd pairs of row a - 1, P3 the even pair of row a - 2, which the thread
        // above (rp - 1, or rp = 7 of the previous step) drew as its row a and hands over in Zx
        unsigned blk = (unsigned)((long long)(ya - 4 + 2 * rp) * nq + (gx >> 2));
        const unsigned dstep = (unsigned)(kK * nq), drow = (unsigned)nq;
        auto zx = [&](int par, int r) { return Zx + ((par * (kK / 2) + r) * kNG + g) * 2; };
        const bool hasP = gx >= 0 && gx < n;
        const bool p1 = gx + 1 < n, p2 = gx + 2 < n, p3 = gx + 3 < n;
        const bool hasS = g >= 1 && g <= kBW / 4 && gx < n;
        float* const xout = J->L.x + J->L.base + gx;
        const long long pitch = J->L.pitch;
        auto prow = [&](int jc) { return ((jc - jcb) % kPRing) * kPX + 2 * g + 1; };
        const Stream9Maps* M = maps + run.jb;
        auto issue = [&](int k) {
            const int q = k % kNB;
            mbar_expect_tx(&bar[q], 7 * kBox + kPBox);
            const int prw = base + kBK * k + 1;
            tma_load_2d(Xr + q * kBK * kSX, &M->x, x0 - 4, prw, &bar[q]);
#pragma unroll
            for (int t = 0; t < 5; ++t) tma_load_2d(Cr + t * kFS + q * kBK * kSX, &M->c[t], x0 - 4, prw, &bar[q]);
            tma_load_2d(Fr + q * kBK * kSX, &M->f, x0 - 4, prw, &bar[q]);
            tma_load_2d(Pr + q * kPK * kPX, &M->p, x0 >> 1, jcb + kPK * k + 1, &bar[q]);
        };
        fence_proxy_async();
        __syncthreads();
        int issued = min(KB, kNB - 1), waited = -1;
        if (tid == 0)
            for (int k = 0; k <= issued; ++k) issue(k);
        int r3 = 2 * rp;  // ring row of a - 3 for the thread's even row a of step 0
        auto roff = [&](int r, int i) { return wrap(r + i, kRing) * kSX + 4 + 4 * g; };
        // P3, colour (0,0), on row a - 2 of the step whose row a - 3 sits in ring row r;
        // then its final state
        auto p3_step = [&](int a, int r, float z0, float z1) {
            const bool v2 = (unsigned)(a - 2) < (unsigned)n;
            const int o3 = roff(r, 0), o2 = roff(r, 1), o1 = roff(r, 2);
            Rows9 q;
            load9<0>(q, Xr, Cr, Fr, o3, o2, o1);
            const float4 o = upd9<0>(q, z0 * zs, z1 * zs, v2 && c30, v2 && c32);
            st4(Xr + o2, o);
            if (hasS && a - 2 >= ya && a - 2 < yb) st4(xout + pitch * (a - 2), o);
        };
        // the two blocks of step s are drawn in its first interval; P3's hand-over is read
        // in its second
        float z30 = 0.f, z31 = 0.f;
        for (int s = 0; s < S; ++s) {
            const int R = ya - 4 + kK * s;
            // the barrier also ends P2 of step s - 1
            const bool ok = wait_blocks<kNB>(bar, ph, waited, min(2 * s + 2, KB), cs.wait_ns);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) give_up<kNB>(J->cs, bar, ph, waited, issued);
                __syncthreads();
                return;
            }
            const int a = R + 2 * rp;  // even row of the thread
            const int o2 = roff(r3, 1), o1 = roff(r3, 2), o0 = roff(r3, 3), op = roff(r3, 4);
            const bool vp = (unsigned)(a + 1) < (unsigned)n, v0 = (unsigned)a < (unsigned)n,
                       v1 = (unsigned)(a - 1) < (unsigned)n;
            // theta' + P psi on rows a (even: coarse rows a/2 - 1, a/2 with weight 1/2) and
            // a + 1 (odd: coarse row a/2, weight 1); fine site gx + c takes the coarse columns
            // b - 1, b (c = 0), b (c = 1), b, b + 1 (c = 2), b + 1 (c = 3), b = gx / 2
            if (hasP) {
                const float* q0 = Pr + prow((a >> 1) - 1);
                const float* q1 = Pr + prow(a >> 1);
                const float p00 = q0[0], p01 = q0[1], p02 = q0[2], p10 = q1[0], p11 = q1[1], p12 = q1[2];
                if (v0) {
                    const float wy = 0.5f;
                    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
                    a0 += 1.0f * wy * 0.5f * p00;
                    a0 += 1.0f * wy * 0.5f * p01;
                    a1 += 1.0f * wy * 1.0f * p01;
                    a2 += 1.0f * wy * 0.5f * p01;
                    a2 += 1.0f * wy * 0.5f * p02;
                    a3 += 1.0f * wy * 1.0f * p02;
                    a0 += 1.0f * wy * 0.5f * p10;
                    a0 += 1.0f * wy * 0.5f * p11;
                    a1 += 1.0f * wy * 1.0f * p11;
                    a2 += 1.0f * wy * 0.5f * p11;
                    a2 += 1.0f * wy * 0.5f * p12;
                    a3 += 1.0f * wy * 1.0f * p12;
                    float4 x = ld4(Xr + o0);
                    x.x = x.x + a0;
                    x.y = p1 ? x.y + a1 : x.y;
                    x.z = p2 ? x.z + a2 : x.z;
                    x.w = p3 ? x.w + a3 : x.w;
                    st4(Xr + o0, x);
                }
                if (vp) {
                    const float wy = 1.0f;
                    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
                    a0 += 1.0f * wy * 0.5f * p10;
                    a0 += 1.0f * wy * 0.5f * p11;
                    a1 += 1.0f * wy * 1.0f * p11;
                    a2 += 1.0f * wy * 0.5f * p11;
                    a2 += 1.0f * wy * 0.5f * p12;
                    a3 += 1.0f * wy * 1.0f * p12;
                    float4 x = ld4(Xr + op);
                    x.x = x.x + a0;
                    x.y = p1 ? x.y + a1 : x.y;
                    x.z = p2 ? x.z + a2 : x.z;
                    x.w = p3 ? x.w + a3 : x.w;
                    st4(Xr + op, x);
                }
            }
            // alongside the prolongation: P3 of step s - 1 (rows up to R - 4; its neighbours are
            // final since the barrier)
            if (s > 0) p3_step(a - kK, wrap(r3 + kRing - kK, kRing), z30, z31);
            const Quad qa = draw_q(ctr, blk, K), qm = draw_q(ctr, blk - drow, K);
            {
                float* z = zx(s & 1, rp);
                z[0] = qa.a0;
                z[1] = qa.a1;
            }
            fence_proxy_async();
            __syncthreads();
            // blocks 2s - 2 and 2s - 1 were last read by P3 above: blocks 2s + 3, 2s + 4 take
            // their slots
            if (s > 0 && tid == 0)
                for (int k = 2 * s + 3; k <= min(2 * s + 4, KB); ++k) issue(k);
            if (s > 0) issued = max(issued, min(2 * s + 4, KB));
            // P3's even-column pair of row a - 2 (written before the barrier above; the slot is
            // written again two steps later, rp = 7's one step later)
            if (rp > 0 || s > 0) {
                const float* z = rp > 0 ? zx(s & 1, rp - 1) : zx((s + 1) & 1, kK / 2 - 1);
                z30 = z[0];
                z31 = z[1];
            } else {
                const Quad qu = draw_q(ctr, blk - 2 * drow, K);
                z30 = qu.a0;
                z31 = qu.a1;
            }
            // P0, colour (1,0), row a
            {
                Rows9 r;
                load9<1>(r, Xr, Cr, Fr, o1, o0, op);
                st4(Xr + o0, upd9<1>(r, qa.b0 * zs, qa.b1 * zs, v0 && c01, v0 && c03));
            }
            __syncthreads();
            // P1, colour (0,1), and P2, colour (1,1), on row a - 1
            Rows9 r;
            load9<0>(r, Xr, Cr, Fr, o2, o1, o0);
            r.x0 = upd9<0>(r, qm.a0 * zs, qm.a1 * zs, v1 && c10, v1 && c12);
            st4(Xr + o1, r.x0);
            __syncthreads();
            {
                // the right column of row a - 1 is the right group's P1 result
                r.exm = Xr[o2 + 4];
                r.ex0 = Xr[o1 + 4];
                r.exp = Xr[o0 + 4];
                r.c1e = 0.f;
                r.c4me = 0.f;
                r.c2me = Cr[2 * kFS + o2 + 4];
                const float4 o = upd9<1>(r, qm.b0 * zs, qm.b1 * zs, v1 && c21, v1 && c23);
                st4(Xr + o1, o);
                if (hasS && a - 1 >= ya && a - 1 < yb) st4(xout + pitch * (a - 1), o);
            }
            blk += dstep;
            r3 = wrap(r3 + kK, kRing);
        }
        __syncthreads();
        p3_step(ya - 4 + kK * (S - 1) + 2 * rp, wrap(r3 + kRing - kK, kRing), z30, z31);
    }
}

// 2D tiled map of a padded FP32 field: columns 0 .. n_cols - 1 (through the right
// ghost), rows 0 .. n_rows - 1 (both ghost rows), box bw x bh; reads outside are zero
bool encode9(CUtensorMap* m, const float* base, int pitch, int n_cols, int n_rows, int bw, int bh)
{
    EncodeTiled fn = tensor_map_encoder();
    if (!fn || !base) return false;
    cuuint64_t dims[2] = {(cuuint64_t)n_cols, (cuuint64_t)n_rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int g_s9_ctas = 0;  // resident CTAs per SM of the forward kernel (the larger one)
int g_s9_sms = 0;

}  // namespace

cudaError_t stream9_prepare()
{
    if (g_s9_ctas > 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_s9_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_stream9_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_stream9_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem);
    int nb = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stream9_fwd, kNT, kFwdSmem);
    if (e == cudaSuccess && !tensor_map_encoder()) e = cudaErrorNotSupported;
    if (e == cudaSuccess) g_s9_ctas = nb > 0 ? nb : 1;
    return e;
}

bool make_stream9_maps(const DevLevel<float>& L, const DevLevel<float>& C, Stream9Maps* out)
{
    std::memset(out, 0, sizeof(*out));
    const int cols = L.n + 5, rows = L.n + 2;
    bool ok = encode9(&out->x, L.x2, L.pitch, cols, rows, kBoxW, kBoxH);
    for (int t = 0; t < 5; ++t)
        ok = ok && encode9(&out->c[t], L.coef + (long long)t * L.alloc, L.pitch, cols, rows, kBoxW, kBoxH);
    ok = ok && encode9(&out->f, L.f, L.pitch, cols, rows, kBoxW, kBoxH);
    ok = ok && encode9(&out->p, C.x, C.pitch, C.n + 5, C.n + 2, kPBoxW, kPBoxH);
    return ok;
}

int stream9_grid(long long strips)
{
    const long long sms = g_s9_sms > 0 ? g_s9_sms : 1;
    const long long full = sms * (g_s9_ctas > 0 ? g_s9_ctas : 1);
    long long grid = strips >= 4 * full ? full : sms;
    if (grid > strips) grid = strips;
    return (int)std::max(1LL, grid);
}

void launch_stream9(const StreamJob* jobs, const Stream9Maps* maps, int njobs, long long strips, int grid, bool bwd,
                    cudaStream_t st, int& launches)
{
    if (strips <= 0 || grid <= 0) return;
    if (bwd)
        launch_pdl(k_stream9_bwd, dim3((unsigned)grid), dim3(kNT), kBwdSmem, st, jobs, maps, njobs, strips);
    else
        launch_pdl(k_stream9_fwd, dim3((unsigned)grid), dim3(kNT), kFwdSmem, st, jobs, maps, njobs, strips);
    ++launches;
}

}  // namespace mgmc
