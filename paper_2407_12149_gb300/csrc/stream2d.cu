// stream2d.cu -- the finest 2D grid (5-point stencil, FP32) streamed in bands.
//
// The finest grid of every chain is cut into bands of 128 columns and each band
// into strips of 16 rows.  A CTA owns a contiguous range of strips (spanning
// bands and chains where it must) and streams down each band it meets, one
// strip per pipeline step, through a ring of eight 8-row blocks of the state
// and of the operator field s kappa^2 in shared memory (the copies of a block
// are issued two steps before it is needed).  A block is one TMA box of
// 136 x 8 per field: the band's columns plus a 4-column halo on each
// side.  The phases of a step form a wavefront one row apart:
//   forward  red on rows [R, R+16), black on [R-1, R+15), residual
//            r = 0 - A theta*_s on [R-2, R+14), restriction f_c = P^T r of the
//            coarse rows whose three fine rows are complete, store of the final
//            rows [R-1, R+15) (Alg. 1 pre-smoothing and restriction, Alg. 3
//            sweep with ω = 1);
//   backward theta += P psi on [R, R+16), black on [R-1, R+15), red on
//            [R-2, R+14), store of the final rows [R-2, R+14) (Alg. 1
//            prolongation and post-smoothing, colours in reverse order); the
//            red phase of a step runs in the next step's first barrier
//            interval, beside that step's prolongation (their rows are
//            disjoint), so a step has two barriers;
// so every value a phase reads is the one a global colour sweep gives.  Only
// the first step of a run recomputes rows above the run, and across a band
// edge each colour phase updates the halo one column further than the next
// phase needs (the neighbouring band computes the same values: the noise is
// counter-based).
//
// The per-site arithmetic, the noise draws and the sums of the residual,
// restriction and prolongation are those of the tile kernels (tile2d.cu) in the
// same order, so both paths produce bitwise identical states.  The products
// w_t theta(site_t) of Alg. 3's z = B^T theta are not formed here: the low-rank
// kernel reads the state at the observation entries itself.
#include <algorithm>
#include <cstring>

#include "stencil.cuh"
#include "stream2d.cuh"
#include "stream_core.cuh"
#include "tma.cuh"

namespace mgmc {

namespace {

using namespace sc;

constexpr int kBW = kStreamBand;
constexpr int kK = kStreamRows;
constexpr int kNG = kBW / 4 + 2;   // 4-site groups per staged row: one halo group on each side
constexpr int kNT = kNG * kK / 2;  // threads: one group of two adjacent rows each
constexpr int kSX = 4 * kNG;       // staged row (floats)
constexpr int kBK = kK / 2;        // rows per TMA block (two blocks per step)
constexpr int kNB = 8;             // ring slots (blocks)
constexpr int kRing = kNB * kBK;   // rows of the state and operator rings
constexpr int kRW = kBW + 4;       // residual row: the groups of columns x0 .. x0 + kBW + 3
constexpr int kRRing = 64;         // rows of the residual ring
constexpr int kPX = kBW / 2 + 8;   // staged coarse columns
constexpr int kPK = kBK / 2;       // coarse rows per block
constexpr int kPRing = kNB * kPK;  // rows of the psi ring
// TMA boxes (columns x rows) and the bytes each delivers: the tensor maps and the
// mbarrier's expected transaction bytes both use these
constexpr int kBoxW = kSX, kBoxH = kBK, kPBoxW = kPX, kPBoxH = kPK;
constexpr unsigned kBox = kBoxW * kBoxH * 4;
constexpr unsigned kPBox = kPBoxW * kPBoxH * 4;
constexpr size_t kHead = 256;      // mbarriers; also keeps the reads one float left of the ring inside shared memory
// hand-off of site normals between the threads of consecutive rows: [step parity][rp][g][2]
constexpr int kZx = 2 * (kK / 2) * kNG * 2;
constexpr size_t kFwdSmem = 128 + kHead + 4 * (2 * (size_t)kRing * kSX + (size_t)kRRing * kRW + kZx);
constexpr size_t kBwdSmem = 128 + kHead + 4 * (2 * (size_t)kRing * kSX + (size_t)kPRing * kPX + kZx);
static_assert(kNT <= 1024 && kNT >= 8 * 32, "thread layout: the restriction needs 8 x 32 threads");
static_assert(kRing == 64 && kRRing == 64 && kPRing == 32 && kNB == 8, "power-of-two rings");
static_assert(kBox % 128 == 0 && kPBox % 128 == 0, "TMA destinations on 128-byte boundaries");
static_assert(kSX <= 256 && kPX <= 256 && (kSX * 4) % 16 == 0 && (kPX * 4) % 16 == 0, "TMA box");
static_assert(kNB * 8 <= (int)kHead, "mbarriers");

// The two same-colour sites (components PX and PX + 2) of a 4-site group r0, given
// the group one row above (ru) and below (rd), s kappa^2 of the group (c) and the
// column outside the group (e: left of the group for PX = 0, right for PX = 1);
// the other two components (the other colour) are returned unchanged.
template <int PX>
__device__ __forceinline__ float4 gibbs_upd(float4 r0, float4 ru, float4 rd, float4 c, float e, float w, float z0,
                                            float z1, bool v0, bool v1)
{
    float4 r = r0;
    if (PX == 0) {
        const float na = fine_site(r0.x, ru.x, e, r0.y, rd.x, c.x, w, z0);
        const float nb = fine_site(r0.z, ru.z, r0.y, r0.w, rd.z, c.z, w, z1);
        r.x = v0 ? na : r.x;
        r.z = v1 ? nb : r.z;
    } else {
        const float na = fine_site(r0.y, ru.y, r0.x, r0.z, rd.y, c.y, w, z0);
        const float nb = fine_site(r0.w, ru.w, r0.z, e, rd.w, c.w, w, z1);
        r.y = v0 ? na : r.y;
        r.w = v1 ? nb : r.w;
    }
    return r;
}

// r = 0 - A theta of the 4 sites of the group r0 (el, er: the columns left and right of it)
__device__ __forceinline__ float4 residual4(float4 r0, float4 ru, float4 rd, float4 c, float el, float er, float w)
{
    return make_float4(0.0f - fine_ax(r0.x, ru.x, el, r0.y, rd.x, c.x, w),
                       0.0f - fine_ax(r0.y, ru.y, r0.x, r0.z, rd.y, c.y, w),
                       0.0f - fine_ax(r0.z, ru.z, r0.y, r0.w, rd.z, c.z, w),
                       0.0f - fine_ax(r0.w, ru.w, r0.z, er, rd.w, c.w, w));
}

// Forward pass of the finest grids: one launch over all strips of all chains.
__global__ void __launch_bounds__(kNT, 2)
    k_stream_fwd(const StreamJob* __restrict__ jobs, const StreamMaps* __restrict__ maps, int njobs, long long total)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* sm = smem_align_up<128>(smem_dyn);
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm);
    float* const Xr = reinterpret_cast<float*>(sm + kHead);
    float* const Kr = Xr + kRing * kSX;
    float* const Rr = Kr + kRing * kSX;
    float* const Zx = Rr + kRRing * kRW;
    const int tid = threadIdx.x;
    const int g = tid % kNG, rp = tid / kNG;  // group g of rows R + 2 rp (even) and R + 2 rp + 1 of each step
    pdl_launch_dependents();
    if (tid == 0) {
        for (int q = 0; q < kNB; ++q) mbar_init(&bar[q]);
        fence_mbar_init();
    }
    __syncthreads();
    pdl_wait();
    const long long s_beg = total * blockIdx.x / gridDim.x, s_end = total * (blockIdx.x + 1) / gridDim.x;
    unsigned ph = 0;  // bit q: parity of the next phase of mbarrier q
    for (long long gs = s_beg; gs < s_end;) {
        const Run run = next_run<kK, kBW>(jobs, njobs, gs, s_end);
        const StreamJob* J = jobs + run.jb;
        const int n = run.n, nc = run.nc, x0 = run.x0, ya = run.ya, yb = run.yb;
        // coarse rows J with centre row 2J + 1 in [ya, yb)
        const int jend = yb >> 1;
        // steps: step s completes rows [ya - 3 + 16 s, ya + 13 + 16 s); the coarse rows
        // [ya/2 - 3 + 8 s, ya/2 + 5 + 8 s) are restricted once step s is complete
        const int S = max(max(cdiv_pos(yb - ya - (kK - 2), kK), cdiv_pos(jend - (ya >> 1) - (kK / 2 - 3), kK / 2)) + 1, 1);
        const int KB = 2 * S;  // last block: rows [ya - 3 + 8 KB, ya + 5 + 8 KB)
        const float w = J->L.woff;
        const CycleState cs = *J->cs;
        const uint4 ctr = noise_counter(cs, 0u, 0u, J->L.level, 0u);
        const RoundKeys K = round_keys((unsigned)cs.seed, (unsigned)(cs.seed >> 32));
        const float zs = cs.noise ? 1.0f : 0.0f;
        const int nq = (n + 3) >> 2;
        const int gx = x0 - 4 + 4 * g;  // first column of the thread's group
        auto col = [&](int i, int lo, int hi) { return i >= lo && i <= hi && i >= 0 && i < n; };
        // columns each colour must update: red [x0-2, x0+kBW+2], black [x0-1, x0+kBW+1];
        // parity-0 sites gx, gx + 2 (even rows), parity-1 sites gx + 1, gx + 3 (odd rows)
        const bool cr0 = col(gx, x0 - 2, x0 + kBW + 2), cr1 = col(gx + 2, x0 - 2, x0 + kBW + 2);
        const bool cr2 = col(gx + 1, x0 - 2, x0 + kBW + 2), cr3 = col(gx + 3, x0 - 2, x0 + kBW + 2);
        const bool cb0 = col(gx, x0 - 1, x0 + kBW + 1), cb1 = col(gx + 2, x0 - 1, x0 + kBW + 1);
        const bool cb2 = col(gx + 1, x0 - 1, x0 + kBW + 1), cb3 = col(gx + 3, x0 - 1, x0 + kBW + 1);
        // site-noise block of the thread's even row in step 0 (row ya - 2 + 2 rp, group gx / 4);
        // the block of the row below is nq further.  A block gives the even columns' pair
        // (red on an even row, black on an odd one) and the odd columns' pair
        unsigned blk = (unsigned)((long long)(ya - 2 + 2 * rp) * nq + (gx >> 2));
        const unsigned dstep = (unsigned)(kK * nq), drow = (unsigned)nq;
        // the even-column pair of the odd row below: black there, which is the next row
        // pair's thread (rp + 1, or rp = 0 of the next step) -- handed over in Zx
        auto zx = [&](int par, int r) { return Zx + ((par * (kK / 2) + r) * kNG + g) * 2; };
        const bool hasR = g >= 1;
        const bool rin = gx < n, r1 = gx + 1 < n, r2 = gx + 2 < n, r3 = gx + 3 < n;
        const bool hasS = g >= 1 && g <= kBW / 4 && gx < n;  // the band's own columns
        const int ci = tid & 31, cj = tid >> 5;  // restriction: coarse columns I, I + 1, coarse row R/2 - 2 + cj
        const int I = (x0 >> 1) + 2 * ci;
        const bool hasC = tid < 8 * 32 && I < nc;
        const bool pairC = I + 1 < nc;
        float* const xout = J->L.x2 + J->L.base + gx;
        const long long pitch = J->L.pitch;
        float* const fc = J->C.f + J->C.base + I;
        const long long cpitch = J->C.pitch;
        auto xrow = [&](int j) { return ((j - ya + 3) & (kRing - 1)) * kSX + 4 * g; };
        auto rrow = [&](int j) { return ((j - ya + 4) & (kRRing - 1)) * kRW; };
        // restriction of the coarse rows of step t: f_c = sum_p w(p) r(2I + p), fine columns 2I .. 2I + 4
        auto restrict_step = [&](int t) {
            const int Jc = ((ya - 2 + kK * t) >> 1) - 2 + cj;
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
        const CUtensorMap* mx = &maps[run.jb].x;
        const CUtensorMap* mk = &maps[run.jb].k;
        // block k: rows [ya - 3 + 8 k, ya + 5 + 8 k) of the state and the operator
        auto issue = [&](int k) {
            const int q = k & (kNB - 1);
            mbar_expect_tx(&bar[q], 2 * kBox);
            const int prow = ya - 3 + kBK * k + 1;
            tma_load_2d(Xr + q * kBK * kSX, mx, x0, prow, &bar[q]);
            tma_load_2d(Kr + q * kBK * kSX, mk, x0, prow, &bar[q]);
        };
        // the rings are free: every thread is done with the previous run
        fence_proxy_async();
        __syncthreads();
        int issued = min(KB, 4), waited = -1;
        if (tid == 0)
            for (int k = 0; k <= issued; ++k) issue(k);
        for (int s = 0; s < S; ++s) {
            const int R = ya - 2 + kK * s;
            // blocks up to 2s + 2 (rows up to R + 16) are in shared memory
            const bool ok = wait_blocks<kNB>(bar, ph, waited, min(2 * s + 2, KB), cs.wait_ns);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) give_up<kNB>(J->cs, bar, ph, waited, issued);
                __syncthreads();
                return;
            }
            // blocks 2s - 3 and 2s - 2 are no longer read: blocks 2s + 5, 2s + 6 go into their slots
            if (tid == 0)
                for (int k = 2 * s + 5; k <= min(2 * s + 6, KB); ++k) issue(k);
            issued = max(issued, min(2 * s + 6, KB));
            const int ja = R + 2 * rp;  // even row of the thread
            const int oY = xrow(ja - 3), oZ = xrow(ja - 2), oA = xrow(ja - 1), oB = xrow(ja), oC = xrow(ja + 1),
                      oD = xrow(ja + 2);
            const bool va = (unsigned)ja < (unsigned)n, vb = (unsigned)(ja + 1) < (unsigned)n,
                       vu = (unsigned)(ja - 1) < (unsigned)n, vz = (unsigned)(ja - 2) < (unsigned)n;
            // red on rows ja (parity 0: the even columns' pair of its block) and ja + 1
            // (parity 1: the odd columns' pair); the other halves are black's
            const Quad qa = draw_q(ctr, blk, K), qb = draw_q(ctr, blk + drow, K);
            {
                float* z = zx(s & 1, rp);
                z[0] = qb.a0;
                z[1] = qb.a1;
                const float4 ra = ld4(Xr + oB), rb = ld4(Xr + oC), ru = ld4(Xr + oA), rd = ld4(Xr + oD);
                const float4 ca = ld4(Kr + oB), cb = ld4(Kr + oC);
                const float ea = Xr[oB - 1], eb = Xr[oC + 4];
                st4(Xr + oB, gibbs_upd<0>(ra, ru, rb, ca, ea, w, qa.a0 * zs, qa.a1 * zs, va && cr0, va && cr1));
                st4(Xr + oC, gibbs_upd<1>(rb, ra, rd, cb, eb, w, qb.b0 * zs, qb.b1 * zs, vb && cr2, vb && cr3));
            }
            __syncthreads();
            // black on rows ja - 1 (parity 0) and ja (parity 1); then their final states
            {
                // row ja - 1's block: the thread above (rp - 1, or rp = 7 of the previous step)
                // drew it; at the start of a run it is drawn here
                float z0, z1;
                if (rp > 0 || s > 0) {
                    const float* z = rp > 0 ? zx(s & 1, rp - 1) : zx((s + 1) & 1, kK / 2 - 1);
                    z0 = z[0];
                    z1 = z[1];
                } else {
                    const Quad qu = draw_q(ctr, blk - drow, K);
                    z0 = qu.a0;
                    z1 = qu.a1;
                }
                const float z2 = qa.b0, z3 = qa.b1;
                const float4 ra = ld4(Xr + oA), rb = ld4(Xr + oB), ru = ld4(Xr + oZ), rd = ld4(Xr + oC);
                const float4 ca = ld4(Kr + oA), cb = ld4(Kr + oB);
                const float ea = Xr[oA - 1], eb = Xr[oB + 4];
                const float4 na = gibbs_upd<0>(ra, ru, rb, ca, ea, w, z0 * zs, z1 * zs, vu && cb0, vu && cb1);
                const float4 nb = gibbs_upd<1>(rb, ra, rd, cb, eb, w, z2 * zs, z3 * zs, va && cb2, va && cb3);
                st4(Xr + oA, na);
                st4(Xr + oB, nb);
                if (hasS && ja - 1 >= ya && ja - 1 < yb) st4(xout + pitch * (ja - 1), na);
                if (hasS && ja >= ya && ja < yb) st4(xout + pitch * ja, nb);
            }
            __syncthreads();
            // residual on rows ja - 2 and ja - 1 (0 outside the grid)
            if (hasR) {
                const float4 xy = ld4(Xr + oY), xz = ld4(Xr + oZ), xa = ld4(Xr + oA), xb = ld4(Xr + oB);
                const float4 kz = ld4(Kr + oZ), ka = ld4(Kr + oA);
                const float ezl = Xr[oZ - 1], ezr = Xr[oZ + 4], eal = Xr[oA - 1], ear = Xr[oA + 4];
                float4 rz = make_float4(0.f, 0.f, 0.f, 0.f), ra = rz;
                if (rin && vz) rz = residual4(xz, xy, xa, kz, ezl, ezr, w);
                if (rin && vu) ra = residual4(xa, xz, xb, ka, eal, ear, w);
                rz.y = r1 ? rz.y : 0.f;
                rz.z = r2 ? rz.z : 0.f;
                rz.w = r3 ? rz.w : 0.f;
                ra.y = r1 ? ra.y : 0.f;
                ra.z = r2 ? ra.z : 0.f;
                ra.w = r3 ? ra.w : 0.f;
                st4(Rr + rrow(ja - 2) + 4 * (g - 1), rz);
                st4(Rr + rrow(ja - 1) + 4 * (g - 1), ra);
            }
            // the coarse rows of the previous step (its residual rows are complete)
            if (s > 0) restrict_step(s - 1);
            fence_proxy_async();
            blk += dstep;
        }
        __syncthreads();
        restrict_step(S - 1);
    }
}

// Backward pass of the finest grids: one launch over all strips of all chains.
__global__ void __launch_bounds__(kNT, 2)
    k_stream_bwd(const StreamJob* __restrict__ jobs, const StreamMaps* __restrict__ maps, int njobs, long long total)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* sm = smem_align_up<128>(smem_dyn);
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm);
    float* const Xr = reinterpret_cast<float*>(sm + kHead);
    float* const Kr = Xr + kRing * kSX;
    float* const Pr = Kr + kRing * kSX;
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
        // step s completes rows [ya - 4 + 16 s, ya + 12 + 16 s)
        const int S = cdiv_pos(yb - ya - (kK - 4), kK) + 1;
        const int KB = 2 * S;  // last block: rows [ya - 2 + 8 KB, ...), coarse rows [ya/2 - 2 + 4 KB, ...)
        const float w = J->L.woff;
        const CycleState cs = *J->cs;
        const uint4 ctr = noise_counter(cs, 0u, 0u, J->L.level, 1u);
        const RoundKeys K = round_keys((unsigned)cs.seed, (unsigned)(cs.seed >> 32));
        const float zs = cs.noise ? 1.0f : 0.0f;
        const int nq = (n + 3) >> 2;
        const int gx = x0 - 4 + 4 * g;
        auto col = [&](int i, int lo, int hi) { return i >= lo && i <= hi && i >= 0 && i < n; };
        // columns each colour must update: black [x0-1, x0+kBW], red [x0, x0+kBW-1]
        const bool cb0 = col(gx, x0 - 1, x0 + kBW), cb1 = col(gx + 2, x0 - 1, x0 + kBW);
        const bool cb2 = col(gx + 1, x0 - 1, x0 + kBW), cb3 = col(gx + 3, x0 - 1, x0 + kBW);
        const bool cr0 = col(gx, x0, x0 + kBW - 1), cr1 = col(gx + 2, x0, x0 + kBW - 1);
        const bool cr2 = col(gx + 1, x0, x0 + kBW - 1), cr3 = col(gx + 3, x0, x0 + kBW - 1);
        // site-noise block of the thread's odd row ja - 1 in step 0 (row ya - 3 + 2 rp, group
        // gx / 4); the even row ja below it is nq further.  Black takes the even columns'
        // pair of row ja - 1 and the odd columns' pair of row ja; red the odd columns' pair
        // of row ja - 1 and the even columns' pair of row ja - 2, which the thread above
        // (rp - 1, or rp = 7 of the previous step) drew as its row ja and hands over in Zx
        unsigned blk = (unsigned)((long long)(ya - 3 + 2 * rp) * nq + (gx >> 2));
        const unsigned dstep = (unsigned)(kK * nq), drow = (unsigned)nq;
        auto zx = [&](int par, int r) { return Zx + ((par * (kK / 2) + r) * kNG + g) * 2; };
        const bool hasP = gx >= 0 && gx < n;
        const bool p1 = gx + 1 < n, p2 = gx + 2 < n, p3 = gx + 3 < n;
        const bool hasS = g >= 1 && g <= kBW / 4 && gx < n;
        float* const xout = J->L.x + J->L.base + gx;
        const long long pitch = J->L.pitch;
        const int jcb = (ya >> 1) - 2;  // first coarse row of psi block 0
        auto xrow = [&](int j) { return ((j - ya + 2) & (kRing - 1)) * kSX + 4 * g; };
        auto prow = [&](int jc) { return ((jc - jcb) & (kPRing - 1)) * kPX + 2 * g + 1; };
        const CUtensorMap* mx = &maps[run.jb].x;
        const CUtensorMap* mk = &maps[run.jb].k;
        const CUtensorMap* mp = &maps[run.jb].p;
        // block k: rows [ya - 2 + 8 k, ya + 6 + 8 k) of the state and the operator,
        // coarse rows [jcb + 4 k, jcb + 4 k + 4) of psi, coarse columns from x0/2 - 4
        auto issue = [&](int k) {
            const int q = k & (kNB - 1);
            mbar_expect_tx(&bar[q], 2 * kBox + kPBox);
            const int prw = ya - 2 + kBK * k + 1;
            tma_load_2d(Xr + q * kBK * kSX, mx, x0, prw, &bar[q]);
            tma_load_2d(Kr + q * kBK * kSX, mk, x0, prw, &bar[q]);
            tma_load_2d(Pr + q * kPK * kPX, mp, x0 >> 1, jcb + kPK * k + 1, &bar[q]);
        };
        // red on step t's rows ja - 2 (even, parity 0) and ja - 1 (odd, parity 1) with the
        // noise z; then their final states
        auto red_step = [&](int t, float z0, float z1, float z2, float z3) {
            const int ja = ya - 2 + kK * t + 2 * rp;
            const int oZ = xrow(ja - 3), oA = xrow(ja - 2), oB = xrow(ja - 1), oC = xrow(ja);
            const bool va = (unsigned)(ja - 2) < (unsigned)n, vb = (unsigned)(ja - 1) < (unsigned)n;
            const float4 ra = ld4(Xr + oA), rb = ld4(Xr + oB), ru = ld4(Xr + oZ), rd = ld4(Xr + oC);
            const float4 ca = ld4(Kr + oA), cb = ld4(Kr + oB);
            const float ea = Xr[oA - 1], eb = Xr[oB + 4];
            const float4 na = gibbs_upd<0>(ra, ru, rb, ca, ea, w, z0 * zs, z1 * zs, va && cr0, va && cr1);
            const float4 nb = gibbs_upd<1>(rb, ra, rd, cb, eb, w, z2 * zs, z3 * zs, vb && cr2, vb && cr3);
            st4(Xr + oA, na);
            st4(Xr + oB, nb);
            if (hasS && ja - 2 >= ya && ja - 2 < yb) st4(xout + pitch * (ja - 2), na);
            if (hasS && ja - 1 >= ya && ja - 1 < yb) st4(xout + pitch * (ja - 1), nb);
        };
        fence_proxy_async();
        __syncthreads();
        int issued = min(KB, 4), waited = -1;
        if (tid == 0)
            for (int k = 0; k <= issued; ++k) issue(k);
        // noise drawn one barrier interval ahead of its use: the two blocks of step s in the
        // first interval of step s (of step 0 here); red's hand-over read in the black phase
        float zb0, zb1, zb2, zb3, zr0 = 0.f, zr1 = 0.f, zr2 = 0.f, zr3 = 0.f;
        auto draw_step = [&](int s) {
            const Quad qm = draw_q(ctr, blk, K), qo = draw_q(ctr, blk + drow, K);
            zb0 = qm.a0;
            zb1 = qm.a1;
            zb2 = qo.b0;
            zb3 = qo.b1;
            zr2 = qm.b0;
            zr3 = qm.b1;
            float* z = zx(s & 1, rp);
            z[0] = qo.a0;
            z[1] = qo.a1;
        };
        draw_step(0);
        for (int s = 0; s < S; ++s) {
            const int R = ya - 2 + kK * s;
            // blocks up to 2s + 2 (psi of row R + 15) are in shared memory; the barrier also
            // ends the black phase of step s - 1
            const bool ok = wait_blocks<kNB>(bar, ph, waited, min(2 * s + 2, KB), cs.wait_ns);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) give_up<kNB>(J->cs, bar, ph, waited, issued);
                __syncthreads();
                return;
            }
            const int ja = R + 2 * rp;  // even row of the thread
            const int oA = xrow(ja - 2), oB = xrow(ja - 1), oC = xrow(ja), oD = xrow(ja + 1);
            const bool vc = (unsigned)ja < (unsigned)n, vd = (unsigned)(ja + 1) < (unsigned)n,
                       vb = (unsigned)(ja - 1) < (unsigned)n;
            // theta' + P psi on rows ja (even: coarse rows ja/2 - 1, ja/2 with weight 1/2) and
            // ja + 1 (odd: coarse row ja/2, weight 1); fine site gx + c takes the coarse columns
            // a - 1, a (c = 0), a (c = 1), a, a + 1 (c = 2), a + 1 (c = 3), a = gx / 2.
            // Alongside, the red phase of step s - 1 (rows up to R - 3; its black neighbours are
            // final since the barrier)
            if (hasP) {
                const float* q0 = Pr + prow((ja >> 1) - 1);
                const float* q1 = Pr + prow(ja >> 1);
                const float p00 = q0[0], p01 = q0[1], p02 = q0[2], p10 = q1[0], p11 = q1[1], p12 = q1[2];
                if (vc) {
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
                    float4 x = ld4(Xr + oC);
                    x.x = x.x + a0;
                    x.y = p1 ? x.y + a1 : x.y;
                    x.z = p2 ? x.z + a2 : x.z;
                    x.w = p3 ? x.w + a3 : x.w;
                    st4(Xr + oC, x);
                }
                if (vd) {
                    const float wy = 1.0f;
                    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
                    a0 += 1.0f * wy * 0.5f * p10;
                    a0 += 1.0f * wy * 0.5f * p11;
                    a1 += 1.0f * wy * 1.0f * p11;
                    a2 += 1.0f * wy * 0.5f * p11;
                    a2 += 1.0f * wy * 0.5f * p12;
                    a3 += 1.0f * wy * 1.0f * p12;
                    float4 x = ld4(Xr + oD);
                    x.x = x.x + a0;
                    x.y = p1 ? x.y + a1 : x.y;
                    x.z = p2 ? x.z + a2 : x.z;
                    x.w = p3 ? x.w + a3 : x.w;
                    st4(Xr + oD, x);
                }
            }
            if (s > 0) {
                red_step(s - 1, zr0, zr1, zr2, zr3);
                draw_step(s);
            }
            fence_proxy_async();
            __syncthreads();
            // blocks 2s - 3 and 2s - 2 were last read by the red phase above: blocks 2s + 5,
            // 2s + 6 go into their slots
            if (tid == 0)
                for (int k = 2 * s + 5; k <= min(2 * s + 6, KB); ++k) issue(k);
            issued = max(issued, min(2 * s + 6, KB));
            // black on rows ja - 1 (odd, parity 0) and ja (even, parity 1)
            {
                const float4 ra = ld4(Xr + oB), rb = ld4(Xr + oC), ru = ld4(Xr + oA), rd = ld4(Xr + oD);
                const float4 ca = ld4(Kr + oB), cb = ld4(Kr + oC);
                const float ea = Xr[oB - 1], eb = Xr[oC + 4];
                st4(Xr + oB, gibbs_upd<0>(ra, ru, rb, ca, ea, w, zb0 * zs, zb1 * zs, vb && cb0, vb && cb1));
                st4(Xr + oC, gibbs_upd<1>(rb, ra, rd, cb, eb, w, zb2 * zs, zb3 * zs, vc && cb2, vc && cb3));
            }
            // red's even-column pair of row ja - 2 (written before the barrier above; the
            // slot is written again two steps later, rp = 7's one step later)
            if (rp > 0 || s > 0) {
                const float* z = rp > 0 ? zx(s & 1, rp - 1) : zx((s + 1) & 1, kK / 2 - 1);
                zr0 = z[0];
                zr1 = z[1];
            } else {
                const Quad qu = draw_q(ctr, blk - drow, K);
                zr0 = qu.a0;
                zr1 = qu.a1;
            }
            blk += dstep;
        }
        __syncthreads();
        red_step(S - 1, zr0, zr1, zr2, zr3);
    }
}

// 2D tiled map of a padded FP32 field: columns 0 .. n_cols - 1 (through the right
// ghost), rows 0 .. n_rows - 1 (both ghost rows), box bw x bh; reads outside are zero
bool encode_padded(CUtensorMap* m, const float* base, int pitch, int n_cols, int n_rows, int bw, int bh)
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

int g_stream_ctas = 0;  // resident CTAs per SM of the forward kernel (the larger one)
int g_stream_sms = 0;

}  // namespace

cudaError_t stream_prepare()
{
    if (g_stream_ctas > 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_stream_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_stream_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_stream_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem);
    int nb = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stream_fwd, kNT, kFwdSmem);
    if (e == cudaSuccess && !tensor_map_encoder()) e = cudaErrorNotSupported;
    if (e == cudaSuccess) g_stream_ctas = nb > 0 ? nb : 1;
    return e;
}

bool make_stream_maps(const DevLevel<float>& L, const DevLevel<float>& C, bool bwd, StreamMaps* out)
{
    std::memset(out, 0, sizeof(*out));
    bool ok = encode_padded(&out->x, bwd ? L.x2 : L.x, L.pitch, L.n + 5, L.n + 2, kBoxW, kBoxH) &&
              encode_padded(&out->k, L.diag, L.pitch, L.n + 5, L.n + 2, kBoxW, kBoxH);
    if (bwd) ok = ok && encode_padded(&out->p, C.x, C.pitch, C.n + 5, C.n + 2, kPBoxW, kPBoxH);
    return ok;
}

int stream_grid(long long strips)
{
    const long long sms = g_stream_sms > 0 ? g_stream_sms : 1;
    const long long full = sms * (g_stream_ctas > 0 ? g_stream_ctas : 1);
    // every run costs about one step of pipeline fill: with few strips per SM one
    // CTA per SM keeps the runs long, with many the second CTA hides latency
    long long grid = strips >= 8 * full ? full : sms;
    if (grid > strips) grid = strips;
    return (int)std::max(1LL, grid);
}

void launch_stream_fine(const StreamJob* jobs, const StreamMaps* maps, int njobs, long long strips, int grid,
                        bool bwd, cudaStream_t st, int& launches)
{
    if (strips <= 0 || grid <= 0) return;
    if (bwd)
        launch_pdl(k_stream_bwd, dim3((unsigned)grid), dim3(kNT), kBwdSmem, st, jobs, maps, njobs, strips);
    else
        launch_pdl(k_stream_fwd, dim3((unsigned)grid), dim3(kNT), kFwdSmem, st, jobs, maps, njobs, strips);
    ++launches;
}

}  // namespace mgmc
