// stream_core.cuh -- pieces shared by the streaming band kernels (stream2d.cu,
// stream9.cu): the strip schedule, the bounded waits on the TMA ring, and the
// Philox4x32-10 draws with round keys computed once per run.
#pragma once
#include "common.cuh"
#include "stream2d.cuh"
#include "tma.cuh"

namespace mgmc {
namespace sc {

__device__ __forceinline__ int cdiv_pos(int a, int b) { return a > 0 ? (a + b - 1) / b : 0; }

__device__ __forceinline__ int find_stream_job(const StreamJob* jobs, int njobs, long long s)
{
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].strip0 <= s)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// Philox4x32-10 round keys of one key (Weyl schedule), computed once per run so that
// the rounds do not recompute them; the same block as philox10 of common.cuh
struct RoundKeys {
    unsigned a[10], b[10];
};
__device__ __forceinline__ RoundKeys round_keys(unsigned k0, unsigned k1)
{
    RoundKeys K;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        K.a[r] = k0;
        K.b[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return K;
}
__device__ __forceinline__ uint4 philox_k(uint4 c, unsigned block, const RoundKeys& K)
{
    c.x = block;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((unsigned)(p1 >> 32) ^ c.y ^ K.a[r], (unsigned)p1, (unsigned)(p0 >> 32) ^ c.w ^ K.b[r],
                       (unsigned)p0);
    }
    return c;
}
// the four site normals of one block (normal_quad of common.cuh)
struct Quad {
    float a0, a1, b0, b1;  // a: the even columns of the group, b: the odd ones
};
__device__ __forceinline__ Quad draw_q(uint4 c, unsigned block, const RoundKeys& K)
{
    Quad q;
    normal_quad(philox_k(c, block, K), q.a0, q.a1, q.b0, q.b1);
    return q;
}
// wait (bounded) for blocks (waited, upto] of a ring of NB slots (bit q of ph: the parity of
// slot q's next phase); false if a wait gave up
template <int NB>
__device__ __forceinline__ bool wait_blocks(unsigned long long* bar, unsigned& ph, int& waited, int upto,
                                            long long limit_ns)
{
    while (waited < upto) {
        const int q = (waited + 1) % NB;
        if (!mbar_wait(&bar[q], (ph >> q) & 1u, limit_ns)) return false;
        ph ^= 1u << q;
        ++waited;
    }
    return true;
}

// a wait gave up: flag the chain (MGMC_ERR_TIMEOUT) and let the copies in flight land
template <int NB>
__device__ __forceinline__ void give_up(CycleState* cs, unsigned long long* bar, unsigned ph, int waited, int issued)
{
    atomicOr(&cs->status, kStatusTimeout);
    __threadfence();
    for (int k = waited + 1; k <= issued; ++k) {
        const int q = k % NB;
        if (mbar_wait(&bar[q], (ph >> q) & 1u)) ph ^= 1u << q;
    }
}

// the run of a CTA: strips [gs, ge) of one band of chain jb, rows [ya, yb) (strips of K rows,
// bands of BW columns)
struct Run {
    int jb, n, nc, x0, ya, yb;
};
template <int K, int BW>
__device__ __forceinline__ Run next_run(const StreamJob* jobs, int njobs, long long& gs, long long s_end)
{
    Run r;
    r.jb = find_stream_job(jobs, njobs, gs);
    const StreamJob* J = jobs + r.jb;
    r.n = J->L.n;
    r.nc = J->C.n;
    const int ls = (int)(gs - J->strip0);
    const int band = ls / J->spb, st0 = ls % J->spb;
    const long long ge = min(s_end, J->strip0 + (long long)(band + 1) * J->spb);
    r.ya = K * st0;
    r.yb = min(K * (st0 + (int)(ge - gs)), r.n);
    r.x0 = BW * band;
    gs = ge;
    return r;
}

}  // namespace sc
}  // namespace mgmc
