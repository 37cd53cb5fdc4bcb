// tma.cuh -- device helpers for TMA bulk tensor copies and mbarriers (PTX ISA:
// cp.async.bulk.tensor, mbarrier.*).  Every wait is bounded in time.
#pragma once
#include <cuda.h>
#include <cstdint>

namespace mgmc {

// host: cuTensorMapEncodeTiled, looked up once through the runtime's driver
// entry-point query (no link against the driver library); NULL if unavailable
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled tensor_map_encoder();

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
// p advanced to the next multiple of A bytes (A a power of two), by pointer arithmetic
// on the shared array itself: rounding the generic address as an integer would make
// the compiler lose the address space and turn every access through the result into
// a generic load or store
template <unsigned A>
__device__ __forceinline__ unsigned char* smem_align_up(unsigned char* p)
{
    return p + ((A - (smem_addr(p) & (A - 1u))) & (A - 1u));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// wait for the completion of the barrier phase of the given parity; false once the
// bound has passed (limit_ns: 0 the default 1 s, > 0 that many ns, < 0 give up at
// once -- a test of the give-up path; the drains after a give-up use the default)
constexpr unsigned long long kWaitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long long limit_ns = 0)
{
    if (limit_ns < 0) return false;
    const unsigned long long bound = limit_ns > 0 ? (unsigned long long)limit_ns : kWaitNs;
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1; it < (1u << 30); ++it) {
        if (mbar_test(bar, parity)) return true;
        if ((it & 63) == 0 && global_ns() - t0 > bound) return false;
    }
    return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];\n" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}
// orders this thread's generic-proxy accesses of shared memory before later
// async-proxy (TMA) writes to it
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_init_count(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

}  // namespace mgmc
