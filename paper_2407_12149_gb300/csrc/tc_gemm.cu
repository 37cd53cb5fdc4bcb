// tc_gemm.cu -- BF16 GEMM on the 5th-generation (tcgen05) tensor cores:
//   C[M][N] = A[M][K] * B[N][K]^T, FP32 accumulation in tensor memory (TMEM).
//
// One CTA of 128 threads computes a 128 x BN tile of C:
//   warp 0, lane 0: TMA producer -- 128 x 64 tiles of A and BN x 64 tiles of B
//                   (128-byte swizzled, the layout the MMA descriptors name) into
//                   a 4-stage ring, each stage completing on a "full" mbarrier;
//   warp 1, lane 0: MMA issuer -- 4 x tcgen05.mma (M = 128, N = BN, K = 16) per
//                   stage into the TMEM accumulator, then tcgen05.commit to the
//                   stage's "empty" mbarrier (frees the stage when the MMAs are done);
//   all 4 warps:    epilogue -- warp w reads TMEM lanes 32w .. 32w + 31 (rows of
//                   the tile) with tcgen05.ld and stores them with the epilogue ops.
// Every mbarrier wait is bounded (1 s); a wait that gives up sets *status = 2,
// the CTA waits (bounded) for its own copies in flight, frees its TMEM and ends.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "tc_gemm.cuh"
#include "tma.cuh"

namespace mgmc {

namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;        // one 128-byte swizzle row of BF16
constexpr int kStages = 4;
constexpr int kThreads = 128;

// --- tcgen05 helpers (PTX ISA, "Tensor Core 5th Generation Family Instructions") ---

// shared-memory matrix descriptor of a K-major operand tile stored in the
// 128-byte-swizzled layout (rows of 128 bytes, 8-row groups 1024 bytes apart):
// start address >> 4 (bits 0-13), leading byte offset >> 4 (bits 16-29; not used
// by swizzled K-major layouts, set to 1), stride byte offset >> 4 = 1024 >> 4
// (bits 32-45), descriptor version 1 (bits 46-47), swizzle mode 2 = 128 B (bits 61-63)
__device__ __forceinline__ unsigned long long sw128_desc(unsigned saddr)
{
    unsigned long long d = 0;
    d |= (unsigned long long)((saddr & 0x3FFFFu) >> 4);
    d |= 1ull << 16;
    d |= (unsigned long long)(1024 >> 4) << 32;
    d |= 1ull << 46;
    d |= 2ull << 61;
    return d;
}

// instruction descriptor of kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16 (bits
// 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 (bits 17-22),
// M >> 4 (bits 24-28)
template <int BN>
__device__ __forceinline__ unsigned idesc_bf16()
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(BN >> 3) << 17) | ((unsigned)(kBM >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(unsigned tmem_d, unsigned long long da, unsigned long long db, unsigned idesc,
                                       unsigned accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned long long* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }

// 32 lanes x 32 consecutive 32-bit columns of TMEM into r[0..31] (this warp's lanes)
__device__ __forceinline__ void tmem_ld32(unsigned taddr, unsigned* r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

template <int BN>
constexpr int tmem_cols()
{
    return BN < 32 ? 32 : BN;
}
template <int BN>
constexpr size_t gemm_smem()
{
    return (size_t)kStages * (kBM * kBK * 2 + BN * kBK * 2) + 1024;  // + alignment slack
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, void* C, int M,
              int N, int K, int k_per_split, int epi, const float* __restrict__ bias, int* status)
{
    constexpr int A_BYTES = kBM * kBK * 2;
    constexpr int B_BYTES = BN * kBK * 2;
    constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    constexpr unsigned TCOLS = tmem_cols<BN>();
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    // 128-byte-swizzled operand tiles start on 1024-byte boundaries
    unsigned char* sm = smem_align_up<1024>(smem_dyn);
    __shared__ unsigned long long full[kStages], empty[kStages], done;
    __shared__ unsigned tmem_base;
    __shared__ int aborted, issued, consumed;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int kbeg = blockIdx.z * k_per_split;
    const int kend = min(K, kbeg + k_per_split);
    const int nkb = kend > kbeg ? (kend - kbeg + kBK - 1) / kBK : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s]);
            mbar_init(&empty[s]);
        }
        mbar_init(&done);
        fence_mbar_init();
        aborted = 0;
        issued = 0;
        consumed = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tmem_base)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        int kb = 0;
        for (; kb < nkb; ++kb) {
            const int s = kb % kStages, use = kb / kStages;
            if (use > 0 && !mbar_wait(&empty[s], (unsigned)((use - 1) & 1))) {
                aborted = 1;
                break;
            }
            unsigned char* st = sm + s * STAGE_BYTES;
            mbar_expect_tx(&full[s], STAGE_BYTES);
            tma_load_2d(st, &mapA, kbeg + kb * kBK, m0, &full[s]);
            tma_load_2d(st + A_BYTES, &mapB, kbeg + kb * kBK, n0, &full[s]);
        }
        issued = kb;
    } else if (warp == 1 && lane == 0) {
        const unsigned idesc = idesc_bf16<BN>();
        int kb = 0;
        for (; kb < nkb; ++kb) {
            const int s = kb % kStages, use = kb / kStages;
            if (!mbar_wait(&full[s], (unsigned)(use & 1))) {
                aborted = 1;
                break;
            }
            tc_fence_after();
            const unsigned sa = smem_addr(sm + s * STAGE_BYTES);
            const unsigned long long da = sw128_desc(sa), db = sw128_desc(sa + A_BYTES);
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)  // K = 16 per MMA: 32 bytes along the swizzled row
                tc_mma(tmem, da + 2ull * k, db + 2ull * k, idesc, (kb > 0 || k > 0) ? 1u : 0u);
            tc_commit(&empty[s]);
        }
        consumed = kb;
        tc_commit(&done);  // arrives once every MMA issued above has completed
    }
    __syncwarp();
    const bool ok = mbar_wait(&done, 0u);
    tc_fence_after();
    __syncthreads();
    const bool good = ok && !aborted && nkb > 0;

    // epilogue: row m0 + 32 warp + lane, columns n0 + c0 .. n0 + c0 + 31
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < BN; c0 += 32) {
        unsigned r[32];
        tmem_ld32(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0, r);
        if (!good || row >= M) continue;
        float v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            float x = __uint_as_float(r[j]);
            const int col = n0 + c0 + j;
            if ((epi & kEpiBias) && col < N) x += bias[col];
            if (epi & kEpiRelu) x = fmaxf(x, 0.f);
            v[j] = x;
        }
        const int col0 = n0 + c0;
        if (epi & kEpiBF16) {
            __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(C) + (long long)row * N + col0;
            if (col0 + 32 <= N && ((N & 7) == 0)) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    __nv_bfloat162 h[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) h[t] = __floats2bfloat162_rn(v[8 * q + 2 * t], v[8 * q + 2 * t + 1]);
                    *reinterpret_cast<uint4*>(out + 8 * q) = *reinterpret_cast<uint4*>(h);
                }
            } else {
                for (int j = 0; j < 32 && col0 + j < N; ++j) out[j] = __float2bfloat16_rn(v[j]);
            }
        } else {
            float* out = reinterpret_cast<float*>(C) + (long long)blockIdx.z * M * N + (long long)row * N + col0;
            if (col0 + 32 <= N && ((N & 3) == 0)) {
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    *reinterpret_cast<float4*>(out + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            } else {
                for (int j = 0; j < 32 && col0 + j < N; ++j) out[j] = v[j];
            }
        }
    }
    if (threadIdx.x == 0 && !good && nkb > 0) {
        *status = 2;
        // copies issued but never consumed may still be in flight: wait for them (bounded)
        for (int kb = consumed; kb < issued; ++kb) mbar_wait(&full[kb % kStages], (unsigned)((kb / kStages) & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TCOLS) : "memory");
}

__global__ void k_reduce_splits(const float* __restrict__ part, int splits, long long count, float* __restrict__ out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        float acc = part[i];
        for (int z = 1; z < splits; ++z) acc += part[(long long)z * count + i];
        out[i] = acc;
    }
}

bool encode_bf16(CUtensorMap* m, const void* base, int ld, int rows, int cols, int box_rows)
{
    EncodeTiled fn = tensor_map_encoder();
    if (!fn || !base || (ld & 7) || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
cudaError_t launch(const TcGemm& g, void* C, int epi, const float* bias, int* status, cudaStream_t st)
{
    static bool prepared = false;  // per process (one device in use at a time)
    if (!prepared) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)gemm_smem<BN>());
        if (e != cudaSuccess) return e;
        prepared = true;
    }
    dim3 grid((unsigned)((g.M + kBM - 1) / kBM), (unsigned)((g.N + BN - 1) / BN), (unsigned)g.splits);
    k_tc_gemm<BN><<<grid, kThreads, gemm_smem<BN>(), st>>>(g.a, g.b, C, g.M, g.N, g.K, g.k_per_split, epi, bias,
                                                          status);
    return cudaGetLastError();
}

}  // namespace

EncodeTiled tensor_map_encoder()
{
    static EncodeTiled fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<EncodeTiled>(p);
        return (EncodeTiled) nullptr;
    }();
    return fn;
}

bool tc_gemm_plan(TcGemm* g, const void* A, int lda, const void* B, int ldb, int M, int N, int K, int splits)
{
    std::memset(g, 0, sizeof(*g));
    if (M <= 0 || N <= 0 || K <= 0 || lda < K || ldb < K || splits < 1) return false;
    g->M = M;
    g->N = N;
    g->K = K;
    g->bn = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
    const int kblocks = (K + kBK - 1) / kBK;
    if (splits > kblocks) splits = kblocks;
    const int per = (kblocks + splits - 1) / splits;
    g->k_per_split = per * kBK;
    g->splits = (kblocks + per - 1) / per;  // every split has at least one K block
    return encode_bf16(&g->a, A, lda, M, K, kBM) && encode_bf16(&g->b, B, ldb, N, K, g->bn);
}

cudaError_t tc_gemm_run(const TcGemm& g, void* C, int epilogue, const float* bias, int* status, cudaStream_t st)
{
    if (g.splits > 1 && epilogue != kEpiF32) return cudaErrorInvalidValue;
    switch (g.bn) {
        case 32: return launch<32>(g, C, epilogue, bias, status, st);
        case 64: return launch<64>(g, C, epilogue, bias, status, st);
        case 128: return launch<128>(g, C, epilogue, bias, status, st);
        default: return launch<256>(g, C, epilogue, bias, status, st);
    }
}

cudaError_t tc_reduce_splits(const float* part, int splits, long long count, float* out, cudaStream_t st)
{
    long long blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_reduce_splits<<<(unsigned)blocks, 256, 0, st>>>(part, splits, count, out);
    return cudaGetLastError();
}

}  // namespace mgmc
