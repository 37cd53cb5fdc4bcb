// unet.cu -- learned warm start for the sampler: a U-Net maps (kappa^2, the
// observation mask, the observed values) to an estimate of the posterior mean,
// used only as the chain's initial state x_0.  Its convolutions are GEMMs on the
// tcgen05 tensor cores (tc_gemm.cu); this file holds the C ABI.
#include <cuda_runtime.h>

#include <string>

#include "../../include/mgmc.h"
#include "common.cuh"
#include "tc_gemm.cuh"

namespace mgmc {
namespace {

// scratch for split-K partials and the status word of the exported GEMM
struct GemmScratch {
    float* part = nullptr;
    size_t part_bytes = 0;
    int* status = nullptr;
};
thread_local GemmScratch g_scratch;

}  // namespace
}  // namespace mgmc

using namespace mgmc;

extern "C" mgmc_status mgmc_tc_gemm(const void* A, int lda, const void* B, int ldb, void* C, int M, int N, int K,
                                    int splits, int epilogue, const float* bias, void* stream)
{
    if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0 || splits < 1 || (epilogue & ~7) ||
        ((epilogue & kEpiBias) && !bias)) {
        set_last_error("mgmc_tc_gemm: bad arguments");
        return MGMC_ERR_ARG;
    }
    if (splits > 1 && epilogue != kEpiF32) {
        set_last_error("mgmc_tc_gemm: split-K needs the plain FP32 epilogue");
        return MGMC_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    TcGemm g;
    if (!tc_gemm_plan(&g, A, lda, B, ldb, M, N, K, splits)) {
        set_last_error("mgmc_tc_gemm: TMA descriptor encoding failed (alignment, lda/ldb)");
        return MGMC_ERR_ARG;
    }
    GemmScratch& sc = g_scratch;
    if (!sc.status) {
        if (cudaMalloc(&sc.status, sizeof(int)) != cudaSuccess) return MGMC_ERR_CUDA;
        cudaMemset(sc.status, 0, sizeof(int));
    }
    void* out = C;
    if (g.splits > 1) {
        const size_t need = sizeof(float) * (size_t)g.splits * M * N;
        if (need > sc.part_bytes) {
            if (sc.part) cudaFree(sc.part);
            sc.part = nullptr;
            sc.part_bytes = 0;
            if (cudaMalloc(&sc.part, need) != cudaSuccess) return MGMC_ERR_OOM;
            sc.part_bytes = need;
        }
        out = sc.part;
    }
    if (tc_gemm_run(g, out, epilogue, bias, sc.status, st) != cudaSuccess) {
        set_last_error("mgmc_tc_gemm: launch failed");
        return MGMC_ERR_CUDA;
    }
    if (g.splits > 1 && tc_reduce_splits(sc.part, g.splits, (long long)M * N, (float*)C, st) != cudaSuccess)
        return MGMC_ERR_CUDA;
    return MGMC_OK;
}
