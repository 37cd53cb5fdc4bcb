// tc_gemm.cuh -- BF16 GEMM on the tcgen05 tensor cores (tc_gemm.cu).
//
//   C[M][N] = A[M][K] * B[N][K]^T
//
// A and B are row-major BF16 with K contiguous (both operands "K-major"), the
// accumulator is FP32 in tensor memory.  The epilogue adds a bias per column,
// applies ReLU and stores FP32 or BF16, or stores the FP32 partial sum of one
// K range (split-K; C + z * M * N for split z).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

namespace mgmc {

enum TcEpilogue : int {
    kEpiF32 = 0,        // C (float) = acc                      (split z writes C + z * M * N)
    kEpiBias = 1,       // + bias[n]
    kEpiRelu = 2,       // max(., 0)
    kEpiBF16 = 4,       // store BF16 instead of FP32
};

struct TcGemm {
    CUtensorMap a, b;   // TMA descriptors of A (box 64 x 128) and B (box 64 x bn)
    int M, N, K;
    int bn;             // N tile: 32, 64, 128 or 256
    int splits;         // K ranges (each a multiple of 64 elements)
    int k_per_split;
};

// Describe C = A B^T for row-major BF16 A [M][lda] and B [N][ldb] (lda, ldb >= K,
// multiples of 8 elements; device pointers 16-byte aligned).  splits > 1 only
// with the FP32 epilogue.  Returns false if the descriptors cannot be encoded.
bool tc_gemm_plan(TcGemm* g, const void* A, int lda, const void* B, int ldb, int M, int N, int K, int splits);
// Launch; C is float or __nv_bfloat16 [M][N] (row-major), bias float [N] or NULL.
// status: device int set to 2 if a bounded wait inside the kernel gave up.
cudaError_t tc_gemm_run(const TcGemm& g, void* C, int epilogue, const float* bias, int* status, cudaStream_t st);
// Sum of `splits` FP32 partials [splits][count] into out [count] (fixed order).
cudaError_t tc_reduce_splits(const float* part, int splits, long long count, float* out, cudaStream_t st);

}  // namespace mgmc
