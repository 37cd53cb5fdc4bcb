// stream9.cuh -- streaming kernels of the 9-point Galerkin grids of the 2D
// V-cycle (FP32): the forward pass (Alg. 1 pre-smoothing from psi = 0 + residual
// + restriction) and the backward pass (prolongation + post-smoothing) of one
// grid depth of every chain of a batch, one launch each.
#pragma once
#include <cuda.h>

#include "stream2d.cuh"

namespace mgmc {

// TMA descriptors of one chain's grid: the state the backward pass reads (the
// second state buffer), the five operator fields (slot 0 = row sum, slots 1..4 the
// couplings to the right, upper-left, upper and upper-right neighbours), the dense
// right-hand side and the coarse psi
struct Stream9Maps {  // CUtensorMap is 64-byte aligned
    CUtensorMap x;
    CUtensorMap c[5];
    CUtensorMap f;
    CUtensorMap p;
};

constexpr int kStream9Band = 64;   // interior columns per band
constexpr int kStream9Rows = 16;   // rows per strip (one pipeline step)

// resident CTAs per SM of the two kernels (once per device)
cudaError_t stream9_prepare();
bool make_stream9_maps(const DevLevel<float>& L, const DevLevel<float>& C, Stream9Maps* out);
int stream9_grid(long long strips);
// StreamJob.spb = ceil(n / 16), nbands = ceil(n / 64) for these kernels
void launch_stream9(const StreamJob* jobs, const Stream9Maps* maps, int njobs, long long strips, int grid, bool bwd,
                    cudaStream_t st, int& launches);

}  // namespace mgmc
