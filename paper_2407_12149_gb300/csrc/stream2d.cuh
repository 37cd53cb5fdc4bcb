// stream2d.cuh -- streaming kernels of the finest 2D grid (5-point, FP32): the
// forward pass (Alg. 1 pre-smoothing + residual + restriction) and the backward
// pass (prolongation + post-smoothing) of every chain of a batch, one launch each.
#pragma once
#include <cuda.h>

#include "common.cuh"

namespace mgmc {

// The finest grid of one chain, cut into bands of 128 columns and each band into
// strips of 16 rows; global strips [strip0, strip0 + nbands * spb) belong to it,
// band by band, top to bottom within a band.
struct StreamJob {
    DevLevel<float> L;   // the finest grid
    DevLevel<float> C;   // the next coarser grid (restriction target, coarse correction psi)
    CycleState* cs;
    long long strip0;
    int spb;             // strips per band: ceil(n / 16)
    int nbands;          // ceil(n / 128)
};

// TMA descriptors of one chain: the state the pass reads (theta forward, the
// second state buffer backward), the operator field s kappa^2, the coarse psi
struct StreamMaps {  // CUtensorMap is 64-byte aligned
    CUtensorMap x;
    CUtensorMap k;
    CUtensorMap p;
};

constexpr int kStreamBand = 128;  // interior columns per band
constexpr int kStreamRows = 16;   // rows per strip (one pipeline step)

// resident CTAs per SM of the two kernels (once per device)
cudaError_t stream_prepare();
bool make_stream_maps(const DevLevel<float>& L, const DevLevel<float>& C, bool bwd, StreamMaps* out);
// CTAs of one launch over `strips` strips: one or two per SM, whichever the
// step count of the most loaded CTA favours
int stream_grid(long long strips);
void launch_stream_fine(const StreamJob* jobs, const StreamMaps* maps, int njobs, long long strips, int grid,
                        bool bwd, cudaStream_t st, int& launches);

}  // namespace mgmc
