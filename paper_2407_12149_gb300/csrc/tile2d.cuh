// tile2d.cuh -- launchers of the fused 2D tile kernels (tile2d.cu).
#pragma once
#include <cuda.h>

#include "common.cuh"

namespace mgmc {

// One chain's grid in a batched tile launch: blocks [tile0, tile0 + ntiles).
// The descriptors are held by value so that a CTA fetches everything it needs
// with one parallel copy into shared memory.
template <typename T>
struct TileJob {
    DevLevel<T> L;
    DevLevel<T> C;
    DevProblem P;
    int tile0;
    int ntiles;
};
// TMA descriptors of one tile job: the state source, the operator fields, the
// dense right-hand side (9-point grids) and, backward, the coarse psi
constexpr int kTileMaxMaps = 8;
struct TileMaps {  // CUtensorMap is 64-byte aligned
    CUtensorMap m[kTileMaxMaps];
};

// one chain's grid in a batched low-rank launch: blocks [block0, block0 + nblocks)
template <typename T>
struct LowrankJob {
    DevLevel<T> L;
    DevLevel<T> C;
    DevProblem P;
    int block0;
    int nblocks;
};

// shared-memory limits and occupancy of the tile kernels (once per device)
template <typename T>
cudaError_t tile_prepare_batch();
// TMA descriptors of level L's forward (bwd = false) or backward tile job
template <typename T>
bool make_tile_maps(const DevLevel<T>& L, const DevLevel<T>& C, bool bwd, TileMaps* out);
// one persistent launch over the ntiles tiles of a grid depth of every chain;
// per: the common tile count of every job (0 if they differ); x_zero: the forward
// sweep starts from psi = 0 (every grid but the finest)
template <typename T>
void launch_tile_batch(const TileJob<T>* jobs, const TileMaps* maps, int njobs, int per, int ntiles, bool fine,
                       bool bwd, bool x_zero, cudaStream_t st, int& launches);
// per: the common block count of every job (0 if they differ)
template <typename T>
void launch_lowrank_batch(const LowrankJob<T>* jobs, int njobs, int per, int nblocks, bool down, cudaStream_t st,
                          int& launches);
int lowrank_blocks(int rows);

}  // namespace mgmc
