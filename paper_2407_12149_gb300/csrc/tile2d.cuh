// tile2d.cuh -- launchers of the fused 2D tile kernels (tile2d.cu).
#pragma once
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
// one chain's grid in a batched low-rank launch: blocks [block0, block0 + nblocks)
template <typename T>
struct LowrankJob {
    DevLevel<T> L;
    DevLevel<T> C;
    DevProblem P;
    int block0;
    int nblocks;
};

// raise the dynamic shared-memory limit of the tile kernels (once per device)
template <typename T>
cudaError_t tile_prepare();
// forward sweep of level L fused with the residual restriction into C.f;
// x_zero: the sweep starts from psi = 0 (every grid but the finest)
template <typename T>
void launch_tile_fwd(const DevLevel<T>& L, const DevLevel<T>& C, const DevProblem& P, bool x_zero, cudaStream_t st,
                     int& launches);
// prolongation of C.x into L and the backward sweep
template <typename T>
void launch_tile_bwd(const DevLevel<T>& L, const DevLevel<T>& C, const DevProblem& P, cudaStream_t st, int& launches);
// low-rank correction after a fused sweep (down: forward G, H fix-up, d_{l-1})
template <typename T>
void launch_lowrank_fused(const DevLevel<T>& L, const DevLevel<T>& C, const DevProblem& P, bool down, cudaStream_t st,
                          int& launches);

template <typename T>
cudaError_t tile_prepare_batch();
// per: the common block count of every job (0 if they differ)
template <typename T>
void launch_tile_batch(const TileJob<T>* jobs, int njobs, int per, int nblocks, bool fine, bool bwd, bool x_zero,
                       cudaStream_t st, int& launches);
template <typename T>
void launch_lowrank_batch(const LowrankJob<T>* jobs, int njobs, int per, int nblocks, bool down, cudaStream_t st,
                          int& launches);
int lowrank_blocks(int rows);

}  // namespace mgmc
