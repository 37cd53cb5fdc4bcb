// kernels.cuh -- launch wrappers of the V-cycle kernels (see kernels.cu).
#pragma once
#include "common.cuh"
#include "stencil.cuh"

namespace mgmc {

template <typename T>
void launch_sweep(const DevLevel<T>& L, const DevProblem& P, int dir, unsigned slot, cudaStream_t st, int& launches);
// dir < 0: only d_{l-1} = d_l - B^T theta (no correction)
template <typename T>
void launch_lowrank(const DevLevel<T>& L, const DevProblem& P, int dir, unsigned slot, bool dnext, cudaStream_t st,
                    int& launches);
template <typename T>
void launch_restrict(const DevLevel<T>& F, const DevLevel<T>& C, cudaStream_t st, int& launches);
// exact coarsest sample of the general path with the noise slot of the grid's visit
template <typename T>
void launch_coarsest_slot(const DevLevel<T>& L, const DevProblem& P, const double* chol, int n0, unsigned slot,
                          cudaStream_t st, int& launches);
// the small grids of the general path (2D) in one CTA: a list of phases {code, level, slot,
// flags} the host builds from the cycle's recursion (kernels.cu, k_cycle_small)
enum { kOpSweep = 0, kOpLowrank = 1, kOpRestrict = 2, kOpZero = 3, kOpCoarsest = 4, kOpProlong = 5 };
constexpr int kSmallCycleThreads = 512;
constexpr int kSmallMaxLevels = 16;   // grids 0..top held by the kernel (top < 16)
constexpr int kSmallMaxOps = 1024;    // phases staged in shared memory (later ones read from global)
// zb: scratch of n^2 doubles for the largest 25-point grid held (the normals of a sweep)
template <typename T>
void launch_cycle_small(const DevLevel<T>* levels_dev, int top, const DevProblem& P, const double* chol, int n0,
                        const int4* ops, int n_ops, double* zb, cudaStream_t st, int& launches);
template <typename T>
void launch_prolong(const DevLevel<T>& C, const DevLevel<T>& F, cudaStream_t st, int& launches);
// one chain of a batched coarse-grid launch
template <typename T>
struct CoarseJob {
    const DevLevel<T>* levels;   // device descriptors of grids 0 .. L-1
    int top;
    int is_finest;
    const DevProblem* P;
    const double* chol;
    int n0;
};
// one chain of a batched QoI launch
template <typename T>
struct QoiJob {
    const T* x;                  // finest-grid state
    int n_qoi;
    const long long* q_site;
    const double* q_w;
    CycleState* cs;
};
template <typename T>
cudaError_t coarse_prepare_batch(size_t smem_bytes);
template <typename T>
void launch_coarse_batch(const CoarseJob<T>* jobs, int n, int threads, size_t smem_bytes, cudaStream_t st,
                         int& launches);
template <typename T>
void launch_qoi_batch(const QoiJob<T>* jobs, int n, cudaStream_t st, int& launches);
void launch_set_cycle_batch(CycleState* const* cs, int n, unsigned long long seed, unsigned long long cycle, int noise,
                            double* qoi, long long n_steps, cudaStream_t st);

// the V-cycle of grids 0..top in one CTA with shared-memory state (coarse.cu)
// grids a coarse kernel holds at most (their descriptors are staged in shared memory)
constexpr int kCoarseMaxLevels = 8;
// coarsest grids with at most this many unknowns are solved by one warp from a factor
// staged in shared memory
constexpr int kCoarsestWarp = 32;
// elements of the coarse kernel's dynamic shared memory; top_is_fd_finest: the top
// grid is the finest grid in its 5/7-point finite-difference form (one operator field)
long long coarse_smem_elems(int dim, const int* n_of_level, int top, bool top_is_fd_finest);
template <typename T>
cudaError_t coarse_prepare(int dim, size_t smem_bytes);
template <typename T>
void launch_coarse(const DevLevel<T>* levels_dev, int dim, int top, bool is_finest, const DevProblem& P,
                   const double* chol, int n0, int nu1, int nu2, size_t smem_bytes, cudaStream_t st, int& launches);
template <typename T>
void launch_qoi(const DevLevel<T>& L, int n_qoi, const long long* q_site, const double* q_w, const DevProblem& P,
                cudaStream_t st, int& launches);
void launch_set_cycle(CycleState* cs, unsigned long long seed, unsigned long long cycle, unsigned chain, int noise,
                      double* qoi, cudaStream_t st);
template <typename T>
void launch_pack(const DevLevel<T>& L, T* dense, bool to_padded, cudaStream_t st);
// 2D dense user fields <-> padded finest-level states of many chains, one launch per
// kPackChunk chains; jobs[c] is the static part, dense[c] the caller's array
template <typename T>
struct PackJob {
    T* x;            // padded finest-level state
    int n;
    int pitch;
    long long base;
};
constexpr int kPackChunk = 256;
template <typename T>
void launch_pack_batch(const PackJob<T>* jobs, void* const* dense, int count, int max_n, bool to_padded,
                       cudaStream_t st);
template <typename T>
void launch_resid(const DevLevel<T>& L, const DevProblem& P, double* u, double* partial, int max_partial,
                  double* out, cudaStream_t st);

}  // namespace mgmc
