// api.cu -- the C ABI (include/mgmc.h): handle life cycle, device upload of
// the hierarchy, CUDA-graph capture of one V-cycle and the sampling loop.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "setup.hpp"
#include "stream2d.cuh"
#include "stream9.cuh"
#include "tile2d.cuh"

using namespace mgmc;

namespace {

thread_local std::string g_last_error;

mgmc_status fail(mgmc_status code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

#define CUDA_TRY(expr)                                                                                         \
    do {                                                                                                       \
        cudaError_t _e = (expr);                                                                               \
        if (_e != cudaSuccess)                                                                                 \
            return fail(MGMC_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));                     \
    } while (0)

// elements per padded row: 4 leading elements, the n interior sites and R trailing
// halo elements (R = stencil radius), rounded up to 128 bytes
long long padded_pitch(int n, int elem_bytes, int R = 1)
{
    int align = 128 / elem_bytes;
    return ((long long)(n + 4 + R) + align - 1) / align * align;
}

struct Buffers {
    mgmc_allocator alloc{};
    bool use_cuda_malloc = true;
    cudaStream_t stream = nullptr;
    std::vector<void*> list;
    void* get(size_t bytes)
    {
        if (bytes == 0) bytes = 16;
        bytes = (bytes + 255) / 256 * 256;
        void* p = nullptr;
        if (use_cuda_malloc) {
            if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
        } else {
            p = alloc.alloc(bytes, (void*)stream, alloc.ctx);
        }
        if (p) list.push_back(p);
        return p;
    }
    void release()
    {
        for (void* p : list) {
            if (use_cuda_malloc)
                cudaFree(p);
            else
                alloc.free(p, (void*)stream, alloc.ctx);
        }
        list.clear();
    }
};

}  // namespace

namespace mgmc {
// message for mgmc_last_error() from entry points defined in other files
void set_last_error(const char* msg) { g_last_error = msg; }
}  // namespace mgmc

struct mgmc_ctx {
    mgmc_config cfg{};
    int L = 0;            // number of levels
    int top = 0;          // highest level inside the coarse kernel
    int m = 0;
    int device = 0;
    Buffers buf;
    CycleState* cs = nullptr;
    DevProblem P{};
    std::vector<DevLevel<float>> lf;
    std::vector<DevLevel<double>> ld;
    void* levels_dev = nullptr;
    double* chol = nullptr;
    int n0 = 0;
    int n_qoi = 0;
    long long* q_site = nullptr;
    double* q_w = nullptr;
    void* x_stage = nullptr;
    double* u = nullptr;
    double* partial = nullptr;
    double* rnorm = nullptr;
    int max_partial = 0;
    double f_norm = 0.0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
    size_t coarse_smem = 0;   // dynamic shared memory of the coarse-grid kernel
    bool fused = false;   // 2D, nu1 = nu2 = 1: fused tile kernels on the grids above coarse_max_n
    bool recursive = false;   // W-cycle or radius-2 grids: general kernels, cycle enqueued recursively
    // recursive path, 2D: grids 0..small_top run in one k_cycle_small launch per visit of
    // grid small_top (-1: none); the phase lists of the cycle's visits, in cycle order
    int small_top = -1;
    int4* small_ops = nullptr;
    double* small_z = nullptr;   // normals of one sweep of the largest 25-point grid held
    std::vector<int> small_off, small_cnt;
    int small_next = 0;
    DevProblem* P_dev = nullptr;   // device copy of P (batched launches)
    // batch handle: per-chain handles and the job tables of the batched launches
    std::vector<mgmc_ctx*> sub;
    int n_depth = 0;
    std::vector<void*> jobs_tile, jobs_lrd, jobs_lru;
    std::vector<void*> maps_fwd, maps_bwd;   // TileMaps per tile job, per depth
    std::vector<int> njob_tile, nblk_tile, njob_lrd, nblk_lrd, njob_lru, nblk_lru;
    std::vector<int> per_tile, per_lrd, per_lru;
    // FP32 finest grids: the streaming kernels (stream2d.cu) instead of depth-0 tiles
    bool stream_fine = false;
    bool fine0 = true;    // the depth-0 grids have the 5-point finite-difference form
    void* jobs_stream = nullptr;
    void* maps_sfwd = nullptr;
    void* maps_sbwd = nullptr;
    int njob_stream = 0;
    long long stream_strips = 0;
    int stream_ctas = 0;
    // FP32 9-point grids below the finest: the streaming band kernels (stream9.cu) at the
    // depths whose grids all have n >= band_min_n, per depth
    int coarse_threads = 0;   // threads of the batched coarse kernel (0: by the chain count)
    std::vector<char> s9_ok, s9_use;
    std::vector<int> s9_minn;   // smallest grid of the depth
    std::vector<void*> jobs_s9, maps_s9;
    std::vector<int> njob_s9, s9_grid;
    std::vector<long long> s9_strips;
    void* jobs_coarse = nullptr;
    void* jobs_qoi = nullptr;
    void* jobs_pack = nullptr;    // PackJob<T> per chain (2D fused path)
    int pack_max_n = 0;
    CycleState** cs_list = nullptr;
    size_t batch_coarse_smem = 0;
    bool is_batch() const { return !sub.empty(); }
    bool profile = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool fp32() const { return cfg.precision == MGMC_FP32; }
};

namespace {

template <typename T>
mgmc_status build_batch_tables(mgmc_ctx* h);
void apply_band_min(mgmc_ctx* h);

template <typename T>
std::vector<DevLevel<T>>& levels_of(mgmc_ctx* h);
template <>
std::vector<DevLevel<float>>& levels_of<float>(mgmc_ctx* h) { return h->lf; }
template <>
std::vector<DevLevel<double>>& levels_of<double>(mgmc_ctx* h) { return h->ld; }

template <typename V>
V* upload(mgmc_ctx* h, const std::vector<V>& v, mgmc_status& st)
{
    V* p = (V*)h->buf.get(v.size() * sizeof(V));
    if (!p) {
        st = MGMC_ERR_OOM;
        return nullptr;
    }
    if (!v.empty() && cudaMemcpyAsync(p, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice, h->buf.stream) !=
                          cudaSuccess)
        st = MGMC_ERR_CUDA;
    return p;
}

template <typename T>
mgmc_status build_device_levels(mgmc_ctx* h, const HostProblem& hp)
{
    const int d = hp.dim;
    auto& levels = levels_of<T>(h);
    levels.assign(hp.n_levels, DevLevel<T>{});
    mgmc_status st = MGMC_OK;
    for (int l = 0; l < hp.n_levels; ++l) {
        const HostLevel& HL = hp.lev[l];
        DevLevel<T>& D = levels[l];
        std::memset(&D, 0, sizeof(D));
        D.level = l;
        D.dim = d;
        D.n = HL.n;
        // radius-R stencils read R halo rows and columns around the interior
        const int R = hp.R;
        D.rad = R;
        D.pitch = (int)padded_pitch(HL.n, sizeof(T), R);
        D.plane = (long long)D.pitch * (HL.n + 2 * R);
        D.base = 4 + (long long)R * D.pitch + (d == 3 ? D.plane : 0);
        D.alloc = d == 3 ? D.plane * (HL.n + 2) : D.plane;
        auto off = [&](long long s) {
            int i = (int)(s % HL.n), j = (int)((s / HL.n) % HL.n), k = d == 3 ? (int)(s / ((long long)HL.n * HL.n)) : 0;
            return site_offset(d, D.pitch, D.plane, D.base, i, j, k);
        };
        size_t fbytes = (size_t)D.alloc * sizeof(T);
        D.x = (T*)h->buf.get(fbytes);
        if (!D.x) return fail(MGMC_ERR_OOM, "allocator returned NULL");
        CUDA_TRY(cudaMemsetAsync(D.x, 0, fbytes, h->buf.stream));
        const bool finest = l == hp.n_levels - 1;
        // the finite-difference finest grid keeps its 5/7-point form; a Q1 finest grid is
        // stored like the Galerkin grids (stencil fields and a zero dense right-hand side)
        const bool fd_fine = finest && hp.disc == 0;
        if (!fd_fine) {
            D.f = (T*)h->buf.get(fbytes);
            if (!D.f) return fail(MGMC_ERR_OOM, "allocator returned NULL");
            CUDA_TRY(cudaMemsetAsync(D.f, 0, fbytes, h->buf.stream));
        }
        if (fd_fine) {
            D.fine = 1;
            std::vector<T> diag((size_t)D.alloc, T(0));
            for (long long s = 0; s < HL.N; ++s)
                diag[(size_t)off(s)] = sizeof(T) == 4 ? (T)hp.kappa_part[(size_t)s] : (T)HL.st[(size_t)s * hp.NS + hp.C];
            D.diag = upload(h, diag, st);
            D.woff = (T)hp.woff_fine;
        } else {
            D.fine = 0;
            D.ncoef = (hp.NS + 1) / 2;
            std::vector<T> coef((size_t)D.alloc * D.ncoef, T(0));
            std::vector<double> rs;
            if (sizeof(T) == 4) rs = row_sums(hp, l);
            for (long long s = 0; s < HL.N; ++s) {
                long long e = off(s);
                const double* a = &HL.st[(size_t)s * hp.NS];
                coef[(size_t)e] = sizeof(T) == 4 ? (T)rs[(size_t)s] : (T)a[hp.C];
                for (int t = 1; t < D.ncoef; ++t) coef[(size_t)t * D.alloc + e] = (T)a[hp.C + t];
            }
            D.coef = upload(h, coef, st);
            if (R == 2 && sizeof(T) == 8) {
                std::vector<double> aux((size_t)D.alloc * 2, 0.0);
                for (long long s2 = 0; s2 < HL.N; ++s2) {
                    const long long e = off(s2);
                    const double aii = HL.st[(size_t)s2 * hp.NS + hp.C];
                    aux[(size_t)e] = 1.0 / aii;
                    aux[(size_t)D.alloc + (size_t)e] = std::sqrt(aii);
                }
                D.inv_sqrt25 = upload(h, aux, st);
            }
        }
        if (hp.m > 0) {
            // rows of B grouped by grid row, sorted by x index
            long long nrows = d == 3 ? (long long)HL.n * HL.n : HL.n;
            std::vector<std::vector<std::pair<int, std::pair<int, double>>>> rows((size_t)nrows);
            for (int k = 0; k < hp.m; ++k)
                for (int t = HL.bptr[k]; t < HL.bptr[k + 1]; ++t) {
                    long long s = HL.bsite[t];
                    int i = (int)(s % HL.n);
                    long long r = s / HL.n;
                    rows[(size_t)r].push_back({i, {k, HL.bw[t]}});
                }
            std::vector<int> rptr((size_t)nrows + 1, 0), ei, ek;
            std::vector<double> ew;
            for (long long r = 0; r < nrows; ++r) {
                auto& v = rows[(size_t)r];
                std::sort(v.begin(), v.end(), [](const auto& a, const auto& b) {
                    return a.first != b.first ? a.first < b.first : a.second.first < b.second.first;
                });
                for (auto& e : v) {
                    ei.push_back(e.first);
                    ek.push_back(e.second.first);
                    ew.push_back(e.second.second);
                }
                rptr[(size_t)r + 1] = (int)ei.size();
            }
            D.brow_ptr = upload(h, rptr, st);
            D.bent_i = upload(h, ei, st);
            D.bent_k = upload(h, ek, st);
            D.bent_w = upload(h, ew, st);
            std::vector<long long> cs;
            for (long long s : HL.bsite) cs.push_back(off(s));
            D.bcol_ptr = upload(h, HL.bptr, st);
            D.bcol_site = upload(h, cs, st);
            D.bcol_w = upload(h, HL.bw, st);
            for (int dir = 0; dir < 2; ++dir) {
                D.g_rows[dir] = (int)HL.gsite[dir].size();
                std::vector<long long> gs;
                for (long long s : HL.gsite[dir]) gs.push_back(off(s));
                D.g_site[dir] = upload(h, gs, st);
                D.g_val[dir] = upload(h, HL.gval[dir], st);
            }
            std::vector<double> dv(hp.m, 0.0);
            if (finest) dv = hp.y;
            D.d = upload(h, dv, st);
        }
        if (st != MGMC_OK) return fail(st, "device upload failed");
    }
    for (int l = 1; l < hp.n_levels; ++l) levels[l].dnext = levels[l - 1].d;
    // G in the path precision and B^T G for every grid with a smoother
    for (int l = 1; l < hp.n_levels && hp.m > 0; ++l) {
        DevLevel<T>& D = levels[l];
        HostLevel& HL = const_cast<HostLevel&>(hp.lev[l]);
        for (int dir = 0; dir < 2; ++dir) {
            std::vector<T> gt(HL.gval[dir].begin(), HL.gval[dir].end());
            D.gT[dir] = upload(h, gt, st);
        }
        fused_extras(HL, hp, l);
        D.BtG = upload(h, HL.BtG, st);
        if (st != MGMC_OK) return fail(st, "device upload failed");
    }
    // grids inside the coarse kernel: shared-memory indices of the observation and G sites
    for (int l = 0; l <= h->top && hp.m > 0; ++l) {
        const HostLevel& HL = hp.lev[l];
        DevLevel<T>& D = levels[l];
        const int S = HL.n + 2;
        auto sidx = [&](long long s) {
            int i = (int)(s % HL.n), j = (int)((s / HL.n) % HL.n), k = d == 3 ? (int)(s / ((long long)HL.n * HL.n)) : 0;
            return d == 3 ? ((k + 1) * S + (j + 1)) * S + (i + 1) : (j + 1) * S + (i + 1);
        };
        std::vector<int> bss, bdense;
        for (long long s : HL.bsite) {
            bss.push_back(sidx(s));
            bdense.push_back((int)s);
        }
        D.bcol_ss = upload(h, bss, st);
        D.bcol_dense = upload(h, bdense, st);
        for (int dir = 0; dir < 2; ++dir) {
            std::vector<int> gss;
            for (long long s : HL.gsite[dir]) gss.push_back(sidx(s));
            D.g_ss[dir] = upload(h, gss, st);
        }
        if (st != MGMC_OK) return fail(st, "device upload failed");
    }
    {
        std::vector<int> nl;
        for (int l = 0; l < hp.n_levels; ++l) nl.push_back(hp.lev[l].n);
        h->coarse_smem =
            (size_t)coarse_smem_elems(d, nl.data(), h->top, h->top == hp.n_levels - 1 && hp.disc == 0) * sizeof(T);
        cudaError_t e = coarse_prepare<T>(d, h->coarse_smem);
        if (e != cudaSuccess)
            return fail(MGMC_ERR_CUDA, std::string("coarse kernel set-up: ") + cudaGetErrorString(e));
    }
    // general path: residual field of every smoothed grid, low-rank scratch
    if (!h->fused) {
        for (int l = h->top + 1; l < hp.n_levels; ++l) {
            DevLevel<T>& D = levels[l];
            D.res = (T*)h->buf.get((size_t)D.alloc * sizeof(T));
            if (!D.res) return fail(MGMC_ERR_OOM, "allocator returned NULL");
            if (hp.m > 0) D.lrv = upload(h, std::vector<double>((size_t)2 * hp.m, 0.0), st);
        }
        if (st != MGMC_OK) return fail(st, "device upload failed");
    }
    // fused tile path: second state buffer, per-tile observation entries, G/H in T, B^T G
    if (h->fused) {
        for (int l = h->top + 1; l < hp.n_levels; ++l) {
            HostLevel& HL = const_cast<HostLevel&>(hp.lev[l]);
            DevLevel<T>& D = levels[l];
            const DevLevel<T>& Cd = levels[l - 1];
            size_t fbytes = (size_t)D.alloc * sizeof(T);
            D.x2 = (T*)h->buf.get(fbytes);
            if (!D.x2) return fail(MGMC_ERR_OOM, "allocator returned NULL");
            CUDA_TRY(cudaMemsetAsync(D.x2, 0, fbytes, h->buf.stream));
            const int TX = D.fine ? TileShape<T, true>::TX : TileShape<T, false>::TX;
            const int TY = D.fine ? TileShape<T, true>::TY : TileShape<T, false>::TY;
            D.ntx = (HL.n + TX - 1) / TX;
            const int nty = (HL.n + TY - 1) / TY;
            if (hp.m == 0) continue;
            const int ntiles = D.ntx * nty;
            std::vector<std::vector<std::pair<int, int>>> per((size_t)ntiles);
            for (size_t t = 0; t < HL.bsite.size(); ++t) {
                long long s = HL.bsite[t];
                int i = (int)(s % HL.n), j = (int)(s / HL.n);
                int tile = (j / TY) * D.ntx + (i / TX);
                per[(size_t)tile].push_back({(i % TX) | ((j % TY) << 16), (int)t});
            }
            std::vector<int> tptr((size_t)ntiles + 1, 0), tloc, tent;
            for (int t = 0; t < ntiles; ++t) {
                for (auto& e : per[(size_t)t]) {
                    tloc.push_back(e.first);
                    tent.push_back(e.second);
                }
                tptr[(size_t)t + 1] = (int)tloc.size();
            }
            D.tile_ptr = upload(h, tptr, st);
            D.tile_loc = upload(h, tloc, st);
            D.tile_ent = upload(h, tent, st);
            D.zparts = upload(h, std::vector<double>(HL.bsite.size(), 0.0), st);
            const HostLevel& HC = hp.lev[l - 1];
            std::vector<long long> hs;
            for (long long s : HL.hsite) {
                int i = (int)(s % HC.n), j = (int)(s / HC.n);
                hs.push_back(site_offset(d, Cd.pitch, Cd.plane, Cd.base, i, j, 0));
            }
            D.h_rows = (int)hs.size();
            D.h_site = upload(h, hs, st);
            std::vector<T> ht(HL.hval.begin(), HL.hval.end());
            D.hT = upload(h, ht, st);
            if (st != MGMC_OK) return fail(st, "device upload failed");
        }

    }
    // descriptors of all grids (the single-CTA kernel reads 0..top; batched launches any)
    size_t dbytes = sizeof(DevLevel<T>) * (size_t)hp.n_levels;
    h->levels_dev = h->buf.get(dbytes);
    if (!h->levels_dev) return fail(MGMC_ERR_OOM, "allocator returned NULL");
    CUDA_TRY(cudaMemcpyAsync(h->levels_dev, levels.data(), dbytes, cudaMemcpyHostToDevice, h->buf.stream));
    return MGMC_OK;
}

// The 2D nu1 = nu2 = 1 cycle of one chain or of a batch: every phase is one
// launch over the job table of its grid depth (depth 0 = the finest grids).
template <typename T>
void enqueue_cycle_batch(mgmc_ctx* h, cudaStream_t s, int& launches)
{
    const int nc = h->is_batch() ? (int)h->sub.size() : 1;
    const bool prof = h->profile && h->n_depth > 0;
    for (int d = 0; d < h->n_depth; ++d) {
        if (prof && d == 0) cudaEventRecordWithFlags(h->ev[0], s, cudaEventRecordExternal);
        if (d == 0 && h->stream_fine)
            launch_stream_fine((const StreamJob*)h->jobs_stream, (const StreamMaps*)h->maps_sfwd, h->njob_stream,
                               h->stream_strips, h->stream_ctas, false, s, launches);
        else if (h->s9_use[d])
            launch_stream9((const StreamJob*)h->jobs_s9[d], (const Stream9Maps*)h->maps_s9[d], h->njob_s9[d],
                           h->s9_strips[d], h->s9_grid[d], false, s, launches);
        else
            launch_tile_batch<T>((const TileJob<T>*)h->jobs_tile[d], (const TileMaps*)h->maps_fwd[d],
                                 h->njob_tile[d], h->per_tile[d], h->nblk_tile[d], d == 0 && h->fine0, false, d > 0,
                                 s, launches);
        if (prof && d == 0) cudaEventRecordWithFlags(h->ev[1], s, cudaEventRecordExternal);
        launch_lowrank_batch<T>((const LowrankJob<T>*)h->jobs_lrd[d], h->njob_lrd[d], h->per_lrd[d], h->nblk_lrd[d],
                                true, s, launches);
    }
    // one CTA per chain: 1024 threads while the chains leave SMs free (latency-bound
    // grids), 256 once several chains share an SM
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    const int coarse_threads =
        h->coarse_threads > 0 ? h->coarse_threads : ((!h->is_batch() || nc <= 2 * sms) ? 1024 : 256);
    launch_coarse_batch<T>((const CoarseJob<T>*)h->jobs_coarse, nc, coarse_threads, h->batch_coarse_smem, s, launches);
    for (int d = h->n_depth - 1; d >= 0; --d) {
        if (prof && d == 0) cudaEventRecordWithFlags(h->ev[2], s, cudaEventRecordExternal);
        if (d == 0 && h->stream_fine)
            launch_stream_fine((const StreamJob*)h->jobs_stream, (const StreamMaps*)h->maps_sbwd, h->njob_stream,
                               h->stream_strips, h->stream_ctas, true, s, launches);
        else if (h->s9_use[d])
            launch_stream9((const StreamJob*)h->jobs_s9[d], (const Stream9Maps*)h->maps_s9[d], h->njob_s9[d],
                           h->s9_strips[d], h->s9_grid[d], true, s, launches);
        else
            launch_tile_batch<T>((const TileJob<T>*)h->jobs_tile[d], (const TileMaps*)h->maps_bwd[d],
                                 h->njob_tile[d], h->per_tile[d], h->nblk_tile[d], d == 0 && h->fine0, true, false, s,
                                 launches);
        if (prof && d == 0) cudaEventRecordWithFlags(h->ev[3], s, cudaEventRecordExternal);
        launch_lowrank_batch<T>((const LowrankJob<T>*)h->jobs_lru[d], h->njob_lru[d], h->per_lru[d], h->nblk_lru[d],
                                false, s, launches);
    }
    launch_qoi_batch<T>((const QoiJob<T>*)h->jobs_qoi, nc, s, launches);
}

// The phases of one visit of grid l <= small_top and everything below it, with the slots
// of the per-launch path (enqueue_level).
void small_phases(const mgmc_ctx* h, int l, std::vector<int>& visit, std::vector<int4>& ops)
{
    const int v = visit[(size_t)l]++;
    if (l == 0) {
        ops.push_back(make_int4(kOpCoarsest, 0, v, 0));
        return;
    }
    const int S = std::max(1, std::max(h->cfg.nu1, h->cfg.nu2));
    for (int j = 0; j < h->cfg.nu1; ++j) {
        const int slot = 2 * (v * S + j);
        ops.push_back(make_int4(kOpSweep, l, slot, 0));
        ops.push_back(make_int4(kOpLowrank, l, slot, j == h->cfg.nu1 - 1 ? 4 : 0));
    }
    if (h->cfg.nu1 == 0) ops.push_back(make_int4(kOpLowrank, l, 0, 2 | 4));
    ops.push_back(make_int4(kOpRestrict, l, 0, 0));
    ops.push_back(make_int4(kOpZero, l - 1, 0, 0));
    const int calls = l == h->L - 1 ? 1 : h->cfg.gamma;
    for (int g = 0; g < calls; ++g) small_phases(h, l - 1, visit, ops);
    ops.push_back(make_int4(kOpProlong, l, 0, 0));
    for (int j = 0; j < h->cfg.nu2; ++j) {
        const int slot = 2 * (v * S + j) + 1;
        ops.push_back(make_int4(kOpSweep, l, slot, 1));
        ops.push_back(make_int4(kOpLowrank, l, slot, 1));
    }
}

// The visits of one cycle in the order enqueue_level makes them; every visit of grid
// small_top gets its phase list.
void plan_small(mgmc_ctx* h, int l, std::vector<int>& visit, std::vector<int4>& ops)
{
    if (l <= h->small_top) {
        h->small_off.push_back((int)ops.size());
        small_phases(h, l, visit, ops);
        h->small_cnt.push_back((int)ops.size() - h->small_off.back());
        return;
    }
    ++visit[(size_t)l];
    if (l == 0) return;
    const int calls = l == h->L - 1 ? 1 : h->cfg.gamma;
    for (int g = 0; g < calls; ++g) plan_small(h, l - 1, visit, ops);
}

// Alg. 1 on grid l of the general path, recursively: the v-th visit of the grid uses the
// noise slots 2 (v S + j) / 2 (v S + j) + 1, the coarsest grid's v-th sample slot v; the
// finest grid calls grid l-1 once, every other grid cfg.gamma times from psi = 0.
template <typename T>
void enqueue_level(mgmc_ctx* h, int l, std::vector<int>& visit, cudaStream_t s, int& launches)
{
    auto& lv = levels_of<T>(h);
    const DevProblem& P = h->P;
    const int Lf = h->L - 1;
    if (l <= h->small_top) {
        // this visit's phase list (built at creation in the same visit order)
        const int k = h->small_next++;
        launch_cycle_small<T>((const DevLevel<T>*)h->levels_dev, h->small_top, P, h->chol, h->n0,
                              h->small_ops + h->small_off[k], h->small_cnt[k], h->small_z, s, launches);
        return;
    }
    const int v = visit[(size_t)l]++;
    if (l == 0) {
        launch_coarsest_slot<T>(lv[0], P, h->chol, h->n0, (unsigned)v, s, launches);
        return;
    }
    const DevLevel<T>& D = lv[l];
    const int S = std::max(1, std::max(h->cfg.nu1, h->cfg.nu2));
    const bool prof = h->profile && l == Lf;
    for (int j = 0; j < h->cfg.nu1; ++j) {
        const unsigned slot = (unsigned)(2 * (v * S + j));
        if (prof && j == 0) cudaEventRecordWithFlags(h->ev[0], s, cudaEventRecordExternal);
        launch_sweep<T>(D, P, 0, slot, s, launches);
        if (prof && j == 0) cudaEventRecordWithFlags(h->ev[1], s, cudaEventRecordExternal);
        launch_lowrank<T>(D, P, 0, slot, j == h->cfg.nu1 - 1, s, launches);
    }
    if (h->cfg.nu1 == 0) launch_lowrank<T>(D, P, -1, 0u, true, s, launches);
    launch_restrict<T>(D, lv[l - 1], s, launches);
    cudaMemsetAsync(lv[l - 1].x, 0, (size_t)lv[l - 1].alloc * sizeof(T), s);
    const int calls = l == Lf ? 1 : h->cfg.gamma;
    for (int g = 0; g < calls; ++g) enqueue_level<T>(h, l - 1, visit, s, launches);
    launch_prolong<T>(lv[l - 1], D, s, launches);
    for (int j = 0; j < h->cfg.nu2; ++j) {
        const unsigned slot = (unsigned)(2 * (v * S + j) + 1);
        if (prof && j == 0) cudaEventRecordWithFlags(h->ev[2], s, cudaEventRecordExternal);
        launch_sweep<T>(D, P, 1, slot, s, launches);
        if (prof && j == 0) cudaEventRecordWithFlags(h->ev[3], s, cudaEventRecordExternal);
        launch_lowrank<T>(D, P, 1, slot, false, s, launches);
    }
}

template <typename T>
void enqueue_cycle(mgmc_ctx* h, cudaStream_t s, int& launches)
{
    if (h->is_batch() || h->fused) {
        enqueue_cycle_batch<T>(h, s, launches);
        return;
    }
    if (h->recursive && !h->cfg.gibbs) {
        h->small_next = 0;
        std::vector<int> visit((size_t)h->L, 0);
        enqueue_level<T>(h, h->L - 1, visit, s, launches);
        launch_qoi<T>(levels_of<T>(h)[h->L - 1], h->n_qoi, h->q_site, h->q_w, h->P, s, launches);
        return;
    }
    auto& lv = levels_of<T>(h);
    const int Lf = h->L - 1;
    const DevProblem& P = h->P;
    const bool prof = h->profile && h->top < Lf;
    if (h->cfg.gibbs) {
        // plain Gibbs sampler (Sec. 5.1.3): the finest grid's sweeps of the V-cycle, no coarse correction
        const DevLevel<T>& D = lv[Lf];
        for (int j = 0; j < h->cfg.nu1; ++j) {
            if (prof && j == 0) cudaEventRecordWithFlags(h->ev[0], s, cudaEventRecordExternal);
            launch_sweep<T>(D, P, 0, (unsigned)(2 * j), s, launches);
            if (prof && j == 0) cudaEventRecordWithFlags(h->ev[1], s, cudaEventRecordExternal);
            launch_lowrank<T>(D, P, 0, (unsigned)(2 * j), false, s, launches);
        }
        for (int j = 0; j < h->cfg.nu2; ++j) {
            if (prof && j == 0) cudaEventRecordWithFlags(h->ev[2], s, cudaEventRecordExternal);
            launch_sweep<T>(D, P, 1, (unsigned)(2 * j + 1), s, launches);
            if (prof && j == 0) cudaEventRecordWithFlags(h->ev[3], s, cudaEventRecordExternal);
            launch_lowrank<T>(D, P, 1, (unsigned)(2 * j + 1), false, s, launches);
        }
        launch_qoi<T>(D, h->n_qoi, h->q_site, h->q_w, P, s, launches);
        return;
    }
    for (int l = Lf; l > h->top; --l) {
        const DevLevel<T>& D = lv[l];
        if (l < Lf) cudaMemsetAsync(D.x, 0, (size_t)D.alloc * sizeof(T), s);
        for (int j = 0; j < h->cfg.nu1; ++j) {
            if (prof && l == Lf && j == 0) cudaEventRecordWithFlags(h->ev[0], s, cudaEventRecordExternal);
            launch_sweep<T>(D, P, 0, (unsigned)(2 * j), s, launches);
            if (prof && l == Lf && j == 0) cudaEventRecordWithFlags(h->ev[1], s, cudaEventRecordExternal);
            launch_lowrank<T>(D, P, 0, (unsigned)(2 * j), j == h->cfg.nu1 - 1, s, launches);
        }
        if (h->cfg.nu1 == 0) launch_lowrank<T>(D, P, -1, 0u, true, s, launches);
        launch_restrict<T>(D, lv[l - 1], s, launches);
    }
    launch_coarse<T>((const DevLevel<T>*)h->levels_dev, h->cfg.dim, h->top, h->top == Lf, P, h->chol, h->n0,
                     h->cfg.nu1, h->cfg.nu2, h->coarse_smem, s, launches);
    for (int l = h->top + 1; l <= Lf; ++l) {
        const DevLevel<T>& D = lv[l];
        launch_prolong<T>(lv[l - 1], D, s, launches);
        for (int j = 0; j < h->cfg.nu2; ++j) {
            if (prof && l == Lf && j == 0) cudaEventRecordWithFlags(h->ev[2], s, cudaEventRecordExternal);
            launch_sweep<T>(D, P, 1, (unsigned)(2 * j + 1), s, launches);
            if (prof && l == Lf && j == 0) cudaEventRecordWithFlags(h->ev[3], s, cudaEventRecordExternal);
            launch_lowrank<T>(D, P, 1, (unsigned)(2 * j + 1), false, s, launches);
        }
    }
    launch_qoi<T>(lv[Lf], h->n_qoi, h->q_site, h->q_w, P, s, launches);
}

mgmc_status ensure_graph(mgmc_ctx* h)
{
    if (h->exec) return MGMC_OK;
    cudaGraph_t graph = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    int launches = 0;
    if (h->fp32())
        enqueue_cycle<float>(h, h->cap_stream, launches);
    else
        enqueue_cycle<double>(h, h->cap_stream, launches);
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
    if (e != cudaSuccess) return fail(MGMC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        h->exec = nullptr;
        return fail(MGMC_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    h->launches = launches;
    return MGMC_OK;
}

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

mgmc_status check_device()
{
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
        cudaGetLastError();
        return fail(MGMC_ERR_CUDA, "no CUDA device available (the sampler has no CPU fallback)");
    }
    return MGMC_OK;
}

// The sticky status bits of every chain of a handle (the work queued on `s` is
// waited for first): reported as a status and cleared, so that the handle can be
// used again.  Timeouts are reported before non-finite values.
mgmc_status take_status(mgmc_ctx* h, cudaStream_t s)
{
    CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<mgmc_ctx*> chains = h->is_batch() ? h->sub : std::vector<mgmc_ctx*>{h};
    int bits = 0, first = -1;
    for (size_t c = 0; c < chains.size(); ++c) {
        int v = 0;
        CUDA_TRY(cudaMemcpy(&v, &chains[c]->cs->status, sizeof(int), cudaMemcpyDeviceToHost));
        if (v && first < 0) first = (int)c;
        bits |= v;
        if (v) CUDA_TRY(cudaMemset(&chains[c]->cs->status, 0, sizeof(int)));
    }
    const std::string who = h->is_batch() ? " (chain " + std::to_string(first) + " first)" : std::string();
    if (bits & kStatusLayout)
        return fail(MGMC_ERR_CUDA, "a kernel's shared-memory layout exceeded its launch (not run)" + who);
    if (bits & kStatusTimeout) return fail(MGMC_ERR_TIMEOUT, "a kernel's bounded staging wait gave up" + who);
    if (bits & kStatusNumeric) return fail(MGMC_ERR_NUMERIC, "non-finite QoI produced" + who);
    return MGMC_OK;
}

}  // namespace

extern "C" {

const char* mgmc_last_error(void) { return g_last_error.c_str(); }

mgmc_status mgmc_check_status(mgmc_handle h, void* stream)
{
    if (!h) return fail(MGMC_ERR_ARG, "handle is NULL");
    CUDA_TRY(cudaSetDevice(h->device));
    return take_status(h, (cudaStream_t)stream);
}

mgmc_status mgmc_set_wait_limit(mgmc_handle h, int64_t limit_ns)
{
    if (!h) return fail(MGMC_ERR_ARG, "handle is NULL");
    CUDA_TRY(cudaSetDevice(h->device));
    CUDA_TRY(cudaDeviceSynchronize());
    std::vector<mgmc_ctx*> chains = h->is_batch() ? h->sub : std::vector<mgmc_ctx*>{h};
    const long long v = (long long)limit_ns;
    for (mgmc_ctx* c : chains) CUDA_TRY(cudaMemcpy(&c->cs->wait_ns, &v, sizeof(v), cudaMemcpyHostToDevice));
    return MGMC_OK;
}

mgmc_status mgmc_config_default(mgmc_config* cfg, int dim, int n)
{
    if (!cfg) return fail(MGMC_ERR_ARG, "cfg is NULL");
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->dim = dim;
    cfg->n = n;
    cfg->n_levels = 0;
    cfg->nu1 = 1;
    cfg->nu2 = 1;
    cfg->precision = MGMC_FP64;
    cfg->scale_hd = 1;
    cfg->coarse_max_n = 0;
    cfg->gibbs = 0;
    cfg->band_min_n = 0;
    return MGMC_OK;
}

mgmc_status mgmc_point_obs_rows(int dim, int n, int m, const double* xyz, int32_t* obs_site, double* obs_w)
{
    if ((dim != 2 && dim != 3) || n < 1 || m < 0 || (m > 0 && (!xyz || !obs_site || !obs_w)))
        return fail(MGMC_ERR_ARG, "mgmc_point_obs_rows: bad arguments");
    const double h = 1.0 / (double)(n + 1);
    const int nc = 1 << dim;
    for (int k = 0; k < m; ++k) {
        long long cell[3];
        double t[3];
        for (int a = 0; a < dim; ++a) {
            double v = xyz[(size_t)k * dim + a];
            if (!(v > 0.0 && v < 1.0)) return fail(MGMC_ERR_ARG, "observation point outside (0,1)^dim");
            long long c = (long long)std::floor(v / h);
            if (c > n) c = n;
            cell[a] = c;
            t[a] = v / h - (double)c;
        }
        for (int corner = 0; corner < nc; ++corner) {
            double w = 1.0;
            long long idx[3] = {0, 0, 0};
            bool inside = true;
            for (int a = 0; a < dim; ++a) {
                int up = (corner >> a) & 1;
                w *= up ? t[a] : (1.0 - t[a]);
                idx[a] = cell[a] + up - 1;
                if (idx[a] < 0 || idx[a] >= n) inside = false;
            }
            size_t o = (size_t)k * nc + corner;
            if (inside && w != 0.0) {
                obs_site[o] = (int32_t)(idx[0] + n * (idx[1] + (dim == 3 ? (long long)n * idx[2] : 0)));
                obs_w[o] = w;
            } else {
                obs_site[o] = -1;
                obs_w[o] = 0.0;
            }
        }
    }
    return MGMC_OK;
}

mgmc_status mgmc_create(const mgmc_config* cfg_in, const mgmc_allocator* alloc, void* stream,
                        const double* kappa2, double kappa2_const, int m, const int32_t* obs_site,
                        const double* obs_w, int nnz_per_obs, const double* Gamma, const double* y, int n_qoi,
                        const int32_t* qoi_site, const double* qoi_w, mgmc_handle* out)
{
    if (!out) return fail(MGMC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg_in) return fail(MGMC_ERR_ARG, "cfg is NULL");
    mgmc_config cfg = *cfg_in;
    if (cfg.dim != 2 && cfg.dim != 3) return fail(MGMC_ERR_ARG, "dim must be 2 or 3");
    if (cfg.n < 1 || ((cfg.n + 1) & cfg.n) != 0) return fail(MGMC_ERR_ARG, "n must be 2^k - 1");
    if (cfg.precision != MGMC_FP32 && cfg.precision != MGMC_FP64) return fail(MGMC_ERR_ARG, "bad precision");
    if (cfg.nu1 < 0 || cfg.nu2 < 0 || cfg.nu1 > 16 || cfg.nu2 > 16) return fail(MGMC_ERR_ARG, "nu1/nu2 out of range");
    if (cfg.band_min_n < 0) return fail(MGMC_ERR_ARG, "band_min_n must be >= 0");
    if (m < 0 || m > MGMC_MAX_OBS) return fail(MGMC_ERR_ARG, "number of observations out of range");
    if (m > 0 && (!obs_site || !obs_w || !Gamma || !y || nnz_per_obs < 1))
        return fail(MGMC_ERR_ARG, "observation arrays missing");
    if (n_qoi < 0 || (n_qoi > 0 && (!qoi_site || !qoi_w))) return fail(MGMC_ERR_ARG, "QoI arrays missing");
    if (!kappa2 && !(std::isfinite(kappa2_const) && kappa2_const >= 0.0))
        return fail(MGMC_ERR_ARG, "kappa2_const must be finite and non-negative");
    long long N = 1;
    for (int a = 0; a < cfg.dim; ++a) N *= cfg.n;
    if (N > (1LL << 31) - 1) return fail(MGMC_ERR_ARG, "grid too large");
    int max_levels = 1;
    for (int nn = cfg.n; nn >= 3; nn = (nn - 1) / 2) ++max_levels;
    if (cfg.n_levels == 0) cfg.n_levels = max_levels;
    if (cfg.n_levels < 1 || cfg.n_levels > max_levels) return fail(MGMC_ERR_ARG, "n_levels out of range");
    if (cfg.disc == MGMC_SSL && cfg.precision != MGMC_FP64)
        return fail(MGMC_ERR_ARG, "the squared shifted Laplacian runs in FP64");
    if (cfg.gamma < 0 || cfg.gamma > 2) return fail(MGMC_ERR_ARG, "gamma must be 0, 1 or 2");
    if (cfg.gamma == 0) cfg.gamma = cfg.disc == MGMC_SSL ? 2 : 1;
    {
        // the noise slots of the last visit of the coarsest grid must fit 16 bits
        double visits = 1.0;
        for (int l = cfg.n_levels - 2; l >= 1; --l) visits *= cfg.gamma;
        const int S = std::max(1, std::max(cfg.nu1, cfg.nu2));
        if (2.0 * visits * S > 65536.0) return fail(MGMC_ERR_ARG, "too many grid visits per cycle for the noise slots");
    }
    if (cfg.gibbs != 0 && cfg.gibbs != 1) return fail(MGMC_ERR_ARG, "gibbs must be 0 or 1");
    if (cfg.gibbs && cfg.n_levels < 2) return fail(MGMC_ERR_ARG, "the Gibbs sampler needs n_levels >= 2");
    for (int t = 0; t < n_qoi; ++t)
        if (qoi_site[t] < 0 || qoi_site[t] >= N || !std::isfinite(qoi_w[t]))
            return fail(MGMC_ERR_ARG, "QoI site out of range or weight not finite");
    mgmc_status dst = check_device();
    if (dst != MGMC_OK) return dst;

    HostProblem hp;
    int code = MGMC_OK;
    std::string err = build_hierarchy(hp, cfg.dim, cfg.n, cfg.n_levels, cfg.scale_hd, cfg.disc, kappa2, kappa2_const, m,
                                      obs_site, obs_w, nnz_per_obs, Gamma, y, &code);
    if (!err.empty()) return fail((mgmc_status)code, err);

    mgmc_ctx* h = new mgmc_ctx();
    h->cfg = cfg;
    h->L = cfg.n_levels;
    h->m = m;
    cudaGetDevice(&h->device);
    h->buf.stream = (cudaStream_t)stream;
    if (alloc && alloc->alloc && alloc->free) {
        h->buf.alloc = *alloc;
        h->buf.use_cuda_malloc = false;
    }
    // grids inside the single-CTA coarse kernel: n <= coarse_max_n, and the state and
    // right-hand side of all of them must fit in shared memory
    int cmax = cfg.coarse_max_n > 0 ? cfg.coarse_max_n : (cfg.dim == 2 ? 63 : 15);
    h->top = 0;
    {
        const size_t esz = cfg.precision == MGMC_FP32 ? 4 : 8;
        const size_t budget = 200 * 1024;
        std::vector<int> nl;
        for (int l = 0; l < h->L; ++l) nl.push_back(hp.lev[l].n);
        for (int l = 0; l < h->L && l < kCoarseMaxLevels; ++l) {
            size_t bytes = (size_t)coarse_smem_elems(cfg.dim, nl.data(), l, l == h->L - 1 && cfg.disc == 0) * esz;
            if (hp.lev[l].n <= cmax && bytes + 16384 <= budget) h->top = l;
        }
    }
    // the Gibbs sampler sweeps the finest grid with the unfused kernels, outside the coarse
    // kernel; W-cycles and radius-2 grids run every grid above the coarsest on the general
    // path, the cycle enqueued recursively
    h->recursive = cfg.gamma == 2 || cfg.disc == MGMC_SSL;
    if (cfg.gibbs || h->recursive) h->top = 0;
    h->n0 = hp.n0;
    h->f_norm = hp.f_norm;
    h->fused = cfg.dim == 2 && cfg.nu1 == 1 && cfg.nu2 == 1 && !cfg.gibbs && !h->recursive;
    auto cleanup = [&](mgmc_status s) {
        h->buf.release();
        delete h;
        return s;
    };
    mgmc_status st = MGMC_OK;
    h->cs = (CycleState*)h->buf.get(sizeof(CycleState));
    if (!h->cs) return cleanup(fail(MGMC_ERR_OOM, "allocator returned NULL"));
    if (cudaMemsetAsync(h->cs, 0, sizeof(CycleState), h->buf.stream) != cudaSuccess)
        return cleanup(fail(MGMC_ERR_CUDA, "memset failed"));
    h->P.m = m;
    h->P.cs = h->cs;
    h->P.gamma_diag = hp.gamma_diag ? 1 : 0;
    if (m > 0) {
        h->P.Gamma_inv = upload(h, hp.Gamma_inv, st);
        h->P.LG = upload(h, hp.LG, st);
    }
    h->chol = upload(h, hp.chol0, st);
    if (st != MGMC_OK) return cleanup(fail(st, "device upload failed"));
    st = h->fp32() ? build_device_levels<float>(h, hp) : build_device_levels<double>(h, hp);
    if (st != MGMC_OK) return cleanup(st);
    // recursive path (2D): the grids with n <= coarse_max_n (0: 63) in one CTA per visit
    if (h->recursive && !cfg.gibbs && cfg.dim == 2) {
        const int thr = cfg.coarse_max_n > 0 ? cfg.coarse_max_n : 63;
        for (int l = 0; l < h->L && l < kSmallMaxLevels; ++l)
            if (hp.lev[l].n <= thr) h->small_top = l;
        if (h->small_top >= 1) {
            std::vector<int> visit((size_t)h->L, 0);
            std::vector<int4> ops;
            plan_small(h, h->L - 1, visit, ops);
            h->small_ops = upload(h, ops, st);
            long long zmax = 1;
            for (int l = 0; l <= h->small_top; ++l) zmax = std::max(zmax, (long long)hp.lev[l].n * hp.lev[l].n);
            h->small_z = (double*)h->buf.get((size_t)zmax * sizeof(double));
            if (!h->small_z) return cleanup(fail(MGMC_ERR_OOM, "allocator returned NULL"));
            if (st != MGMC_OK) return cleanup(fail(st, "device upload failed"));
        } else {
            h->small_top = -1;
        }
    }
    h->P_dev = (DevProblem*)h->buf.get(sizeof(DevProblem));
    if (!h->P_dev) return cleanup(fail(MGMC_ERR_OOM, "allocator returned NULL"));
    if (cudaMemcpyAsync(h->P_dev, &h->P, sizeof(DevProblem), cudaMemcpyHostToDevice, h->buf.stream) != cudaSuccess)
        return cleanup(fail(MGMC_ERR_CUDA, "upload failed"));
    // QoI (finest-level padded offsets)
    h->n_qoi = n_qoi;
    {
        const HostLevel& F = hp.lev[h->L - 1];
        const int pitch = h->fp32() ? h->lf[h->L - 1].pitch : h->ld[h->L - 1].pitch;
        const long long plane = h->fp32() ? h->lf[h->L - 1].plane : h->ld[h->L - 1].plane;
        const long long base = h->fp32() ? h->lf[h->L - 1].base : h->ld[h->L - 1].base;
        std::vector<long long> qs;
        std::vector<double> qw;
        for (int t = 0; t < n_qoi; ++t) {
            long long s = qoi_site[t];
            int i = (int)(s % F.n), j = (int)((s / F.n) % F.n), k = cfg.dim == 3 ? (int)(s / ((long long)F.n * F.n)) : 0;
            qs.push_back(site_offset(cfg.dim, pitch, plane, base, i, j, k));
            qw.push_back(qoi_w[t]);
        }
        h->q_site = upload(h, qs, st);
        h->q_w = upload(h, qw, st);
    }
    // staging and mean-solve scratch
    size_t esz = h->fp32() ? 4 : 8;
    h->x_stage = h->buf.get((size_t)N * esz);
    h->u = (double*)h->buf.get(sizeof(double) * (m > 0 ? m : 1));
    h->max_partial = (int)((N + 255) / 256);
    h->partial = (double*)h->buf.get(sizeof(double) * h->max_partial);
    h->rnorm = (double*)h->buf.get(sizeof(double) * 2);
    if (!h->x_stage || !h->u || !h->partial || !h->rnorm || st != MGMC_OK)
        return cleanup(fail(MGMC_ERR_OOM, "allocator returned NULL"));
    // job tables of the fused 2D cycle (needs the QoI arrays above)
    if (h->fused) {
        st = h->fp32() ? build_batch_tables<float>(h) : build_batch_tables<double>(h);
        if (st != MGMC_OK) return cleanup(st);
    }
    if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return cleanup(fail(MGMC_ERR_CUDA, "stream creation failed"));
    cudaError_t e = cudaStreamSynchronize(h->buf.stream);
    if (e != cudaSuccess) {
        cudaStreamDestroy(h->cap_stream);
        return cleanup(fail(MGMC_ERR_CUDA, std::string("set-up upload: ") + cudaGetErrorString(e)));
    }
    *out = h;
    return MGMC_OK;
}

mgmc_status mgmc_fine_operator(const mgmc_config* cfg, const double* kappa2, double kappa2_const, double* out)
{
    if (!cfg || !out || (cfg->dim != 2 && cfg->dim != 3) || cfg->n < 1)
        return fail(MGMC_ERR_ARG, "mgmc_fine_operator: bad arguments");
    {
        int k = cfg->n + 1;
        while (k % 2 == 0) k /= 2;
        if (k != 1) return fail(MGMC_ERR_ARG, "n must be 2^k - 1");
    }
    HostProblem hp;
    hp.dim = cfg->dim;
    hp.R = cfg->disc == MGMC_SSL ? 2 : 1;
    hp.NS = cfg->dim == 2 ? (2 * hp.R + 1) * (2 * hp.R + 1) : 27;
    hp.C = (hp.NS - 1) / 2;
    hp.n_levels = 1;
    hp.scale_hd = cfg->scale_hd;
    hp.disc = cfg->disc;
    hp.lev.assign(1, HostLevel());
    hp.lev[0].n = cfg->n;
    hp.lev[0].N = cfg->dim == 2 ? (long long)cfg->n * cfg->n : (long long)cfg->n * cfg->n * cfg->n;
    if (cfg->disc != MGMC_FD && cfg->disc != MGMC_Q1 && cfg->disc != MGMC_SSL)
        return fail(MGMC_ERR_ARG, "disc must be MGMC_FD, MGMC_Q1 or MGMC_SSL");
    if (cfg->disc != MGMC_FD && kappa2)
        return fail(MGMC_ERR_ARG, "the Q1 and squared-operator discretisations take a constant kappa^2 (kappa2 = NULL)");
    if (cfg->disc == MGMC_SSL && cfg->dim != 2)
        return fail(MGMC_ERR_ARG, "the squared shifted Laplacian is two-dimensional");
    std::string err = fine_operator(hp, cfg->dim, cfg->n, cfg->scale_hd, cfg->disc, kappa2, kappa2_const);
    if (!err.empty()) return fail(MGMC_ERR_ARG, err);
    const std::vector<double>& st = hp.lev[0].st;
    std::memcpy(out, st.data(), st.size() * sizeof(double));
    return MGMC_OK;
}

mgmc_status mgmc_info(mgmc_handle h, int* n_levels, int* precision, int* dim)
{
    if (!h) return fail(MGMC_ERR_ARG, "handle is NULL");
    if (n_levels) *n_levels = h->L;
    if (precision) *precision = h->cfg.precision;
    if (dim) *dim = h->cfg.dim;
    return MGMC_OK;
}

mgmc_status mgmc_level_n(mgmc_handle h, int l, int* n)
{
    if (!h || !n || l < 0 || l >= h->L) return fail(MGMC_ERR_ARG, "bad level query");
    *n = h->fp32() ? h->lf[l].n : h->ld[l].n;
    return MGMC_OK;
}

mgmc_status mgmc_launches_per_cycle(mgmc_handle h, int* launches)
{
    if (!h || !launches) return fail(MGMC_ERR_ARG, "bad arguments");
    mgmc_status st = ensure_graph(h);
    if (st != MGMC_OK) return st;
    *launches = h->launches;
    return MGMC_OK;
}

static mgmc_status pack_in(mgmc_ctx* h, void* x, bool host, cudaStream_t s, long long N)
{
    size_t esz = h->fp32() ? 4 : 8;
    void* src = x;
    if (host) {
        CUDA_TRY(cudaMemcpyAsync(h->x_stage, x, (size_t)N * esz, cudaMemcpyHostToDevice, s));
        src = h->x_stage;
    }
    if (h->jobs_pack) {
        void* d[1] = {src};
        if (h->fp32())
            launch_pack_batch<float>((const PackJob<float>*)h->jobs_pack, d, 1, h->pack_max_n, true, s);
        else
            launch_pack_batch<double>((const PackJob<double>*)h->jobs_pack, d, 1, h->pack_max_n, true, s);
    } else if (h->fp32()) {
        launch_pack<float>(h->lf[h->L - 1], (float*)src, true, s);
    } else {
        launch_pack<double>(h->ld[h->L - 1], (double*)src, true, s);
    }
    return MGMC_OK;
}

static mgmc_status pack_out(mgmc_ctx* h, void* x, bool host, cudaStream_t s, long long N)
{
    size_t esz = h->fp32() ? 4 : 8;
    void* dst = host ? h->x_stage : x;
    if (h->jobs_pack) {
        void* d[1] = {dst};
        if (h->fp32())
            launch_pack_batch<float>((const PackJob<float>*)h->jobs_pack, d, 1, h->pack_max_n, false, s);
        else
            launch_pack_batch<double>((const PackJob<double>*)h->jobs_pack, d, 1, h->pack_max_n, false, s);
    } else if (h->fp32()) {
        launch_pack<float>(h->lf[h->L - 1], (float*)dst, false, s);
    } else {
        launch_pack<double>(h->ld[h->L - 1], (double*)dst, false, s);
    }
    if (host) CUDA_TRY(cudaMemcpyAsync(x, h->x_stage, (size_t)N * esz, cudaMemcpyDeviceToHost, s));
    return MGMC_OK;
}

mgmc_status mgmc_sample(mgmc_handle h, int64_t n_steps, uint64_t seed, uint64_t step_offset, uint32_t chain,
                        void* x_inout, double* qoi_out, void* stream)
{
    if (!h) return fail(MGMC_ERR_ARG, "handle is NULL");
    if (n_steps < 0) return fail(MGMC_ERR_ARG, "n_steps < 0");
    if (chain > 0xFFFFu) return fail(MGMC_ERR_ARG, "chain must be < 65536");
    if (n_steps == 0) return MGMC_OK;
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaSetDevice(h->device));
    long long N = 1;
    for (int a = 0; a < h->cfg.dim; ++a) N *= h->cfg.n;
    const bool resume = x_inout == nullptr;
    bool xhost = !resume && !is_device_ptr(x_inout);
    bool qhost = qoi_out && !is_device_ptr(qoi_out);
    double* qdev = qoi_out;
    if (qhost) {
        CUDA_TRY(cudaMallocAsync((void**)&qdev, sizeof(double) * (size_t)n_steps, s));
    }
    mgmc_status st = ensure_graph(h);
    if (st != MGMC_OK) return st;
    if (!resume) {
        st = pack_in(h, x_inout, xhost, s, N);
        if (st != MGMC_OK) return st;
    }
    launch_set_cycle(h->cs, seed, step_offset, chain, 1, qdev, s);
    for (int64_t t = 0; t < n_steps; ++t) CUDA_TRY(cudaGraphLaunch(h->exec, s));
    if (!resume) {
        st = pack_out(h, x_inout, xhost, s, N);
        if (st != MGMC_OK) return st;
    }
    if (qhost) {
        CUDA_TRY(cudaMemcpyAsync(qoi_out, qdev, sizeof(double) * (size_t)n_steps, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaFreeAsync(qdev, s));
    }
    CUDA_TRY(cudaGetLastError());
    if (xhost || qhost) return take_status(h, s);
    return MGMC_OK;
}

mgmc_status mgmc_mean_solve(mgmc_handle h, double rtol, int max_cycles, void* mean_out, int* cycles_done,
                            double* rel_residual, void* stream)
{
    if (!h || !mean_out) return fail(MGMC_ERR_ARG, "bad arguments");
    if (max_cycles < 0 || !(rtol >= 0.0)) return fail(MGMC_ERR_ARG, "bad rtol / max_cycles");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaSetDevice(h->device));
    long long N = 1;
    for (int a = 0; a < h->cfg.dim; ++a) N *= h->cfg.n;
    bool xhost = !is_device_ptr(mean_out);
    mgmc_status st = ensure_graph(h);
    if (st != MGMC_OK) return st;
    st = pack_in(h, mean_out, xhost, s, N);
    if (st != MGMC_OK) return st;
    launch_set_cycle(h->cs, 0, 0, 0, 0, nullptr, s);
    auto resid = [&](double& rr) -> mgmc_status {
        if (h->fp32())
            launch_resid<float>(h->lf[h->L - 1], h->P, h->u, h->partial, h->max_partial, h->rnorm, s);
        else
            launch_resid<double>(h->ld[h->L - 1], h->P, h->u, h->partial, h->max_partial, h->rnorm, s);
        double r2 = 0.0;
        CUDA_TRY(cudaMemcpyAsync(&r2, h->rnorm, sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        double r = std::sqrt(r2);
        rr = h->f_norm > 0.0 ? r / h->f_norm : (r == 0.0 ? 0.0 : INFINITY);
        return MGMC_OK;
    };
    double rr = 0.0;
    st = resid(rr);
    if (st != MGMC_OK) return st;
    int c = 0;
    while (rr > rtol && c < max_cycles) {
        int chunk = c < 4 ? 1 : 2;
        for (int t = 0; t < chunk && c < max_cycles; ++t, ++c) CUDA_TRY(cudaGraphLaunch(h->exec, s));
        st = resid(rr);
        if (st != MGMC_OK) return st;
        if (!std::isfinite(rr)) return fail(MGMC_ERR_NUMERIC, "mean solve diverged");
    }
    st = pack_out(h, mean_out, xhost, s, N);
    if (st != MGMC_OK) return st;
    st = take_status(h, s);
    if (st != MGMC_OK) return st;
    if (cycles_done) *cycles_done = c;
    if (rel_residual) *rel_residual = rr;
    return MGMC_OK;
}

mgmc_status mgmc_set_profiling(mgmc_handle h, int enable)
{
    if (!h) return fail(MGMC_ERR_ARG, "handle is NULL");
    bool want = enable != 0;
    if (want == h->profile) return MGMC_OK;
    CUDA_TRY(cudaSetDevice(h->device));
    if (want && !h->ev[0])
        for (int i = 0; i < 4; ++i) CUDA_TRY(cudaEventCreate(&h->ev[i]));
    h->profile = want;
    if (h->exec) {
        CUDA_TRY(cudaDeviceSynchronize());
        cudaGraphExecDestroy(h->exec);
        h->exec = nullptr;
    }
    return MGMC_OK;
}

mgmc_status mgmc_set_band_min_n(mgmc_handle h, int band_min_n)
{
    if (!h) return fail(MGMC_ERR_ARG, "handle is NULL");
    if (band_min_n < 0) return fail(MGMC_ERR_ARG, "band_min_n must be >= 0");
    CUDA_TRY(cudaSetDevice(h->device));
    h->cfg.band_min_n = band_min_n;
    const std::vector<char> before = h->s9_use;
    apply_band_min(h);
    if (h->exec && h->s9_use != before) {
        CUDA_TRY(cudaDeviceSynchronize());
        cudaGraphExecDestroy(h->exec);
        h->exec = nullptr;
    }
    return MGMC_OK;
}

mgmc_status mgmc_set_coarse_threads(mgmc_handle h, int threads)
{
    if (!h) return fail(MGMC_ERR_ARG, "handle is NULL");
    if (threads != 0 && (threads < 64 || threads > 1024 || threads % 32 != 0))
        return fail(MGMC_ERR_ARG, "coarse threads must be 0 or a multiple of 32 in [64, 1024]");
    CUDA_TRY(cudaSetDevice(h->device));
    if (threads == h->coarse_threads) return MGMC_OK;
    h->coarse_threads = threads;
    if (h->exec) {
        CUDA_TRY(cudaDeviceSynchronize());
        cudaGraphExecDestroy(h->exec);
        h->exec = nullptr;
    }
    return MGMC_OK;
}

mgmc_status mgmc_profile_times(mgmc_handle h, float* ms, int n, void* stream)
{
    if (!h || !ms || n < 2) return fail(MGMC_ERR_ARG, "bad arguments");
    const bool tiled = (h->is_batch() || h->fused) ? h->n_depth > 0 : h->top < h->L - 1;
    if (!h->profile || !tiled)
        return fail(MGMC_ERR_STATE, "profiling is off or the finest grid runs in the single-CTA kernel");
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    CUDA_TRY(cudaEventElapsedTime(&ms[0], h->ev[0], h->ev[1]));
    CUDA_TRY(cudaEventElapsedTime(&ms[1], h->ev[2], h->ev[3]));
    return MGMC_OK;
}

}  // extern "C"

namespace {

// which depths run in the streaming band kernels: the eligible ones (FP32 9-point
// grids below the finest) whose smallest grid has n >= band_min_n (default 255)
constexpr int kBandMinDefault = 255;
void apply_band_min(mgmc_ctx* h)
{
    const int band_min = h->cfg.band_min_n > 0 ? h->cfg.band_min_n : kBandMinDefault;
    h->s9_use.assign(h->s9_ok.size(), 0);
    for (size_t d = 0; d < h->s9_ok.size(); ++d) h->s9_use[d] = h->s9_ok[d] && h->s9_minn[d] >= band_min;
}

template <typename T>
mgmc_status build_batch_tables(mgmc_ctx* h)
{
    std::vector<mgmc_ctx*> chains = h->is_batch() ? h->sub : std::vector<mgmc_ctx*>{h};
    const int nc = (int)chains.size();
    mgmc_status st = MGMC_OK;
    int depth = 0;
    for (mgmc_ctx* c : chains) depth = std::max(depth, c->L - 1 - c->top);
    h->n_depth = depth;
    // depth 0: the finest grids (5-point finite differences, or Q1 -- stored like the
    // Galerkin grids); a batch holds one discretisation
    h->fine0 = true;
    for (mgmc_ctx* c : chains)
        if (c->L - 1 > c->top && !levels_of<T>(c)[c->L - 1].fine) h->fine0 = false;
    // FP32 5-point finest grids run in the streaming kernels; their low-rank steps then
    // read the state at the observation entries (no z partials)
    h->stream_fine = false;
    if constexpr (std::is_same<T, float>::value) {
        if (depth > 0 && h->fine0) {
            cudaError_t e = stream_prepare();
            if (e != cudaSuccess)
                return fail(MGMC_ERR_CUDA, std::string("stream kernel set-up: ") + cudaGetErrorString(e));
            std::vector<StreamJob> sj;
            std::vector<StreamMaps> sf, sb;
            long long strips = 0;
            for (mgmc_ctx* c : chains) {
                const int l = c->L - 1;
                if (l <= c->top) continue;
                const auto& lv = levels_of<float>(c);
                StreamJob J{};
                J.L = lv[l];
                J.C = lv[l - 1];
                J.cs = c->cs;
                J.strip0 = strips;
                J.spb = (J.L.n + kStreamRows - 1) / kStreamRows;
                J.nbands = (J.L.n + kStreamBand - 1) / kStreamBand;
                strips += (long long)J.spb * J.nbands;
                sj.push_back(J);
                sf.emplace_back();
                sb.emplace_back();
                if (!make_stream_maps(J.L, J.C, false, &sf.back()) || !make_stream_maps(J.L, J.C, true, &sb.back()))
                    return fail(MGMC_ERR_CUDA, "TMA descriptor encoding failed");
            }
            h->jobs_stream = upload(h, sj, st);
            h->maps_sfwd = upload(h, sf, st);
            h->maps_sbwd = upload(h, sb, st);
            if (st != MGMC_OK) return fail(st, "stream table upload failed");
            h->njob_stream = (int)sj.size();
            h->stream_strips = strips;
            h->stream_ctas = stream_grid(strips);
            h->stream_fine = true;
        }
    }
    for (int d = 0; d < depth; ++d) {
        std::vector<TileJob<T>> tj;
        std::vector<TileMaps> mf, mb;
        std::vector<LowrankJob<T>> ld, lu;
        int tiles = 0, bd = 0, bu = 0;
        // FP32 9-point grids below the finest: the streaming band kernels can take this
        // depth (which of the two kernel families runs is set by band_min_n, see
        // apply_band_min); the low-rank steps then read the state at the observation
        // entries, whichever family wrote it
        bool s9 = false;
        int s9_minn = 0;
        if constexpr (std::is_same<T, float>::value) {
            if (d > 0) {
                s9 = true;
                s9_minn = INT_MAX;
                for (mgmc_ctx* c : chains) {
                    const int l = c->L - 1 - d;
                    if (l <= c->top) continue;
                    const DevLevel<T>& Lh = levels_of<T>(c)[l];
                    if (Lh.fine) s9 = false;
                    s9_minn = std::min(s9_minn, Lh.n);
                }
            }
        }
        h->s9_ok.push_back(s9 ? 1 : 0);
        h->s9_minn.push_back(s9_minn);
        h->jobs_s9.push_back(nullptr);
        h->maps_s9.push_back(nullptr);
        h->njob_s9.push_back(0);
        h->s9_strips.push_back(0);
        h->s9_grid.push_back(0);
        if constexpr (std::is_same<T, float>::value) {
            if (s9) {
                cudaError_t e = stream9_prepare();
                if (e != cudaSuccess)
                    return fail(MGMC_ERR_CUDA, std::string("band kernel set-up: ") + cudaGetErrorString(e));
                std::vector<StreamJob> sj;
                std::vector<Stream9Maps> sm;
                long long strips = 0;
                for (mgmc_ctx* c : chains) {
                    const int l = c->L - 1 - d;
                    if (l <= c->top) continue;
                    const auto& lv = levels_of<float>(c);
                    StreamJob J{};
                    J.L = lv[l];
                    J.C = lv[l - 1];
                    J.cs = c->cs;
                    J.strip0 = strips;
                    J.spb = (J.L.n + kStream9Rows - 1) / kStream9Rows;
                    J.nbands = (J.L.n + kStream9Band - 1) / kStream9Band;
                    strips += (long long)J.spb * J.nbands;
                    sj.push_back(J);
                    sm.emplace_back();
                    if (!make_stream9_maps(J.L, J.C, &sm.back()))
                        return fail(MGMC_ERR_CUDA, "TMA descriptor encoding failed");
                }
                h->jobs_s9.back() = upload(h, sj, st);
                h->maps_s9.back() = upload(h, sm, st);
                h->njob_s9.back() = (int)sj.size();
                h->s9_strips.back() = strips;
                h->s9_grid.back() = stream9_grid(strips);
            }
        }
        for (mgmc_ctx* c : chains) {
            const int l = c->L - 1 - d;
            if (l <= c->top) continue;
            const auto& lv = levels_of<T>(c);
            const DevLevel<T>& Lh = lv[l];
            const DevLevel<T>& Ch = lv[l - 1];
            const int TY = Lh.fine ? TileShape<T, true>::TY : TileShape<T, false>::TY;
            const int nty = (Lh.n + TY - 1) / TY;
            tj.push_back({Lh, Ch, c->P, tiles, Lh.ntx * nty});
            tiles += Lh.ntx * nty;
            mf.emplace_back();
            mb.emplace_back();
            if (!make_tile_maps<T>(Lh, Ch, false, &mf.back()) || !make_tile_maps<T>(Lh, Ch, true, &mb.back()))
                return fail(MGMC_ERR_CUDA, "TMA descriptor encoding failed");
            if (c->m > 0) {
                int rd = std::max(Lh.g_rows[0], Lh.h_rows);
                DevLevel<T> Lz = Lh;
                if ((d == 0 && h->stream_fine) || s9) Lz.zparts = nullptr;   // the low-rank kernel reads the state
                ld.push_back({Lz, Ch, c->P, bd, lowrank_blocks(rd)});
                bd += lowrank_blocks(rd);
                lu.push_back({Lz, Ch, c->P, bu, lowrank_blocks(Lh.g_rows[1])});
                bu += lowrank_blocks(Lh.g_rows[1]);
            }
        }
        // common block count of the jobs of one launch (0: they differ)
        auto common = [](const auto& v, auto count) {
            int per = v.empty() ? 0 : count(v[0]);
            for (const auto& j : v)
                if (count(j) != per) return 0;
            return per;
        };
        h->per_tile.push_back(common(tj, [](const TileJob<T>& j) { return j.ntiles; }));
        h->per_lrd.push_back(common(ld, [](const LowrankJob<T>& j) { return j.nblocks; }));
        h->per_lru.push_back(common(lu, [](const LowrankJob<T>& j) { return j.nblocks; }));
        h->jobs_tile.push_back(upload(h, tj, st));
        h->maps_fwd.push_back(upload(h, mf, st));
        h->maps_bwd.push_back(upload(h, mb, st));
        h->njob_tile.push_back((int)tj.size());
        h->nblk_tile.push_back(tiles);
        h->jobs_lrd.push_back(upload(h, ld, st));
        h->njob_lrd.push_back((int)ld.size());
        h->nblk_lrd.push_back(bd);
        h->jobs_lru.push_back(upload(h, lu, st));
        h->njob_lru.push_back((int)lu.size());
        h->nblk_lru.push_back(bu);
    }
    std::vector<CoarseJob<T>> cj;
    std::vector<QoiJob<T>> qj;
    std::vector<PackJob<T>> pj;
    std::vector<CycleState*> csl;
    size_t smem = 0;
    for (mgmc_ctx* c : chains) {
        cj.push_back({(const DevLevel<T>*)c->levels_dev, c->top, c->top == c->L - 1 ? 1 : 0, c->P_dev, c->chol, c->n0});
        const DevLevel<T>& Fh = levels_of<T>(c)[c->L - 1];
        qj.push_back({Fh.x, c->n_qoi, c->q_site, c->q_w, c->cs});
        pj.push_back({Fh.x, Fh.n, Fh.pitch, Fh.base});
        h->pack_max_n = std::max(h->pack_max_n, Fh.n);
        csl.push_back(c->cs);
        smem = std::max(smem, c->coarse_smem);
    }
    h->jobs_coarse = upload(h, cj, st);
    h->jobs_qoi = upload(h, qj, st);
    h->jobs_pack = upload(h, pj, st);
    h->cs_list = upload(h, csl, st);
    h->batch_coarse_smem = smem;
    if (st != MGMC_OK) return fail(st, "batch table upload failed");
    cudaError_t e = coarse_prepare_batch<T>(smem);
    if (e == cudaSuccess) e = tile_prepare_batch<T>();
    if (e != cudaSuccess) return fail(MGMC_ERR_CUDA, std::string("batch kernel set-up: ") + cudaGetErrorString(e));
    apply_band_min(h);
    (void)nc;
    return MGMC_OK;
}

}  // namespace

extern "C" {

mgmc_status mgmc_create_batch(int n_chains, const mgmc_config* cfgs, const mgmc_problem* problems,
                              const mgmc_allocator* alloc, void* stream, mgmc_handle* out)
{
    if (!out) return fail(MGMC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_chains < 1 || n_chains > 65536 || !cfgs || !problems) return fail(MGMC_ERR_ARG, "bad batch arguments");
    for (int c = 0; c < n_chains; ++c) {
        if (cfgs[c].dim != 2 || cfgs[c].nu1 != 1 || cfgs[c].nu2 != 1)
            return fail(MGMC_ERR_ARG, "batched chains must be 2D with nu1 = nu2 = 1");
        if (cfgs[c].precision != cfgs[0].precision) return fail(MGMC_ERR_ARG, "batched chains share one precision");
        if (cfgs[c].disc != cfgs[0].disc) return fail(MGMC_ERR_ARG, "batched chains share one discretisation");
    }
    mgmc_status dst = check_device();
    if (dst != MGMC_OK) return dst;
    mgmc_ctx* h = new mgmc_ctx();
    h->cfg = cfgs[0];
    cudaGetDevice(&h->device);
    h->buf.stream = (cudaStream_t)stream;
    if (alloc && alloc->alloc && alloc->free) {
        h->buf.alloc = *alloc;
        h->buf.use_cuda_malloc = false;
    }
    auto cleanup = [&](mgmc_status s) {
        for (mgmc_ctx* c : h->sub) mgmc_destroy(c);
        h->sub.clear();
        h->buf.release();
        delete h;
        return s;
    };
    for (int c = 0; c < n_chains; ++c) {
        mgmc_config cfg = cfgs[c];
        if (cfg.gibbs) return cleanup(fail(MGMC_ERR_ARG, "batches run the MGMC V-cycle only (gibbs = 0)"));
        if (cfg.gamma > 1 || cfg.disc == MGMC_SSL)
            return cleanup(fail(MGMC_ERR_ARG, "batches run the V-cycle of the 5/9-point grids only (gamma <= 1, "
                                              "disc != MGMC_SSL)"));
        if (cfg.coarse_max_n == 0) cfg.coarse_max_n = 31;
        const mgmc_problem& p = problems[c];
        mgmc_handle sh = nullptr;
        mgmc_status s = mgmc_create(&cfg, alloc, stream, p.kappa2, p.kappa2_const, p.m, p.obs_site, p.obs_w,
                                    p.nnz_per_obs, p.Gamma, p.y, p.n_qoi, p.qoi_site, p.qoi_w, &sh);
        if (s != MGMC_OK) {
            std::string msg = "chain " + std::to_string(c) + ": " + g_last_error;
            return cleanup(fail(s, msg));
        }
        h->sub.push_back(sh);
    }
    mgmc_status st = h->fp32() ? build_batch_tables<float>(h) : build_batch_tables<double>(h);
    if (st != MGMC_OK) return cleanup(st);
    if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return cleanup(fail(MGMC_ERR_CUDA, "stream creation failed"));
    if (cudaStreamSynchronize(h->buf.stream) != cudaSuccess) return cleanup(fail(MGMC_ERR_CUDA, "set-up failed"));
    *out = h;
    return MGMC_OK;
}

mgmc_status mgmc_sample_batch(mgmc_handle h, int64_t n_steps, uint64_t seed, uint64_t step_offset,
                              void* const* x_inout, double* qoi_out, void* stream)
{
    if (!h || !h->is_batch()) return fail(MGMC_ERR_ARG, "not a batch handle");
    if (n_steps < 0) return fail(MGMC_ERR_ARG, "bad arguments");
    if (n_steps == 0) return MGMC_OK;
    const int nc = (int)h->sub.size();
    const bool resume = x_inout == nullptr;
    // states: all in device memory, or all in host memory (staged through the device)
    int on_host = 0;
    if (!resume) {
        for (int c = 0; c < nc; ++c) {
            if (!x_inout[c]) return fail(MGMC_ERR_ARG, "NULL state pointer");
            on_host += is_device_ptr(x_inout[c]) ? 0 : 1;
        }
        if (on_host != 0 && on_host != nc) return fail(MGMC_ERR_ARG, "batch states must be all device or all host memory");
    }
    const bool xhost = on_host == nc && !resume;
    const bool qhost = qoi_out && !is_device_ptr(qoi_out);
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaSetDevice(h->device));
    mgmc_status st = ensure_graph(h);
    if (st != MGMC_OK) return st;
    const size_t esz = h->fp32() ? 4 : 8;
    std::vector<size_t> bytes((size_t)nc), off((size_t)nc + 1, 0);
    for (int c = 0; c < nc; ++c) {
        const long long n = h->sub[c]->cfg.n;
        bytes[c] = (size_t)(n * n) * esz;
        off[c + 1] = off[c] + bytes[c];
    }
    // host buffers: one stream-ordered staging allocation for the states and the QoI
    const size_t qbytes = qhost ? sizeof(double) * (size_t)nc * (size_t)n_steps : 0;
    char* stage = nullptr;
    if (xhost || qhost) CUDA_TRY(cudaMallocAsync((void**)&stage, (xhost ? off[nc] : 0) + qbytes, s));
    std::vector<void*> dev((size_t)nc, nullptr);
    for (int c = 0; c < nc && !resume; ++c) dev[c] = xhost ? (void*)(stage + off[c]) : x_inout[c];
    double* qdev = qhost ? (double*)(stage + (xhost ? off[nc] : 0)) : qoi_out;
    auto pack = [&](bool in) {
        if (h->fp32())
            launch_pack_batch<float>((const PackJob<float>*)h->jobs_pack, dev.data(), nc, h->pack_max_n, in, s);
        else
            launch_pack_batch<double>((const PackJob<double>*)h->jobs_pack, dev.data(), nc, h->pack_max_n, in, s);
    };
    if (xhost)
        for (int c = 0; c < nc; ++c)
            CUDA_TRY(cudaMemcpyAsync(dev[c], x_inout[c], bytes[c], cudaMemcpyHostToDevice, s));
    if (!resume) pack(true);
    launch_set_cycle_batch(h->cs_list, nc, seed, step_offset, 1, qdev, n_steps, s);
    for (int64_t t = 0; t < n_steps; ++t) CUDA_TRY(cudaGraphLaunch(h->exec, s));
    if (!resume) pack(false);
    if (xhost)
        for (int c = 0; c < nc; ++c)
            CUDA_TRY(cudaMemcpyAsync(x_inout[c], dev[c], bytes[c], cudaMemcpyDeviceToHost, s));
    if (qhost) CUDA_TRY(cudaMemcpyAsync(qoi_out, qdev, qbytes, cudaMemcpyDeviceToHost, s));
    if (stage) CUDA_TRY(cudaFreeAsync(stage, s));
    CUDA_TRY(cudaGetLastError());
    if (xhost || qhost) return take_status(h, s);
    return MGMC_OK;
}

mgmc_status mgmc_get_state(mgmc_handle h, int chain, void* x_out, void* stream)
{
    if (!h || !x_out) return fail(MGMC_ERR_ARG, "handle or x_out is NULL");
    const int nc = h->is_batch() ? (int)h->sub.size() : 1;
    if (chain < 0 || chain >= nc) return fail(MGMC_ERR_ARG, "chain index out of range");
    mgmc_ctx* c = h->is_batch() ? h->sub[chain] : h;
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaSetDevice(h->device));
    long long N = 1;
    for (int a = 0; a < c->cfg.dim; ++a) N *= c->cfg.n;
    const bool host = !is_device_ptr(x_out);
    mgmc_status st = pack_out(c, x_out, host, s, N);
    if (st != MGMC_OK) return st;
    CUDA_TRY(cudaGetLastError());
    if (host) CUDA_TRY(cudaStreamSynchronize(s));
    return MGMC_OK;
}

mgmc_status mgmc_destroy(mgmc_handle h)
{
    if (!h) return MGMC_OK;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    for (mgmc_ctx* c : h->sub) mgmc_destroy(c);
    h->sub.clear();
    for (int i = 0; i < 4; ++i)
        if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->buf.release();
    delete h;
    return MGMC_OK;
}

}  // extern "C"
