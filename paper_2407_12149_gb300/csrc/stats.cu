// stats.cu -- on-device chain statistics of a QoI series (Sec. 5.3.2):
// mean, lagged autocovariance Gamma(t) = 1/(n-t) sum_i (a_i - abar)(a_{i+t} - abar)
// and the integrated autocorrelation time with Wolff's automatic window
// (U. Wolff, Comput. Phys. Commun. 156 (2004) 143, Sec. 3.3): for W = 1, 2, ...
//   tau_W = 1/2 + sum_{t<=W} rho(t),  tau~ = S / ln((2 tau_W + 1)/(2 tau_W - 1)),
//   stop at the first W with exp(-W/tau~) - tau~/sqrt(W n) < 0;
// reported in the paper's convention tau = 2 tau_W, error 2 * 2 tau_W sqrt((W + 1/2 - tau_W)/n).
// Lags are evaluated in chunks of kLagChunk until the window is found.
#include <cmath>
#include <mutex>
#include <string>

#include "common.cuh"

namespace {

constexpr int kLagChunk = 1024;
constexpr int kThreads = 256;

struct WolffState {
    double mean;
    double G0;
    double tint;
    long long next;    // next lag to examine
    long long W;
    int done;
};

__device__ double block_sum(double v)
{
    __shared__ double part[kThreads];
    part[threadIdx.x] = v;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
        __syncthreads();
    }
    double r = part[0];
    __syncthreads();
    return r;
}

__global__ void k_stats_init(const double* __restrict__ a, long long n, WolffState* st)
{
    double acc = 0.0;
    for (long long i = threadIdx.x; i < n; i += kThreads) acc += a[i];
    double mean = block_sum(acc) / (double)n;
    acc = 0.0;
    for (long long i = threadIdx.x; i < n; i += kThreads) {
        double d = a[i] - mean;
        acc += d * d;
    }
    double G0 = block_sum(acc) / (double)n;
    if (threadIdx.x == 0) {
        st->mean = mean;
        st->G0 = G0;
        st->tint = 0.5;
        st->next = 1;
        st->W = 0;
        st->done = G0 > 0.0 ? 0 : 1;
    }
}

// Gamma(t) for t = t0 + blockIdx.x (one block per lag)
__global__ void k_autocov(const double* __restrict__ a, long long n, const WolffState* st, long long t0,
                          long long t1, double* __restrict__ G)
{
    long long t = t0 + blockIdx.x;
    if (t >= t1) return;
    double mean = st->mean;
    double acc = 0.0;
    for (long long i = threadIdx.x; i + t < n; i += kThreads) acc += (a[i] - mean) * (a[i + t] - mean);
    double s = block_sum(acc);
    if (threadIdx.x == 0) G[blockIdx.x] = s / (double)(n - t);
}

__global__ void k_wolff_scan(const double* __restrict__ G, long long t0, long long t1, long long tmax, long long n,
                             double S, WolffState* st)
{
    if (threadIdx.x != 0 || blockIdx.x != 0 || st->done) return;
    double tint = st->tint;
    for (long long w = t0; w < t1; ++w) {
        tint += G[w - t0] / st->G0;
        double tt = tint <= 0.5 ? 1e-6 : S / log((2.0 * tint + 1.0) / (2.0 * tint - 1.0));
        double g = exp(-(double)w / tt) - tt / sqrt((double)w * (double)n);
        if (g < 0.0 || w == tmax) {
            st->W = w;
            st->tint = tint;
            st->done = 1;
            return;
        }
    }
    st->tint = tint;
    st->next = t1;
}

__global__ void k_stats_final(const WolffState* st, long long n, mgmc_stats* out)
{
    mgmc_stats r;
    r.mean = st->mean;
    r.var = st->G0;
    r.n_used = n;
    if (!(st->G0 > 0.0)) {
        r.tau_int = 1.0;
        r.tau_err = 0.0;
        r.window = 0;
    } else {
        double tint = st->tint;
        double W = (double)st->W;
        r.tau_int = 2.0 * tint;
        r.tau_err = 2.0 * (2.0 * tint * sqrt((W + 0.5 - tint) / (double)n));
        r.window = st->W;
    }
    r.ess = (double)n / r.tau_int;
    *out = r;
}

}  // namespace

extern "C" mgmc_status mgmc_qoi_stats(const double* qoi, int64_t n, int64_t burn_in, double S, mgmc_stats* out,
                                      void* stream)
{
    if (!qoi || !out || burn_in < 0 || n - burn_in < 2) {
        mgmc::set_last_error("mgmc_qoi_stats: NULL pointer or fewer than 2 samples after burn-in");
        return MGMC_ERR_ARG;
    }
    if (!(S > 0.0)) S = 1.5;
    cudaStream_t s = (cudaStream_t)stream;
    const double* a = qoi + burn_in;
    long long nn = n - burn_in;
    long long tmax = nn / 2;
    WolffState* st = nullptr;
    double* G = nullptr;
    mgmc_stats* dout = nullptr;
    mgmc_status rc = MGMC_OK;
    const char* msg = nullptr;
    // every exit below frees what was allocated (stream-ordered)
    if (cudaMallocAsync((void**)&st, sizeof(WolffState), s) != cudaSuccess ||
        cudaMallocAsync((void**)&G, sizeof(double) * kLagChunk, s) != cudaSuccess ||
        cudaMallocAsync((void**)&dout, sizeof(mgmc_stats), s) != cudaSuccess) {
        rc = MGMC_ERR_CUDA;
        msg = "mgmc_qoi_stats: stream-ordered allocation failed";
    }
    if (rc == MGMC_OK) {
        k_stats_init<<<1, kThreads, 0, s>>>(a, nn, st);
        long long t0 = 1;
        while (t0 <= tmax) {
            long long t1 = t0 + kLagChunk < tmax + 1 ? t0 + kLagChunk : tmax + 1;
            k_autocov<<<(unsigned)(t1 - t0), kThreads, 0, s>>>(a, nn, st, t0, t1, G);
            k_wolff_scan<<<1, 1, 0, s>>>(G, t0, t1, tmax, nn, S, st);
            WolffState hs;
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                rc = MGMC_ERR_CUDA;
                msg = "mgmc_qoi_stats: kernel launch or copy failed";
                break;
            }
            if (hs.done) break;
            t0 = t1;
        }
    }
    if (rc == MGMC_OK) {
        k_stats_final<<<1, 1, 0, s>>>(st, nn, dout);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(out, dout, sizeof(mgmc_stats), cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            rc = MGMC_ERR_CUDA;
            msg = "mgmc_qoi_stats: kernel launch or copy failed";
        }
    }
    if (st) cudaFreeAsync(st, s);
    if (G) cudaFreeAsync(G, s);
    if (dout) cudaFreeAsync(dout, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == MGMC_OK) {
        rc = MGMC_ERR_CUDA;
        msg = "mgmc_qoi_stats: stream synchronisation failed";
    }
    if (msg) mgmc::set_last_error(msg);
    return rc;
}

// ---------------------------------------------------------------------------
// Allocation-free variant: the scratch (Wolff state, all lags, result) lives
// in one file-scope device array.  In host code the symbol names only a
// host-side stand-in, so its device address is looked up per device with
// cudaGetSymbolAddress and passed to the kernels.
// ---------------------------------------------------------------------------
namespace {

constexpr long long kNoallocMaxLags = MGMC_NOALLOC_MAX_SERIES / 2;
constexpr size_t kNoallocBytes = 256 + sizeof(double) * (kNoallocMaxLags + 1) + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// device address of the scratch on the current device (looked up once per device)
cudaError_t noalloc_scratch(void** ptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *ptr = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" mgmc_status mgmc_qoi_stats_noalloc(const double* qoi, int64_t n, int64_t burn_in, double S,
                                               mgmc_stats* out, void* stream)
{
    if (!qoi || !out || burn_in < 0 || n - burn_in < 2) {
        mgmc::set_last_error("mgmc_qoi_stats_noalloc: need qoi, out and n - burn_in >= 2");
        return MGMC_ERR_ARG;
    }
    if (n - burn_in > MGMC_NOALLOC_MAX_SERIES) {
        mgmc::set_last_error("mgmc_qoi_stats_noalloc: n - burn_in exceeds MGMC_NOALLOC_MAX_SERIES (65536); "
                             "use mgmc_qoi_stats for longer series");
        return MGMC_ERR_ARG;
    }
    if (!(S > 0.0)) S = 1.5;
    cudaStream_t s = (cudaStream_t)stream;
    void* base = nullptr;
    if (noalloc_scratch(&base) != cudaSuccess) {
        mgmc::set_last_error("mgmc_qoi_stats_noalloc: cudaGetSymbolAddress of the scratch array failed");
        return MGMC_ERR_CUDA;
    }
    WolffState* st = (WolffState*)base;
    double* G = (double*)((unsigned char*)base + 256);
    mgmc_stats* dout = (mgmc_stats*)((unsigned char*)base + 256 + sizeof(double) * (kNoallocMaxLags + 1));
    const double* a = qoi + burn_in;
    long long nn = n - burn_in;
    long long tmax = nn / 2;
    // every scratch word read below is written first in the same call
    k_stats_init<<<1, kThreads, 0, s>>>(a, nn, st);
    if (tmax >= 1) {
        k_autocov<<<(unsigned)tmax, kThreads, 0, s>>>(a, nn, st, 1, tmax + 1, G);
        k_wolff_scan<<<1, 1, 0, s>>>(G, 1, tmax + 1, tmax, nn, S, st);
    }
    k_stats_final<<<1, 1, 0, s>>>(st, nn, dout);
    if (cudaGetLastError() != cudaSuccess) return MGMC_ERR_CUDA;
    if (cudaMemcpyAsync(out, dout, sizeof(mgmc_stats), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MGMC_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MGMC_ERR_CUDA;
    return MGMC_OK;
}
