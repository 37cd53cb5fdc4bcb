// unet.cu -- learned warm start for the sampler: a U-Net maps (log kappa^2, the
// observation weights B^T 1, the weighted data B^T y) on the (n+1)^2 grid to an
// estimate of the posterior mean mu = A~^-1 f (Sec. 2.2), used only as a
// chain's initial state x_0: the MGMC chain's law does not depend on x_0, the
// estimate only shortens burn-in.
//
// Network (channels-last [batch][H][W][C], BF16 activations and weights, FP32
// accumulation; c_s = c0 2^s): encoder levels 0..2 of two 3x3 conv + ReLU and a
// 2x2 average pool, two 3x3 conv + ReLU at level 3, decoder levels 2..0 of a
// nearest 2x upsampling, a concatenation [upsampled, skip] and two 3x3 conv +
// ReLU, a 1x1 output convolution.  Loss: mean squared error on the n x n
// interior; optimiser: Adam (Kingma & Ba 2015).
//
// Every 3x3 convolution is an im2col + tcgen05 GEMM (tc_gemm.cu):
//   forward      Y[P][co]      = relu(Xcol[P][9ci] W[co][9ci]^T + b)
//   data grad    dXcol[P][9ci] = dZ[P][co] Wt[9ci][co]^T, then col2im
//   weight grad  dWt[9ci][co]  = XcolT[9ci][P] dZT[co][P]^T (split over P, fixed-order sum)
// All reductions (bias gradients, loss) run in a fixed order: results are
// deterministic.  This file also holds the exported GEMM entry point.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mgmc.h"
#include "common.cuh"
#include "tc_gemm.cuh"

namespace mgmc {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kLayers = 14;
constexpr int kRedBlocks = 256;   // partial-sum blocks of the column reductions

struct LayerDef {
    int level, cin, cout;
};

void layer_table(int c0, LayerDef* L)
{
    const int c[4] = {c0, 2 * c0, 4 * c0, 8 * c0};
    const LayerDef t[kLayers] = {{0, 3, c[0]},           {0, c[0], c[0]},        {1, c[0], c[1]}, {1, c[1], c[1]},
                                 {2, c[1], c[2]},        {2, c[2], c[2]},        {3, c[2], c[3]}, {3, c[3], c[3]},
                                 {2, c[3] + c[2], c[2]}, {2, c[2], c[2]},        {1, c[2] + c[1], c[1]},
                                 {1, c[1], c[1]},        {0, c[1] + c[0], c[0]}, {0, c[0], c[0]}};
    for (int l = 0; l < kLayers; ++l) L[l] = t[l];
}

int round8(int v) { return (v + 7) / 8 * 8; }

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }

// out[p][(ky 3 + kx) cin + c] = x[b][i + ky - 1][j + kx - 1][c] (zero outside); columns
// [9 cin, ldo) are zero
__global__ void k_im2col(const bf16* __restrict__ x, int B, int H, int cin, bf16* __restrict__ out, int ldo)
{
    const long long P = (long long)B * H * H;
    const bf16 z = __float2bfloat16(0.f);
    for (long long it = gtid(); it < P * 9; it += gstride()) {
        const long long p = it / 9;
        const int tap = (int)(it % 9), ky = tap / 3, kx = tap % 3;
        const int j = (int)(p % H), i = (int)((p / H) % H);
        const long long b = p / ((long long)H * H);
        const int si = i + ky - 1, sj = j + kx - 1;
        bf16* o = out + p * ldo + tap * cin;
        if (si < 0 || si >= H || sj < 0 || sj >= H) {
            for (int c = 0; c < cin; ++c) o[c] = z;
        } else {
            const bf16* s = x + ((b * H + si) * H + sj) * cin;
            if ((cin & 7) == 0) {
                for (int c = 0; c < cin; c += 8)
                    *reinterpret_cast<uint4*>(o + c) = *reinterpret_cast<const uint4*>(s + c);
            } else {
                for (int c = 0; c < cin; ++c) o[c] = s[c];
            }
        }
        if (tap == 8)
            for (int c = 9 * cin; c < ldo; ++c) out[p * ldo + c] = z;
    }
}

// out[c][r] = in[r][c] for r < R, c < C (32 x 32 tiles through shared memory)
__global__ void k_transpose(const bf16* __restrict__ in, long long R, int C, long long ldi, bf16* __restrict__ out,
                            long long ldo)
{
    __shared__ bf16 t[32][33];
    const long long r0 = (long long)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const long long r = r0 + k;
        const int c = c0 + threadIdx.x;
        t[k][threadIdx.x] = (r < R && c < C) ? in[r * ldi + c] : __float2bfloat16(0.f);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k;
        const long long r = r0 + threadIdx.x;
        if (c < C && r < R) out[(long long)c * ldo + r] = t[threadIdx.x][k];
    }
}

// dz = bf16(dy * (y > 0)); part[block][c] = sum of dz over the block's rows (C divides 256)
__global__ void k_relu_bwd(const float* __restrict__ dy, const bf16* __restrict__ y, long long P, int C,
                           bf16* __restrict__ dz, float* __restrict__ part)
{
    __shared__ float red[256];
    const int c = threadIdx.x % C, r0 = threadIdx.x / C, rs = blockDim.x / C;
    const long long rows = (P + gridDim.x - 1) / gridDim.x;
    const long long rb = blockIdx.x * rows, re = min(P, rb + rows);
    float acc = 0.f;
    for (long long r = rb + r0; r < re; r += rs) {
        const long long e = r * C + c;
        const bf16 v = __float2bfloat16(__bfloat162float(y[e]) > 0.f ? dy[e] : 0.f);
        dz[e] = v;
        acc += __bfloat162float(v);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < C) {
        float s = 0.f;
        for (int k = 0; k < rs; ++k) s += red[k * C + threadIdx.x];
        part[(long long)blockIdx.x * C + threadIdx.x] = s;
    }
}

// out[c] = sum over nb blocks of part[b][c] (fixed order)
__global__ void k_colsum(const float* __restrict__ part, int nb, int C, float* __restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += part[(long long)b * C + c];
    out[c] = s;
}

// dx[p][c] (+)= sum over taps of dcol[p'][tap cin + c], p' = (i - ky + 1, j - kx + 1)
__global__ void k_col2im(const float* __restrict__ dcol, int ldc, int B, int H, int cin, float* __restrict__ dx,
                         int accumulate)
{
    const long long P = (long long)B * H * H;
    for (long long it = gtid(); it < P * cin; it += gstride()) {
        const long long p = it / cin;
        const int c = (int)(it % cin);
        const int j = (int)(p % H), i = (int)((p / H) % H);
        const long long b = p / ((long long)H * H);
        float s = 0.f;
        for (int ky = 0; ky < 3; ++ky)
            for (int kx = 0; kx < 3; ++kx) {
                const int oi = i - ky + 1, oj = j - kx + 1;
                if (oi < 0 || oi >= H || oj < 0 || oj >= H) continue;
                s += dcol[((b * H + oi) * H + oj) * ldc + (ky * 3 + kx) * cin + c];
            }
        dx[it] = accumulate ? dx[it] + s : s;
    }
}

// 2x2 average pool of x [B][2H][2H][C] into y [B][H][H][C]
__global__ void k_pool_fwd(const bf16* __restrict__ x, int B, int H, int C, bf16* __restrict__ y)
{
    const long long n = (long long)B * H * H * C;
    const int W2 = 2 * H;
    for (long long it = gtid(); it < n; it += gstride()) {
        const int c = (int)(it % C);
        const long long q = it / C;
        const int j = (int)(q % H), i = (int)((q / H) % H);
        const long long b = q / ((long long)H * H);
        auto at = [&](int a, int bb) { return __bfloat162float(x[((b * W2 + 2 * i + a) * W2 + 2 * j + bb) * C + c]); };
        y[it] = __float2bfloat16(0.25f * (at(0, 0) + at(1, 0) + at(0, 1) + at(1, 1)));
    }
}

// dx [B][2H][2H][C] (+)= dy [B][H][H][C] / 4
__global__ void k_pool_bwd(const float* __restrict__ dy, int B, int H, int C, float* __restrict__ dx, int accumulate)
{
    const int W2 = 2 * H;
    const long long n = (long long)B * W2 * W2 * C;
    for (long long it = gtid(); it < n; it += gstride()) {
        const int c = (int)(it % C);
        const long long q = it / C;
        const int j = (int)(q % W2), i = (int)((q / W2) % W2);
        const long long b = q / ((long long)W2 * W2);
        const float v = 0.25f * dy[((b * H + i / 2) * H + j / 2) * C + c];
        dx[it] = accumulate ? dx[it] + v : v;
    }
}

// u [B][H][H][ca + cb] = [nearest 2x upsampling of low [B][H/2][H/2][ca], skip [B][H][H][cb]]
__global__ void k_upcat(const bf16* __restrict__ low, int ca, const bf16* __restrict__ skip, int cb, int B, int H,
                        bf16* __restrict__ u)
{
    const int C = ca + cb, h = H / 2;
    const long long n = (long long)B * H * H * C;
    for (long long it = gtid(); it < n; it += gstride()) {
        const int c = (int)(it % C);
        const long long p = it / C;
        const int j = (int)(p % H), i = (int)((p / H) % H);
        const long long b = p / ((long long)H * H);
        u[it] = c < ca ? low[((b * h + i / 2) * h + j / 2) * ca + c] : skip[p * cb + (c - ca)];
    }
}

// backward of k_upcat: dlow (set) = sum of the 4 children's first ca channels, dskip (set) = the rest
__global__ void k_upcat_bwd(const float* __restrict__ du, int ca, int cb, int B, int H, float* __restrict__ dlow,
                            float* __restrict__ dskip)
{
    const int C = ca + cb, h = H / 2;
    const long long nl = (long long)B * h * h * ca, ns = (long long)B * H * H * cb;
    for (long long it = gtid(); it < nl + ns; it += gstride()) {
        if (it < nl) {
            const int c = (int)(it % ca);
            const long long q = it / ca;
            const int j = (int)(q % h), i = (int)((q / h) % h);
            const long long b = q / ((long long)h * h);
            auto at = [&](int a, int bb) { return du[((b * H + 2 * i + a) * H + 2 * j + bb) * C + c]; };
            dlow[it] = at(0, 0) + at(1, 0) + at(0, 1) + at(1, 1);
        } else {
            const long long e = it - nl;
            const int c = (int)(e % cb);
            const long long p = e / cb;
            dskip[e] = du[p * C + ca + c];
        }
    }
}

// out[p] = sum_c w[c] x[p][c] + b
__global__ void k_out_fwd(const bf16* __restrict__ x, long long P, int C, const float* __restrict__ w,
                          const float* __restrict__ b, float* __restrict__ out)
{
    for (long long p = gtid(); p < P; p += gstride()) {
        float s = 0.f;
        for (int c = 0; c < C; ++c) s += w[c] * __bfloat162float(x[p * C + c]);
        out[p] = s + b[0];
    }
}

// dout = scale (out - t) on the n x n interior (0 on the padding); part[block] = sum (out - t)^2
__global__ void k_loss(const float* __restrict__ out, const float* __restrict__ t, int B, int H, int n, float scale,
                       float* __restrict__ dout, float* __restrict__ part)
{
    __shared__ float red[256];
    const long long P = (long long)B * H * H;
    float acc = 0.f;
    for (long long p = gtid(); p < P; p += gstride()) {
        const int j = (int)(p % H), i = (int)((p / H) % H);
        const long long b = p / ((long long)H * H);
        float d = 0.f;
        if (i < n && j < n) {
            const float e = out[p] - t[(b * n + i) * n + j];
            acc += e * e;
            d = scale * e;
        }
        dout[p] = d;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// output layer backward: dx[p][c] = dout[p] w[c]; part[block][c] = sum_p dout[p] x[p][c] over
// the block's rows, part[block][C] = sum_p dout[p]
__global__ void k_out_bwd(const float* __restrict__ dout, const bf16* __restrict__ x, long long P, int C,
                          const float* __restrict__ w, float* __restrict__ dx, float* __restrict__ part)
{
    const long long rows = (P + gridDim.x - 1) / gridDim.x;
    const long long rb = blockIdx.x * rows, re = min(P, rb + rows);
    for (long long e = rb * C + threadIdx.x; e < re * C; e += blockDim.x) dx[e] = dout[e / C] * w[e % C];
    for (int c = threadIdx.x; c <= C; c += blockDim.x) {
        float s = 0.f;
        for (long long r = rb; r < re; ++r) s += c < C ? dout[r] * __bfloat162float(x[r * C + c]) : dout[r];
        part[(long long)blockIdx.x * (C + 1) + c] = s;
    }
}

// g[co K + k] = dwt[k][co]  (weight gradient in the [cout][3][3][cin] order)
__global__ void k_wt_to_flat(const float* __restrict__ dwt, int K, int Co, float* __restrict__ g)
{
    const long long n = (long long)K * Co;
    for (long long it = gtid(); it < n; it += gstride()) {
        const int k = (int)(it % K), co = (int)(it / K);
        g[it] = dwt[(long long)k * Co + co];
    }
}

__global__ void k_adam(float* __restrict__ th, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, long long n, float lr, float b1, float b2, float eps, float c1,
                       float c2)
{
    for (long long i = gtid(); i < n; i += gstride()) {
        const float mi = b1 * m[i] + (1.f - b1) * g[i];
        const float vi = b2 * v[i] + (1.f - b2) * g[i] * g[i];
        m[i] = mi;
        v[i] = vi;
        th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// BF16 copies of W [Co][K]: Wb [Co][Kp] (zero columns K..Kp) and Wt [Kp][Co] (zero rows K..Kp)
__global__ void k_w_to_bf16(const float* __restrict__ W, int Co, int K, int Kp, bf16* __restrict__ Wb,
                            bf16* __restrict__ Wt)
{
    const long long n = (long long)Co * Kp;
    for (long long it = gtid(); it < n; it += gstride()) {
        const int k = (int)(it % Kp), co = (int)(it / Kp);
        const bf16 v = __float2bfloat16(k < K ? W[(long long)co * K + k] : 0.f);
        Wb[it] = v;
        Wt[(long long)k * Co + co] = v;
    }
}

__global__ void k_round_bf16(const float* __restrict__ a, int n, float* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __bfloat162float(__float2bfloat16(a[i]));
}

// copy samples idx[0..B) of the data set into the batch buffers
__global__ void k_gather(const bf16* __restrict__ in, const float* __restrict__ tgt, const long long* __restrict__ idx,
                         int B, long long in_sz, long long tgt_sz, bf16* __restrict__ inb, float* __restrict__ tgtb)
{
    const long long n = (long long)B * (in_sz + tgt_sz);
    for (long long it = gtid(); it < n; it += gstride()) {
        const long long b = it / (in_sz + tgt_sz), r = it % (in_sz + tgt_sz);
        if (r < in_sz)
            inb[b * in_sz + r] = in[idx[b] * in_sz + r];
        else
            tgtb[b * tgt_sz + (r - in_sz)] = tgt[idx[b] * tgt_sz + (r - in_sz)];
    }
}

// x[b][i n + j] = out[b][i][j] on the n x n interior (grid row i, column j), FP32 or FP64
__global__ void k_crop(const float* __restrict__ out, int B, int H, int n, void* __restrict__ x, int fp64)
{
    const long long N = (long long)B * n * n;
    for (long long it = gtid(); it < N; it += gstride()) {
        const int j = (int)(it % n), i = (int)((it / n) % n);
        const long long b = it / ((long long)n * n);
        const float v = out[(b * H + i) * H + j];
        if (fp64)
            reinterpret_cast<double*>(x)[it] = v;
        else
            reinterpret_cast<float*>(x)[it] = v;
    }
}

unsigned grid_for(long long n, int threads = 256)
{
    long long b = (n + threads - 1) / threads;
    return (unsigned)std::max(1LL, std::min(b, 152LL * 16));
}

// splitmix64 (Steele, Lea, Flood 2014) and Box-Muller, for the seeded initialisation and shuffles
struct SplitMix {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return ((double)(next() >> 11) + 0.5) * 0x1p-53; }
    double normal()
    {
        const double r = std::sqrt(-2.0 * std::log(uniform()));
        return r * std::cos(6.283185307179586 * uniform());
    }
};

}  // namespace

struct UnetCtx {
    int n = 0, H = 0, c0 = 0, bmax = 0, device = 0;
    LayerDef L[kLayers];
    int K[kLayers], Kp[kLayers];
    long long woff[kLayers], boff[kLayers], out_w = 0, out_b = 0, nparam = 0;
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *wout_r = nullptr;
    bf16 *Wb[kLayers] = {}, *Wt[kLayers] = {};
    long long step = 0;
    // activations and gradients (capacity bmax samples)
    bf16* in = nullptr;
    bf16* act[kLayers] = {};
    bf16 *p0 = nullptr, *p1 = nullptr, *p2 = nullptr, *u2 = nullptr, *u1 = nullptr, *u0 = nullptr;
    float *out = nullptr, *dout = nullptr, *tgt = nullptr;
    bf16 *col = nullptr, *colT = nullptr, *dz = nullptr, *dzT = nullptr;
    float *dcol = nullptr, *dwt = nullptr, *wpart = nullptr, *part = nullptr;
    float* dact[kLayers] = {};
    float *du = nullptr, *dp = nullptr;
    long long* idx = nullptr;
    int* status = nullptr;
    size_t wpart_elems = 0;
    mgmc_allocator alloc{};
    bool use_alloc = false;
    cudaStream_t stream = nullptr;
    std::vector<void*> blocks;

    int Hs(int s) const { return H >> s; }
    long long Ps(int s, int B) const { return (long long)B * Hs(s) * Hs(s); }
    const bf16* layer_in(int l) const
    {
        switch (l) {
            case 0: return in;
            case 2: return p0;
            case 4: return p1;
            case 6: return p2;
            case 8: return u2;
            case 10: return u1;
            case 12: return u0;
            default: return act[l - 1];
        }
    }
    void* get(size_t bytes)
    {
        void* p = nullptr;
        bytes = (bytes + 255) / 256 * 256;
        if (use_alloc)
            p = alloc.alloc(bytes, stream, alloc.ctx);
        else if (cudaMalloc(&p, bytes) != cudaSuccess)
            p = nullptr;
        if (p) blocks.push_back(p);
        return p;
    }
    void release()
    {
        for (void* p : blocks) {
            if (use_alloc)
                alloc.free(p, stream, alloc.ctx);
            else
                cudaFree(p);
        }
        blocks.clear();
    }
};

namespace {

mgmc_status unet_fail(mgmc_status s, const std::string& msg)
{
    set_last_error(msg.c_str());
    return s;
}

#define UNET_CUDA(call)                                                                                           \
    do {                                                                                                          \
        cudaError_t e_ = (call);                                                                                  \
        if (e_ != cudaSuccess) return unet_fail(MGMC_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

mgmc_status gemm(UnetCtx* u, const void* A, int lda, const void* B, int ldb, void* C, long long M, int N, long long K,
                 int epi, const float* bias, int splits)
{
    TcGemm g;
    if (!tc_gemm_plan(&g, A, lda, B, ldb, (int)M, N, (int)K, splits))
        return unet_fail(MGMC_ERR_CUDA, "tensor-core GEMM: descriptor encoding failed");
    if (g.splits > 1 && (size_t)g.splits * M * N > u->wpart_elems)
        return unet_fail(MGMC_ERR_STATE, "split-K scratch too small");
    void* out = g.splits > 1 ? (void*)u->wpart : C;
    UNET_CUDA(tc_gemm_run(g, out, epi, bias, u->status, u->stream));
    if (g.splits > 1) UNET_CUDA(tc_reduce_splits(u->wpart, g.splits, M * N, (float*)C, u->stream));
    return MGMC_OK;
}

mgmc_status refresh_bf16(UnetCtx* u)
{
    for (int l = 0; l < kLayers; ++l)
        k_w_to_bf16<<<grid_for((long long)u->L[l].cout * u->Kp[l]), 256, 0, u->stream>>>(
            u->theta + u->woff[l], u->L[l].cout, u->K[l], u->Kp[l], u->Wb[l], u->Wt[l]);
    k_round_bf16<<<(u->c0 + 255) / 256, 256, 0, u->stream>>>(u->theta + u->out_w, u->c0, u->wout_r);
    UNET_CUDA(cudaGetLastError());
    return MGMC_OK;
}

// forward pass of B samples whose inputs are at `input` ([B][H][H][3] BF16)
mgmc_status forward(UnetCtx* u, int B, const bf16* input)
{
    cudaStream_t st = u->stream;
    bf16* saved_in = u->in;
    u->in = const_cast<bf16*>(input);
    mgmc_status rc = MGMC_OK;
    for (int l = 0; l < kLayers && rc == MGMC_OK; ++l) {
        const LayerDef& D = u->L[l];
        const int s = D.level, Hs = u->Hs(s);
        const long long P = u->Ps(s, B);
        if (l == 2) k_pool_fwd<<<grid_for(P * u->L[1].cout), 256, 0, st>>>(u->act[1], B, Hs, u->L[1].cout, u->p0);
        if (l == 4) k_pool_fwd<<<grid_for(P * u->L[3].cout), 256, 0, st>>>(u->act[3], B, Hs, u->L[3].cout, u->p1);
        if (l == 6) k_pool_fwd<<<grid_for(P * u->L[5].cout), 256, 0, st>>>(u->act[5], B, Hs, u->L[5].cout, u->p2);
        if (l == 8)
            k_upcat<<<grid_for(P * D.cin), 256, 0, st>>>(u->act[7], u->L[7].cout, u->act[5], u->L[5].cout, B, Hs,
                                                       u->u2);
        if (l == 10)
            k_upcat<<<grid_for(P * D.cin), 256, 0, st>>>(u->act[9], u->L[9].cout, u->act[3], u->L[3].cout, B, Hs,
                                                       u->u1);
        if (l == 12)
            k_upcat<<<grid_for(P * D.cin), 256, 0, st>>>(u->act[11], u->L[11].cout, u->act[1], u->L[1].cout, B, Hs,
                                                       u->u0);
        k_im2col<<<grid_for(P * 9), 256, 0, st>>>(u->layer_in(l), B, Hs, D.cin, u->col, u->Kp[l]);
        rc = gemm(u, u->col, u->Kp[l], u->Wb[l], u->Kp[l], u->act[l], P, D.cout, u->K[l],
                  kEpiBias | kEpiRelu | kEpiBF16, u->theta + u->boff[l], 1);
    }
    if (rc == MGMC_OK) {
        const long long P0 = u->Ps(0, B);
        k_out_fwd<<<grid_for(P0), 256, 0, st>>>(u->act[13], P0, u->c0, u->wout_r, u->theta + u->out_b, u->out);
        if (cudaGetLastError() != cudaSuccess) rc = unet_fail(MGMC_ERR_CUDA, "U-Net forward launch failed");
    }
    u->in = saved_in;
    return rc;
}

// backward of layer l given dact[l]; dx (FP32 [P][cin]) receives the input gradient (NULL: skip)
mgmc_status conv_backward(UnetCtx* u, int l, int B, const bf16* input, float* dx)
{
    cudaStream_t st = u->stream;
    const LayerDef& D = u->L[l];
    const int s = D.level, Hs = u->Hs(s);
    const long long P = u->Ps(s, B);
    k_relu_bwd<<<kRedBlocks, 256, 0, st>>>(u->dact[l], u->act[l], P, D.cout, u->dz, u->part);
    k_colsum<<<(D.cout + 255) / 256, 256, 0, st>>>(u->part, kRedBlocks, D.cout, u->grad + u->boff[l]);
    const dim3 tb(32, 8);
    k_transpose<<<dim3((unsigned)((P + 31) / 32), (unsigned)((D.cout + 31) / 32)), tb, 0, st>>>(u->dz, P, D.cout,
                                                                                               D.cout, u->dzT, P);
    const bf16* x = l == 0 ? input : u->layer_in(l);
    k_im2col<<<grid_for(P * 9), 256, 0, st>>>(x, B, Hs, D.cin, u->col, u->Kp[l]);
    k_transpose<<<dim3((unsigned)((P + 31) / 32), (unsigned)((u->Kp[l] + 31) / 32)), tb, 0, st>>>(
        u->col, P, u->Kp[l], u->Kp[l], u->colT, P);
    // weight gradient dWt[Kp][co] = colT[Kp][P] dzT[co][P]^T, split over P for ~2 CTAs per SM
    const long long tiles = (u->Kp[l] + 127) / 128;  // N = cout <= 256 is one tile
    const int splits = (int)std::max(1LL, std::min(304LL / tiles, (P + 2047) / 2048));
    mgmc_status rc = gemm(u, u->colT, (int)P, u->dzT, (int)P, u->dwt, u->Kp[l], D.cout, P, kEpiF32, nullptr, splits);
    if (rc != MGMC_OK) return rc;
    k_wt_to_flat<<<grid_for((long long)u->K[l] * D.cout), 256, 0, st>>>(u->dwt, u->K[l], D.cout,
                                                                        u->grad + u->woff[l]);
    if (dx) {
        rc = gemm(u, u->dz, D.cout, u->Wt[l], D.cout, u->dcol, P, u->Kp[l], D.cout, kEpiF32, nullptr, 1);
        if (rc != MGMC_OK) return rc;
        k_col2im<<<grid_for(P * D.cin), 256, 0, st>>>(u->dcol, u->Kp[l], B, Hs, D.cin, dx, 0);
    }
    UNET_CUDA(cudaGetLastError());
    return MGMC_OK;
}

// offset of the loss partials in part[] (the column reductions use its start)
constexpr size_t kLossOff = (size_t)kRedBlocks * 260;

// loss and gradient of the batch at (input, target); gradient into u->grad
mgmc_status loss_grad(UnetCtx* u, int B, const bf16* input, const float* target)
{
    cudaStream_t st = u->stream;
    mgmc_status rc = forward(u, B, input);
    if (rc != MGMC_OK) return rc;
    const long long P0 = u->Ps(0, B);
    const float scale = 2.0f / (float)((long long)B * u->n * u->n);
    k_loss<<<kRedBlocks, 256, 0, st>>>(u->out, target, B, u->H, u->n, scale, u->dout, u->part + kLossOff);
    k_out_bwd<<<kRedBlocks, 256, 0, st>>>(u->dout, u->act[13], P0, u->c0, u->wout_r, u->dact[13], u->part);
    k_colsum<<<1, 256, 0, st>>>(u->part, kRedBlocks, u->c0 + 1, u->grad + u->out_w);
    const int c1 = u->L[2].cout, c2 = u->L[4].cout, c3 = u->L[6].cout, c0 = u->c0;
    auto pb = [&](int s, float* dy, float* dxx, int C) {  // pool of level s-1 -> s, backward
        k_pool_bwd<<<grid_for(u->Ps(s - 1, B) * C), 256, 0, st>>>(dy, B, u->Hs(s), C, dxx, 1);
    };
    auto ub = [&](int s, int ca, int cb, float* dlow, float* dskip) {
        k_upcat_bwd<<<grid_for(u->Ps(s, B) * (ca + cb)), 256, 0, st>>>(u->du, ca, cb, B, u->Hs(s), dlow, dskip);
    };
    if ((rc = conv_backward(u, 13, B, input, u->dact[12])) != MGMC_OK) return rc;
    if ((rc = conv_backward(u, 12, B, input, u->du)) != MGMC_OK) return rc;
    ub(0, c1, c0, u->dact[11], u->dact[1]);
    if ((rc = conv_backward(u, 11, B, input, u->dact[10])) != MGMC_OK) return rc;
    if ((rc = conv_backward(u, 10, B, input, u->du)) != MGMC_OK) return rc;
    ub(1, c2, c1, u->dact[9], u->dact[3]);
    if ((rc = conv_backward(u, 9, B, input, u->dact[8])) != MGMC_OK) return rc;
    if ((rc = conv_backward(u, 8, B, input, u->du)) != MGMC_OK) return rc;
    ub(2, c3, c2, u->dact[7], u->dact[5]);
    if ((rc = conv_backward(u, 7, B, input, u->dact[6])) != MGMC_OK) return rc;
    if ((rc = conv_backward(u, 6, B, input, u->dp)) != MGMC_OK) return rc;
    pb(3, u->dp, u->dact[5], c2);
    if ((rc = conv_backward(u, 5, B, input, u->dact[4])) != MGMC_OK) return rc;
    if ((rc = conv_backward(u, 4, B, input, u->dp)) != MGMC_OK) return rc;
    pb(2, u->dp, u->dact[3], c1);
    if ((rc = conv_backward(u, 3, B, input, u->dact[2])) != MGMC_OK) return rc;
    if ((rc = conv_backward(u, 2, B, input, u->dp)) != MGMC_OK) return rc;
    pb(1, u->dp, u->dact[1], c0);
    if ((rc = conv_backward(u, 1, B, input, u->dact[0])) != MGMC_OK) return rc;
    if ((rc = conv_backward(u, 0, B, input, nullptr)) != MGMC_OK) return rc;
    UNET_CUDA(cudaGetLastError());
    return MGMC_OK;
}

mgmc_status check_status(UnetCtx* u)
{
    int s = 0;
    UNET_CUDA(cudaStreamSynchronize(u->stream));
    UNET_CUDA(cudaMemcpy(&s, u->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (s == 2) return unet_fail(MGMC_ERR_TIMEOUT, "a tensor-core GEMM's bounded wait gave up");
    return MGMC_OK;
}

// mean squared error of the last loss_grad (synchronises the stream)
float host_loss(UnetCtx* u, int B)
{
    std::vector<float> p(kRedBlocks);
    cudaMemcpyAsync(p.data(), u->part + kLossOff, sizeof(float) * kRedBlocks, cudaMemcpyDeviceToHost, u->stream);
    cudaStreamSynchronize(u->stream);
    double s = 0.0;
    for (float v : p) s += v;
    return (float)(s / ((double)B * u->n * u->n));
}

}  // namespace
}  // namespace mgmc

// the handle type of the C ABI
struct mgmc_unet : mgmc::UnetCtx {
};

using namespace mgmc;

extern "C" {

mgmc_status mgmc_unet_create(int n, int c0, int max_batch, uint64_t seed, const mgmc_allocator* alloc, void* stream,
                             mgmc_unet_handle* out)
{
    if (!out) return unet_fail(MGMC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 31 || ((n + 1) & n) != 0 || (c0 != 8 && c0 != 16 && c0 != 32) || max_batch < 1 || max_batch > 64)
        return unet_fail(MGMC_ERR_ARG, "mgmc_unet_create: n = 2^k - 1 >= 31, c0 in {8, 16, 32}, 1 <= batch <= 64");
    mgmc_unet* u = new mgmc_unet();
    u->n = n;
    u->H = n + 1;
    u->c0 = c0;
    u->bmax = max_batch;
    u->stream = (cudaStream_t)stream;
    cudaGetDevice(&u->device);
    if (alloc && alloc->alloc && alloc->free) {
        u->alloc = *alloc;
        u->use_alloc = true;
    }
    auto fail_all = [&](mgmc_status s, const char* msg) {
        u->release();
        delete u;
        return unet_fail(s, msg);
    };
    layer_table(c0, u->L);
    long long o = 0;
    for (int l = 0; l < kLayers; ++l) {
        u->K[l] = 9 * u->L[l].cin;
        u->Kp[l] = round8(u->K[l]);
        u->woff[l] = o;
        o += (long long)u->L[l].cout * u->K[l];
        u->boff[l] = o;
        o += u->L[l].cout;
    }
    u->out_w = o;
    o += c0;
    u->out_b = o;
    o += 1;
    u->nparam = o;
    // He-normal weights (std sqrt(2 / fan_in)), zero biases; output weights std sqrt(1 / c0)
    std::vector<float> th((size_t)o, 0.f);
    SplitMix rng{seed};
    for (int l = 0; l < kLayers; ++l) {
        const double sd = std::sqrt(2.0 / u->K[l]);
        for (long long i = 0; i < (long long)u->L[l].cout * u->K[l]; ++i)
            th[(size_t)(u->woff[l] + i)] = (float)(sd * rng.normal());
    }
    for (int c = 0; c < c0; ++c) th[(size_t)(u->out_w + c)] = (float)(std::sqrt(1.0 / c0) * rng.normal());
    const size_t pb = sizeof(float) * (size_t)o;
    u->theta = (float*)u->get(pb);
    u->m = (float*)u->get(pb);
    u->v = (float*)u->get(pb);
    u->grad = (float*)u->get(pb);
    u->wout_r = (float*)u->get(sizeof(float) * c0);
    u->status = (int*)u->get(sizeof(int));
    if (!u->theta || !u->m || !u->v || !u->grad || !u->wout_r || !u->status)
        return fail_all(MGMC_ERR_OOM, "allocation failed");
    cudaMemcpyAsync(u->theta, th.data(), pb, cudaMemcpyHostToDevice, u->stream);
    cudaMemsetAsync(u->m, 0, pb, u->stream);
    cudaMemsetAsync(u->v, 0, pb, u->stream);
    cudaMemsetAsync(u->grad, 0, pb, u->stream);
    cudaMemsetAsync(u->status, 0, sizeof(int), u->stream);
    // buffers for max_batch samples
    const int B = max_batch;
    size_t col_elems = 0, dact_max = 0, dz_max = 0, dwt_max = 0;
    for (int l = 0; l < kLayers; ++l) {
        const long long P = u->Ps(u->L[l].level, B);
        u->Wb[l] = (bf16*)u->get(sizeof(bf16) * (size_t)u->L[l].cout * u->Kp[l]);
        u->Wt[l] = (bf16*)u->get(sizeof(bf16) * (size_t)u->L[l].cout * u->Kp[l]);
        u->act[l] = (bf16*)u->get(sizeof(bf16) * (size_t)P * u->L[l].cout);
        u->dact[l] = (float*)u->get(sizeof(float) * (size_t)P * u->L[l].cout);
        if (!u->Wb[l] || !u->Wt[l] || !u->act[l] || !u->dact[l]) return fail_all(MGMC_ERR_OOM, "allocation failed");
        col_elems = std::max(col_elems, (size_t)P * u->Kp[l]);
        dact_max = std::max(dact_max, (size_t)P * u->L[l].cin);
        dz_max = std::max(dz_max, (size_t)P * u->L[l].cout);
        dwt_max = std::max(dwt_max, (size_t)u->Kp[l] * u->L[l].cout);
    }
    // split-K partials: splits <= 304 / ceil(Kp / 128), so splits * Kp * cout <= 304 * 128 * 256
    u->wpart_elems = (size_t)304 * 128 * 256;
    const long long P0 = u->Ps(0, B);
    u->in = (bf16*)u->get(sizeof(bf16) * (size_t)P0 * 3);
    u->p0 = (bf16*)u->get(sizeof(bf16) * (size_t)u->Ps(1, B) * u->L[1].cout);
    u->p1 = (bf16*)u->get(sizeof(bf16) * (size_t)u->Ps(2, B) * u->L[3].cout);
    u->p2 = (bf16*)u->get(sizeof(bf16) * (size_t)u->Ps(3, B) * u->L[5].cout);
    u->u2 = (bf16*)u->get(sizeof(bf16) * (size_t)u->Ps(2, B) * u->L[8].cin);
    u->u1 = (bf16*)u->get(sizeof(bf16) * (size_t)u->Ps(1, B) * u->L[10].cin);
    u->u0 = (bf16*)u->get(sizeof(bf16) * (size_t)P0 * u->L[12].cin);
    u->out = (float*)u->get(sizeof(float) * (size_t)P0);
    u->dout = (float*)u->get(sizeof(float) * (size_t)P0);
    u->tgt = (float*)u->get(sizeof(float) * (size_t)B * n * n);
    u->col = (bf16*)u->get(sizeof(bf16) * col_elems);
    u->colT = (bf16*)u->get(sizeof(bf16) * col_elems);
    u->dcol = (float*)u->get(sizeof(float) * col_elems);
    u->dz = (bf16*)u->get(sizeof(bf16) * dz_max);
    u->dzT = (bf16*)u->get(sizeof(bf16) * dz_max);
    u->dwt = (float*)u->get(sizeof(float) * dwt_max);
    u->wpart = (float*)u->get(sizeof(float) * u->wpart_elems);
    u->part = (float*)u->get(sizeof(float) * (kLossOff + kRedBlocks));
    u->du = (float*)u->get(sizeof(float) * dact_max);
    u->dp = (float*)u->get(sizeof(float) * dact_max);
    u->idx = (long long*)u->get(sizeof(long long) * (size_t)B);
    if (!u->in || !u->p0 || !u->p1 || !u->p2 || !u->u2 || !u->u1 || !u->u0 || !u->out || !u->dout || !u->tgt ||
        !u->col || !u->colT || !u->dcol || !u->dz || !u->dzT || !u->dwt || !u->wpart || !u->part || !u->du ||
        !u->dp || !u->idx)
        return fail_all(MGMC_ERR_OOM, "allocation failed");
    if (refresh_bf16(u) != MGMC_OK || cudaStreamSynchronize(u->stream) != cudaSuccess)
        return fail_all(MGMC_ERR_CUDA, "U-Net set-up failed");
    *out = u;
    return MGMC_OK;
}

mgmc_status mgmc_unet_n_params(mgmc_unet_handle u, int64_t* count)
{
    if (!u || !count) return unet_fail(MGMC_ERR_ARG, "bad arguments");
    *count = u->nparam;
    return MGMC_OK;
}

mgmc_status mgmc_unet_get_params(mgmc_unet_handle u, float* host_out)
{
    if (!u || !host_out) return unet_fail(MGMC_ERR_ARG, "bad arguments");
    UNET_CUDA(cudaStreamSynchronize(u->stream));
    UNET_CUDA(cudaMemcpy(host_out, u->theta, sizeof(float) * u->nparam, cudaMemcpyDeviceToHost));
    return MGMC_OK;
}

mgmc_status mgmc_unet_set_params(mgmc_unet_handle u, const float* host_in)
{
    if (!u || !host_in) return unet_fail(MGMC_ERR_ARG, "bad arguments");
    UNET_CUDA(cudaMemcpyAsync(u->theta, host_in, sizeof(float) * u->nparam, cudaMemcpyHostToDevice, u->stream));
    UNET_CUDA(cudaMemsetAsync(u->m, 0, sizeof(float) * u->nparam, u->stream));
    UNET_CUDA(cudaMemsetAsync(u->v, 0, sizeof(float) * u->nparam, u->stream));
    u->step = 0;
    mgmc_status rc = refresh_bf16(u);
    if (rc != MGMC_OK) return rc;
    UNET_CUDA(cudaStreamSynchronize(u->stream));
    return MGMC_OK;
}

mgmc_status mgmc_unet_gradient(mgmc_unet_handle u, int batch, const void* inputs_bf16, const float* targets,
                               float* loss_out, float* grad_out)
{
    if (!u || !inputs_bf16 || !targets || batch < 1 || batch > u->bmax)
        return unet_fail(MGMC_ERR_ARG, "bad arguments");
    UNET_CUDA(cudaMemsetAsync(u->status, 0, sizeof(int), u->stream));
    mgmc_status rc = loss_grad(u, batch, (const bf16*)inputs_bf16, targets);
    if (rc != MGMC_OK) return rc;
    if ((rc = check_status(u)) != MGMC_OK) return rc;
    if (loss_out) *loss_out = host_loss(u, batch);
    if (grad_out) UNET_CUDA(cudaMemcpy(grad_out, u->grad, sizeof(float) * u->nparam, cudaMemcpyDeviceToHost));
    return MGMC_OK;
}

mgmc_status mgmc_unet_train(mgmc_unet_handle u, int64_t n_samples, const void* inputs_bf16, const float* targets,
                            int epochs, int batch, float lr, uint64_t shuffle_seed, float* epoch_loss)
{
    if (!u || !inputs_bf16 || !targets || batch < 1 || batch > u->bmax || n_samples < batch || epochs < 0 ||
        !(lr > 0.f))
        return unet_fail(MGMC_ERR_ARG, "bad arguments");
    cudaStream_t st = u->stream;
    UNET_CUDA(cudaMemsetAsync(u->status, 0, sizeof(int), st));
    const long long in_sz = (long long)u->H * u->H * 3, tgt_sz = (long long)u->n * u->n;
    std::vector<long long> perm((size_t)n_samples);
    SplitMix rng{shuffle_seed};
    std::vector<long long> hidx((size_t)batch);
    for (int e = 0; e < epochs; ++e) {
        for (long long i = 0; i < n_samples; ++i) perm[(size_t)i] = i;
        for (long long i = n_samples - 1; i > 0; --i)
            std::swap(perm[(size_t)i], perm[(size_t)(rng.next() % (uint64_t)(i + 1))]);
        const long long nb = n_samples / batch;
        double acc = 0.0;
        for (long long bi = 0; bi < nb; ++bi) {
            for (int k = 0; k < batch; ++k) hidx[(size_t)k] = perm[(size_t)(bi * batch + k)];
            UNET_CUDA(cudaMemcpyAsync(u->idx, hidx.data(), sizeof(long long) * batch, cudaMemcpyHostToDevice, st));
            k_gather<<<grid_for((long long)batch * (in_sz + tgt_sz)), 256, 0, st>>>(
                (const bf16*)inputs_bf16, targets, u->idx, batch, in_sz, tgt_sz, u->in, u->tgt);
            mgmc_status rc = loss_grad(u, batch, u->in, u->tgt);
            if (rc != MGMC_OK) return rc;
            ++u->step;
            const float c1 = 1.f - std::pow(0.9f, (float)u->step), c2 = 1.f - std::pow(0.999f, (float)u->step);
            k_adam<<<grid_for(u->nparam), 256, 0, st>>>(u->theta, u->m, u->v, u->grad, u->nparam, lr, 0.9f, 0.999f,
                                                      1e-8f, c1, c2);
            if ((rc = refresh_bf16(u)) != MGMC_OK) return rc;
            acc += host_loss(u, batch);  // synchronises: hidx is reused by the next batch
        }
        if (epoch_loss) epoch_loss[e] = (float)(acc / (double)std::max(1LL, nb));
    }
    return check_status(u);
}

mgmc_status mgmc_unet_predict(mgmc_unet_handle u, int64_t n_samples, const void* inputs_bf16, void* x_out,
                              int precision)
{
    if (!u || !inputs_bf16 || !x_out || n_samples < 0 || (precision != MGMC_FP32 && precision != MGMC_FP64))
        return unet_fail(MGMC_ERR_ARG, "bad arguments");
    UNET_CUDA(cudaMemsetAsync(u->status, 0, sizeof(int), u->stream));
    const long long in_sz = (long long)u->H * u->H * 3, nn = (long long)u->n * u->n;
    const size_t esz = precision == MGMC_FP64 ? 8 : 4;
    for (long long b0 = 0; b0 < n_samples; b0 += u->bmax) {
        const int B = (int)std::min<long long>(u->bmax, n_samples - b0);
        mgmc_status rc = forward(u, B, (const bf16*)inputs_bf16 + b0 * in_sz);
        if (rc != MGMC_OK) return rc;
        k_crop<<<grid_for((long long)B * nn), 256, 0, u->stream>>>(
            u->out, B, u->H, u->n, (char*)x_out + (size_t)b0 * nn * esz, precision == MGMC_FP64 ? 1 : 0);
    }
    UNET_CUDA(cudaGetLastError());
    return check_status(u);
}

mgmc_status mgmc_unet_inputs(int n, const double* kappa2, double kappa2_const, int m, const int32_t* obs_site,
                             const double* obs_w, int nnz_per_obs, const double* y, uint16_t* out)
{
    if (n < 1 || !out || m < 0 || (m > 0 && (!obs_site || !obs_w || !y || nnz_per_obs < 1)))
        return unet_fail(MGMC_ERR_ARG, "bad arguments");
    const int H = n + 1;
    std::vector<float> x((size_t)H * H * 3, 0.f);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            const double k2 = kappa2 ? kappa2[(size_t)j * n + i] : kappa2_const;
            if (!(k2 > 0.0)) return unet_fail(MGMC_ERR_ARG, "kappa^2 must be positive");
            x[((size_t)j * H + i) * 3 + 0] = (float)std::log(k2 / 10.0);
        }
    std::vector<double> w1((size_t)H * H, 0.0), w2((size_t)H * H, 0.0);
    for (int k = 0; k < m; ++k)
        for (int t = 0; t < nnz_per_obs; ++t) {
            const int s = obs_site[(size_t)k * nnz_per_obs + t];
            if (s < 0) continue;
            if (s >= n * n) return unet_fail(MGMC_ERR_ARG, "observation site out of range");
            const int i = s % n, j = s / n;
            w1[(size_t)j * H + i] += obs_w[(size_t)k * nnz_per_obs + t];
            w2[(size_t)j * H + i] += obs_w[(size_t)k * nnz_per_obs + t] * y[k];
        }
    for (size_t q = 0; q < (size_t)H * H; ++q) {
        x[q * 3 + 1] = (float)w1[q];
        x[q * 3 + 2] = (float)w2[q];
    }
    for (size_t q = 0; q < x.size(); ++q) {
        uint32_t bits;
        std::memcpy(&bits, &x[q], 4);
        bits += 0x7FFFu + ((bits >> 16) & 1u);  // round to nearest, ties to even (finite values)
        out[q] = (uint16_t)(bits >> 16);
    }
    return MGMC_OK;
}

mgmc_status mgmc_unet_destroy(mgmc_unet_handle u)
{
    if (!u) return MGMC_OK;
    cudaSetDevice(u->device);
    cudaStreamSynchronize(u->stream);
    u->release();
    delete u;
    return MGMC_OK;
}

mgmc_status mgmc_tc_gemm(const void* A, int lda, const void* B, int ldb, void* C, int M, int N, int K, int splits,
                         int epilogue, const float* bias, void* stream)
{
    static thread_local float* part = nullptr;
    static thread_local size_t part_bytes = 0;
    static thread_local int* status = nullptr;
    if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0 || splits < 1 || (epilogue & ~7) ||
        ((epilogue & kEpiBias) && !bias))
        return unet_fail(MGMC_ERR_ARG, "mgmc_tc_gemm: bad arguments");
    if (splits > 1 && epilogue != kEpiF32)
        return unet_fail(MGMC_ERR_ARG, "mgmc_tc_gemm: split-K needs the plain FP32 epilogue");
    cudaStream_t st = (cudaStream_t)stream;
    TcGemm g;
    if (!tc_gemm_plan(&g, A, lda, B, ldb, M, N, K, splits))
        return unet_fail(MGMC_ERR_ARG, "mgmc_tc_gemm: TMA descriptor encoding failed (alignment, lda/ldb)");
    if (!status) {
        UNET_CUDA(cudaMalloc(&status, sizeof(int)));
        UNET_CUDA(cudaMemset(status, 0, sizeof(int)));
    }
    void* out = C;
    if (g.splits > 1) {
        const size_t need = sizeof(float) * (size_t)g.splits * M * N;
        if (need > part_bytes) {
            if (part) cudaFree(part);
            part = nullptr;
            part_bytes = 0;
            UNET_CUDA(cudaMalloc(&part, need));
            part_bytes = need;
        }
        out = part;
    }
    UNET_CUDA(tc_gemm_run(g, out, epilogue, bias, status, st));
    if (g.splits > 1) UNET_CUDA(tc_reduce_splits(part, g.splits, (long long)M * N, (float*)C, st));
    return MGMC_OK;
}

}  // extern "C"
