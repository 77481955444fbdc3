// Warm-start network: forward, backward and Adam kernels (BF16 operands, FP32 accumulation).
//
// Architecture (the same flat parameter layout as the FP64 reference in the tests):
//   block l = 0..3: h <- silu(rmsnorm(conv3x3(h; W_l, b_l, dilation 2^l); g_l)), 2 -> C -> C -> C -> C
//   head:           y <- conv3x3(h; W_4, b_4), C -> 2: predicted (u, v) / k^2
// Layouts: activations NCHW; conv inputs stored in BF16, pre-normalisation outputs and all
// gradients in FP32; weights kept in FP32 (Adam's master copy) with a BF16 copy for the
// convolutions.  Every reduction runs in a fixed order (per-block partials, then one pass).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "ot_ipm.h"

namespace ot {
namespace {

constexpr int kLayers = 5;
constexpr int kDil[kLayers] = {1, 2, 4, 8, 1};
constexpr float kEps = 1e-5f;
constexpr int kPix = 128;     // pixels per CTA in the per-pixel kernels
constexpr int kChunk = 256;   // pixels per CTA of the weight-gradient partials

struct Layer {
    int cin, cout, dil;
    bool norm;
    int64_t W, b, g;   // offsets in the flat parameter array
};

__device__ __forceinline__ float silu_f(float t) { return t / (1.f + __expf(-t)); }

// out[b, o, y, x] = bias[o] + sum_{c, t} W[o, c, t] in[b, c, y + oy_t, x + ox_t] (zero padding)
template <int CIN, int COUT>
__global__ void __launch_bounds__(kPix)
conv_fwd_kernel(int B, int H, int Wd, int dil, const __nv_bfloat16 *__restrict__ in,
                const __nv_bfloat16 *__restrict__ w, const float *__restrict__ bias, float *__restrict__ out) {
    __shared__ __align__(16) float ws[CIN * 9 * COUT];   // [c][t][o]
    for (int q = threadIdx.x; q < CIN * 9 * COUT; q += blockDim.x) {
        const int o = q % COUT, ct = q / COUT, c = ct / 9, t = ct % 9;
        ws[q] = __bfloat162float(w[((int64_t)o * CIN + c) * 9 + t]);
    }
    __syncthreads();
    const int64_t HW = (int64_t)H * Wd;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)B * HW) return;
    const int b = (int)(p / HW);
    const int yx = (int)(p % HW), y = yx / Wd, x = yx % Wd;
    float acc[COUT];
#pragma unroll
    for (int o = 0; o < COUT; ++o) acc[o] = bias[o];
    for (int c = 0; c < CIN; ++c) {
        const __nv_bfloat16 *src = in + ((int64_t)b * CIN + c) * HW;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int yy = y + (t / 3 - 1) * dil, xx = x + (t % 3 - 1) * dil;
            const float v = (yy >= 0 && yy < H && xx >= 0 && xx < Wd) ? __bfloat162float(src[yy * Wd + xx]) : 0.f;
            const float *wr = ws + (c * 9 + t) * COUT;
#pragma unroll
            for (int o = 0; o < COUT; ++o) acc[o] += v * wr[o];
        }
    }
#pragma unroll
    for (int o = 0; o < COUT; ++o) out[((int64_t)b * COUT + o) * HW + yx] = acc[o];
}

// h = silu(g * z / r), r = sqrt(mean_c z^2 + eps), per pixel; h stored in BF16
template <int C>
__global__ void __launch_bounds__(kPix)
norm_act_fwd_kernel(int B, int64_t HW, const float *__restrict__ z, const float *__restrict__ g,
                    float *__restrict__ r, __nv_bfloat16 *__restrict__ h) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)B * HW) return;
    const int64_t b = p / HW, yx = p % HW;
    const float *zp = z + b * C * HW + yx;
    float ss = 0.f;
#pragma unroll
    for (int c = 0; c < C; ++c) ss += zp[c * HW] * zp[c * HW];
    const float rr = sqrtf(ss / C + kEps);
    r[p] = rr;
    __nv_bfloat16 *hp = h + b * C * HW + yx;
#pragma unroll
    for (int c = 0; c < C; ++c) hp[c * HW] = __float2bfloat16(silu_f(g[c] * zp[c * HW] / rr));
}

// dz from dh through silu and the RMS normalisation; partial dg per CTA
template <int C>
__global__ void __launch_bounds__(kPix)
norm_act_bwd_kernel(int B, int64_t HW, const float *__restrict__ z, const float *__restrict__ r,
                    const float *__restrict__ g, const float *__restrict__ dh, float *__restrict__ dz,
                    float *__restrict__ gpart) {
    __shared__ float red[C][kPix / 32];
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float dgl[C];
#pragma unroll
    for (int c = 0; c < C; ++c) dgl[c] = 0.f;
    if (p < (int64_t)B * HW) {
        const int64_t b = p / HW, yx = p % HW;
        const float *zp = z + b * C * HW + yx;
        const float *dp = dh + b * C * HW + yx;
        const float rr = r[p];
        float dxh[C], xh[C];
        float dot = 0.f;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            xh[c] = zp[c * HW] / rr;
            const float yn = g[c] * xh[c];
            const float s = 1.f / (1.f + __expf(-yn));
            const float dyn = dp[c * HW] * (s + yn * s * (1.f - s));
            dgl[c] = dyn * xh[c];
            dxh[c] = dyn * g[c];
            dot += dxh[c] * xh[c];
        }
        dot /= C;
        float *dzp = dz + b * C * HW + yx;
#pragma unroll
        for (int c = 0; c < C; ++c) dzp[c * HW] = (dxh[c] - xh[c] * dot) / rr;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        float v = dgl[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[c][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < C) {
        float v = 0.f;
        for (int w = 0; w < kPix / 32; ++w) v += red[threadIdx.x][w];
        gpart[(int64_t)blockIdx.x * C + threadIdx.x] = v;
    }
}

// din[b, c, y, x] = sum_{o, t} W[o, c, t] dout[b, o, y - oy_t, x - ox_t]
template <int CIN, int COUT>
__global__ void __launch_bounds__(kPix)
conv_bwd_data_kernel(int B, int H, int Wd, int dil, const float *__restrict__ dout,
                     const __nv_bfloat16 *__restrict__ w, float *__restrict__ din) {
    __shared__ __align__(16) float ws[COUT * 9 * CIN];   // [o][t][c]
    for (int q = threadIdx.x; q < COUT * 9 * CIN; q += blockDim.x) {
        const int c = q % CIN, ot = q / CIN, o = ot / 9, t = ot % 9;
        ws[q] = __bfloat162float(w[((int64_t)o * CIN + c) * 9 + t]);
    }
    __syncthreads();
    const int64_t HW = (int64_t)H * Wd;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)B * HW) return;
    const int b = (int)(p / HW);
    const int yx = (int)(p % HW), y = yx / Wd, x = yx % Wd;
    float acc[CIN];
#pragma unroll
    for (int c = 0; c < CIN; ++c) acc[c] = 0.f;
    for (int o = 0; o < COUT; ++o) {
        const float *src = dout + ((int64_t)b * COUT + o) * HW;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int yy = y - (t / 3 - 1) * dil, xx = x - (t % 3 - 1) * dil;
            if (yy < 0 || yy >= H || xx < 0 || xx >= Wd) continue;
            const float gv = src[yy * Wd + xx];
            const float *wr = ws + (o * 9 + t) * CIN;
#pragma unroll
            for (int c = 0; c < CIN; ++c) acc[c] += gv * wr[c];
        }
    }
#pragma unroll
    for (int c = 0; c < CIN; ++c) din[((int64_t)b * CIN + c) * HW + yx] = acc[c];
}

// per-CTA partials of dW[o, c, t] = sum_pix dout[o, pix] in[c, pix + off_t] and db[o] over kChunk
// pixels; thread j owns the (c, t) pairs j, j + blockDim and all COUT outputs
template <int CIN, int COUT>
__global__ void __launch_bounds__(256)
conv_bwd_weight_kernel(int B, int H, int Wd, int dil, const __nv_bfloat16 *__restrict__ in,
                       const float *__restrict__ dout, float *__restrict__ part) {
    __shared__ __align__(16) float dO[kChunk][COUT];
    __shared__ int sb[kChunk], sy[kChunk], sx[kChunk];
    const int64_t HW = (int64_t)H * Wd, P = (int64_t)B * HW;
    const int64_t p0 = (int64_t)blockIdx.x * kChunk;
    for (int i = threadIdx.x; i < kChunk; i += blockDim.x) {
        const int64_t p = min(p0 + i, P - 1);
        const int yx = (int)(p % HW);
        sb[i] = (int)(p / HW);
        sy[i] = yx / Wd;
        sx[i] = yx % Wd;
    }
    for (int q = threadIdx.x; q < kChunk * COUT; q += blockDim.x) {
        const int o = q / kChunk, i = q % kChunk;
        const int64_t p = p0 + i;
        float v = 0.f;
        if (p < P) {
            const int64_t b = p / HW, yx = p % HW;
            v = dout[(b * COUT + o) * HW + yx];
        }
        dO[i][o] = v;
    }
    __syncthreads();
    const int np = (int)(P - p0 < kChunk ? P - p0 : kChunk);
    const int64_t stride = (int64_t)COUT * CIN * 9 + COUT;
    for (int ct = threadIdx.x; ct < CIN * 9; ct += blockDim.x) {
        const int c = ct / 9, t = ct % 9;
        const int oy = (t / 3 - 1) * dil, ox = (t % 3 - 1) * dil;
        float acc[COUT];
#pragma unroll
        for (int o = 0; o < COUT; ++o) acc[o] = 0.f;
        for (int i = 0; i < np; ++i) {
            const int yy = sy[i] + oy, xx = sx[i] + ox;
            if (yy < 0 || yy >= H || xx < 0 || xx >= Wd) continue;
            const float v = __bfloat162float(in[((int64_t)sb[i] * CIN + c) * HW + yy * Wd + xx]);
#pragma unroll
            for (int o = 0; o < COUT; ++o) acc[o] += dO[i][o] * v;
        }
#pragma unroll
        for (int o = 0; o < COUT; ++o) part[blockIdx.x * stride + ((int64_t)o * CIN + c) * 9 + t] = acc[o];
    }
    if (threadIdx.x < COUT) {
        float s = 0.f;
        for (int i = 0; i < np; ++i) s += dO[i][threadIdx.x];
        part[blockIdx.x * stride + (int64_t)COUT * CIN * 9 + threadIdx.x] = s;
    }
}

// out[j] = sum over nblk partial rows (fixed order); row stride `stride`
__global__ void reduce_rows_kernel(int64_t count, int nblk, int64_t stride, const float *__restrict__ part,
                                   float *__restrict__ out) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count; j += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int q = 0; q < nblk; ++q) s += part[(int64_t)q * stride + j];
        out[j] = s;
    }
}

// gauge-invariant loss per image (one CTA per image): t = mean((yu-u)-(yv-v))/2, r = residuals,
// dy = r / (B npix), lpart[b] = sum r^2
__global__ void loss_kernel(int B, int64_t HW, const float *__restrict__ y, const float *__restrict__ tgt,
                            float *__restrict__ dy, float *__restrict__ lpart) {
    __shared__ double sh[32];
    __shared__ double bc;
    const int b = blockIdx.x;
    const float *yu = y + (int64_t)b * 2 * HW, *yv = yu + HW;
    const float *tu = tgt + (int64_t)b * 2 * HW, *tv = tu + HW;
    double s = 0.0;
    for (int64_t q = threadIdx.x; q < HW; q += blockDim.x) s += (double)(yu[q] - tu[q]) - (double)(yv[q] - tv[q]);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) bc = s / (2.0 * (double)HW);
    __syncthreads();
    const float t = (float)bc;
    double l = 0.0;
    const float inv = 1.f / (float)((double)B * (double)HW);
    float *du = dy + (int64_t)b * 2 * HW, *dv = du + HW;
    for (int64_t q = threadIdx.x; q < HW; q += blockDim.x) {
        const float ru = (yu[q] - tu[q]) - t, rv = (yv[q] - tv[q]) + t;
        du[q] = ru * inv;
        dv[q] = rv * inv;
        l += (double)ru * ru + (double)rv * rv;
    }
    l = block_sum(l, sh);
    if (threadIdx.x == 0) lpart[b] = (float)l;
}

__global__ void to_bf16_kernel(int64_t n, const float *__restrict__ x, __nv_bfloat16 *__restrict__ y) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        y[j] = __float2bfloat16(x[j]);
}

__global__ void adam_kernel(int64_t n, const float *__restrict__ grad, float *__restrict__ w, float *__restrict__ m,
                            float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const float g = grad[j];
        const float mj = b1 * m[j] + (1.f - b1) * g;
        const float vj = b2 * v[j] + (1.f - b2) * g * g;
        m[j] = mj;
        v[j] = vj;
        w[j] -= lr * (mj / c1) / (sqrtf(vj / c2) + eps);
    }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace
}  // namespace ot

using namespace ot;

struct ot_cnn {
    int ch = 32;
    Layer L[kLayers];
    int64_t nparam = 0;
    cudaStream_t st = nullptr;
    float *w = nullptr, *m = nullptr, *v = nullptr;   // FP32 master weights and Adam moments
    __nv_bfloat16 *wb = nullptr;                      // BF16 copy
    // activations of the last forward (B, k)
    int B = 0, k = 0;
    int64_t cap_pix = 0;
    __nv_bfloat16 *h[kLayers] = {};   // conv inputs: h[0] = the features
    float *z[kLayers] = {};           // conv outputs (z[4] = prediction)
    float *r[kLayers] = {};           // RMS of the normalised blocks
    float *g1 = nullptr, *g2 = nullptr;  // gradient ping-pong (B x C x HW)
    float *part = nullptr;
    int64_t cap_part = 0;
    float *lpart = nullptr;
    std::string err;
};

namespace {

thread_local std::string g_cnn_err;

int cnn_fail(ot_cnn *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    g_cnn_err = msg;
    return code;
}

void layout(ot_cnn *c) {
    int64_t off = 0;
    int cin = 2;
    for (int l = 0; l < kLayers; ++l) {
        Layer &y = c->L[l];
        y.cin = cin;
        y.cout = l < kLayers - 1 ? c->ch : 2;
        y.dil = kDil[l];
        y.norm = l < kLayers - 1;
        y.W = off;
        off += (int64_t)y.cout * y.cin * 9;
        y.b = off;
        off += y.cout;
        y.g = -1;
        if (y.norm) {
            y.g = off;
            off += y.cout;
        }
        cin = y.cout;
    }
    c->nparam = off;
}

void free_acts(ot_cnn *c) {
    for (int l = 0; l < kLayers; ++l) {
        if (c->h[l]) cudaFree(c->h[l]);
        if (c->z[l]) cudaFree(c->z[l]);
        if (c->r[l]) cudaFree(c->r[l]);
        c->h[l] = nullptr; c->z[l] = nullptr; c->r[l] = nullptr;
    }
    if (c->g1) cudaFree(c->g1);
    if (c->g2) cudaFree(c->g2);
    c->g1 = c->g2 = nullptr;
    c->cap_pix = 0;
}

int ensure_acts(ot_cnn *c, int B, int k) {
    const int64_t pix = (int64_t)B * k * k;
    if (pix > c->cap_pix) {
        free_acts(c);
        const int64_t C = c->ch;
        for (int l = 0; l < kLayers; ++l) {
            const int64_t cin = c->L[l].cin, cout = c->L[l].cout;
            if (cudaMalloc((void **)&c->h[l], sizeof(__nv_bfloat16) * cin * pix) != cudaSuccess ||
                cudaMalloc((void **)&c->z[l], sizeof(float) * cout * pix) != cudaSuccess ||
                cudaMalloc((void **)&c->r[l], sizeof(float) * pix) != cudaSuccess)
                return cnn_fail(c, OT_ERR_OOM, "ot_cnn: activation allocation failed");
        }
        if (cudaMalloc((void **)&c->g1, sizeof(float) * C * pix) != cudaSuccess ||
            cudaMalloc((void **)&c->g2, sizeof(float) * C * pix) != cudaSuccess)
            return cnn_fail(c, OT_ERR_OOM, "ot_cnn: gradient allocation failed");
        c->cap_pix = pix;
    }
    const int64_t nblk = (pix + kChunk - 1) / kChunk;
    const int64_t need = nblk * ((int64_t)c->ch * c->ch * 9 + c->ch) + blocks_for(pix, kPix) * (int64_t)c->ch;
    if (need > c->cap_part) {
        if (c->part) cudaFree(c->part);
        if (cudaMalloc((void **)&c->part, sizeof(float) * need) != cudaSuccess)
            return cnn_fail(c, OT_ERR_OOM, "ot_cnn: partial-sum allocation failed");
        c->cap_part = need;
    }
    if (!c->lpart && cudaMalloc((void **)&c->lpart, sizeof(float) * 4096) != cudaSuccess)
        return cnn_fail(c, OT_ERR_OOM, "ot_cnn: loss buffer allocation failed");
    c->B = B;
    c->k = k;
    return OT_OK;
}

int refresh_bf16(ot_cnn *c) {
    to_bf16_kernel<<<blocks_for(c->nparam, 256), 256, 0, c->st>>>(c->nparam, c->w, c->wb);
    if (cudaGetLastError() != cudaSuccess) return cnn_fail(c, OT_ERR_CUDA, "ot_cnn: launch failed");
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return OT_OK;
}

#define CNN_LAUNCHED(c)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess) return cnn_fail(c, OT_ERR_CUDA, cudaGetErrorString(e_));   \
        g_launches.fetch_add(1, std::memory_order_relaxed);                               \
    } while (0)

}  // namespace

extern "C" {

int64_t ot_cnn_param_count(int32_t channels) {
    if (channels != 32) return -1;
    ot_cnn c;
    c.ch = channels;
    layout(&c);
    return c.nparam;
}

int ot_cnn_create(int32_t channels, const float *params, void *stream, ot_cnn_t **out) {
    if (!out) return cnn_fail(nullptr, OT_ERR_ARG, "ot_cnn_create: out is NULL");
    *out = nullptr;
    if (channels != 32) return cnn_fail(nullptr, OT_ERR_UNSUPPORTED, "ot_cnn_create: only 32 channels are built");
    if (!params) return cnn_fail(nullptr, OT_ERR_ARG, "ot_cnn_create: params is NULL");
    ot_cnn *c = new (std::nothrow) ot_cnn();
    if (!c) return cnn_fail(nullptr, OT_ERR_OOM, "ot_cnn_create: host allocation failed");
    c->ch = channels;
    layout(c);
    c->st = (cudaStream_t)stream;
    const size_t nb = sizeof(float) * c->nparam;
    if (cudaMalloc((void **)&c->w, nb) != cudaSuccess || cudaMalloc((void **)&c->m, nb) != cudaSuccess ||
        cudaMalloc((void **)&c->v, nb) != cudaSuccess ||
        cudaMalloc((void **)&c->wb, sizeof(__nv_bfloat16) * c->nparam) != cudaSuccess) {
        ot_cnn_destroy(c);
        return cnn_fail(nullptr, OT_ERR_OOM, "ot_cnn_create: weight allocation failed");
    }
    cudaMemcpyAsync(c->w, params, nb, cudaMemcpyHostToDevice, c->st);
    cudaMemsetAsync(c->m, 0, nb, c->st);
    cudaMemsetAsync(c->v, 0, nb, c->st);
    int rc = refresh_bf16(c);
    if (rc == OT_OK && cudaStreamSynchronize(c->st) != cudaSuccess) rc = cnn_fail(c, OT_ERR_CUDA, "ot_cnn_create: copy failed");
    if (rc != OT_OK) {
        ot_cnn_destroy(c);
        return rc;
    }
    *out = c;
    return OT_OK;
}

int ot_cnn_get_params(ot_cnn_t *c, float *params, int64_t cap) {
    if (!c || !params) return cnn_fail(c, OT_ERR_ARG, "ot_cnn_get_params: NULL argument");
    if (cap < c->nparam) return cnn_fail(c, OT_ERR_BUF_TOO_SMALL, "ot_cnn_get_params: buffer too small");
    if (cudaMemcpyAsync(params, c->w, sizeof(float) * c->nparam, cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        cudaStreamSynchronize(c->st) != cudaSuccess)
        return cnn_fail(c, OT_ERR_CUDA, "ot_cnn_get_params: copy failed");
    return OT_OK;
}

int ot_cnn_forward(ot_cnn_t *c, int32_t batch, int32_t k, const float *x, float *y) {
    if (!c || !x || batch <= 0 || k <= 0 || batch > 4096) return cnn_fail(c, OT_ERR_ARG, "ot_cnn_forward: bad argument");
    int rc = ensure_acts(c, batch, k);
    if (rc != OT_OK) return rc;
    const int64_t HW = (int64_t)k * k, pix = (int64_t)batch * HW;
    cudaStream_t st = c->st;
    to_bf16_kernel<<<blocks_for(2 * pix, 256), 256, 0, st>>>(2 * pix, x, c->h[0]);
    CNN_LAUNCHED(c);
    const unsigned gp = blocks_for(pix, kPix);
    for (int l = 0; l < kLayers; ++l) {
        const Layer &Ly = c->L[l];
        const __nv_bfloat16 *wl = c->wb + Ly.W;
        const float *bl = c->w + Ly.b;
        if (l == 0)
            conv_fwd_kernel<2, 32><<<gp, kPix, 0, st>>>(batch, k, k, Ly.dil, c->h[0], wl, bl, c->z[0]);
        else if (l < kLayers - 1)
            conv_fwd_kernel<32, 32><<<gp, kPix, 0, st>>>(batch, k, k, Ly.dil, c->h[l], wl, bl, c->z[l]);
        else
            conv_fwd_kernel<32, 2><<<gp, kPix, 0, st>>>(batch, k, k, Ly.dil, c->h[l], wl, bl, c->z[l]);
        CNN_LAUNCHED(c);
        if (Ly.norm) {
            norm_act_fwd_kernel<32><<<gp, kPix, 0, st>>>(batch, HW, c->z[l], c->w + Ly.g, c->r[l], c->h[l + 1]);
            CNN_LAUNCHED(c);
        }
    }
    if (y && cudaMemcpyAsync(y, c->z[kLayers - 1], sizeof(float) * 2 * pix, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return cnn_fail(c, OT_ERR_CUDA, "ot_cnn_forward: copy failed");
    return OT_OK;
}

int ot_cnn_loss(ot_cnn_t *c, const float *target, float *dy, float *loss) {
    if (!c || !target || !dy || !loss || c->B <= 0) return cnn_fail(c, OT_ERR_ARG, "ot_cnn_loss: bad argument");
    const int64_t HW = (int64_t)c->k * c->k;
    loss_kernel<<<c->B, 256, 0, c->st>>>(c->B, HW, c->z[kLayers - 1], target, dy, c->lpart);
    CNN_LAUNCHED(c);
    std::vector<float> lp(c->B);
    if (cudaMemcpyAsync(lp.data(), c->lpart, sizeof(float) * c->B, cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        cudaStreamSynchronize(c->st) != cudaSuccess)
        return cnn_fail(c, OT_ERR_CUDA, "ot_cnn_loss: copy failed");
    double s = 0.0;
    for (int b = 0; b < c->B; ++b) s += lp[b];
    *loss = (float)(s / (2.0 * (double)c->B * (double)HW));
    return OT_OK;
}

int ot_cnn_backward(ot_cnn_t *c, const float *dy, float *grad, float *dx) {
    if (!c || !dy || !grad || c->B <= 0) return cnn_fail(c, OT_ERR_ARG, "ot_cnn_backward: bad argument");
    const int B = c->B, k = c->k;
    const int64_t HW = (int64_t)k * k, pix = (int64_t)B * HW;
    cudaStream_t st = c->st;
    const unsigned gp = blocks_for(pix, kPix);
    const int nchunk = (int)((pix + kChunk - 1) / kChunk);
    const float *gcur = dy;   // gradient with respect to the current layer's output
    float *bufs[2] = {c->g1, c->g2};
    int flip = 0;
    for (int l = kLayers - 1; l >= 0; --l) {
        const Layer &Ly = c->L[l];
        const float *dz = gcur;
        if (Ly.norm) {
            float *out = bufs[flip];
            flip ^= 1;
            norm_act_bwd_kernel<32><<<gp, kPix, 0, st>>>(B, HW, c->z[l], c->r[l], c->w + Ly.g, gcur, out, c->part);
            CNN_LAUNCHED(c);
            reduce_rows_kernel<<<1, 32, 0, st>>>(Ly.cout, (int)gp, Ly.cout, c->part, grad + Ly.g);
            CNN_LAUNCHED(c);
            dz = out;
        }
        const int64_t stride = (int64_t)Ly.cout * Ly.cin * 9 + Ly.cout;
        const __nv_bfloat16 *wl = c->wb + Ly.W;
        if (l == 0)
            conv_bwd_weight_kernel<2, 32><<<nchunk, 256, 0, st>>>(B, k, k, Ly.dil, c->h[0], dz, c->part);
        else if (l < kLayers - 1)
            conv_bwd_weight_kernel<32, 32><<<nchunk, 256, 0, st>>>(B, k, k, Ly.dil, c->h[l], dz, c->part);
        else
            conv_bwd_weight_kernel<32, 2><<<nchunk, 256, 0, st>>>(B, k, k, Ly.dil, c->h[l], dz, c->part);
        CNN_LAUNCHED(c);
        // W and bias are contiguous in the flat layout: one pass over the partial rows
        reduce_rows_kernel<<<blocks_for(stride, 256), 256, 0, st>>>(stride, nchunk, stride, c->part, grad + Ly.W);
        CNN_LAUNCHED(c);
        if (l > 0 || dx) {
            float *out = (l == 0) ? dx : bufs[flip];
            flip ^= 1;
            if (l == 0)
                conv_bwd_data_kernel<2, 32><<<gp, kPix, 0, st>>>(B, k, k, Ly.dil, dz, wl, out);
            else if (l < kLayers - 1)
                conv_bwd_data_kernel<32, 32><<<gp, kPix, 0, st>>>(B, k, k, Ly.dil, dz, wl, out);
            else
                conv_bwd_data_kernel<32, 2><<<gp, kPix, 0, st>>>(B, k, k, Ly.dil, dz, wl, out);
            CNN_LAUNCHED(c);
            gcur = out;
        }
    }
    return OT_OK;
}

int ot_cnn_adam(ot_cnn_t *c, const float *grad, float lr, float beta1, float beta2, float eps, int32_t step) {
    if (!c || !grad || step < 1) return cnn_fail(c, OT_ERR_ARG, "ot_cnn_adam: bad argument");
    const float c1 = 1.f - std::pow(beta1, (float)step), c2 = 1.f - std::pow(beta2, (float)step);
    adam_kernel<<<blocks_for(c->nparam, 256), 256, 0, c->st>>>(c->nparam, grad, c->w, c->m, c->v, lr, beta1, beta2,
                                                                eps, c1, c2);
    CNN_LAUNCHED(c);
    return refresh_bf16(c);
}

const char *ot_cnn_last_error(const ot_cnn_t *c) { return c ? c->err.c_str() : g_cnn_err.c_str(); }

void ot_cnn_destroy(ot_cnn_t *c) {
    if (!c) return;
    free_acts(c);
    for (void *p : {(void *)c->w, (void *)c->m, (void *)c->v, (void *)c->wb, (void *)c->part, (void *)c->lpart})
        if (p) cudaFree(p);
    delete c;
}

}  // extern "C"
