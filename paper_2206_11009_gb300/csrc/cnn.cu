// Warm-start network: forward, backward and Adam kernels (BF16 operands, FP32 accumulation).
//
// Architecture (the same flat parameter layout as the FP64 reference in the tests):
//   block l = 0..3: h <- silu(rmsnorm(conv3x3(h; W_l, b_l, dilation 2^l); g_l)), 2 -> C -> C -> C -> C
//   head:           y <- conv3x3(h; W_4, b_4), C -> 2: predicted (u, v) / k^2
// Layouts: activations NCHW; conv inputs stored in BF16, pre-normalisation outputs and all
// gradients in FP32; weights kept in FP32 (Adam's master copy) with a BF16 copy for the
// convolutions.  The 32 -> 32 convolutions (forward, data and weight gradient) are implicit GEMMs
// on the tensor cores; the 2 -> 32 and 32 -> 2 ones run on the FP32 pipes.  Every reduction runs
// in a fixed order (per-block partials, then one pass).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "ot_ipm.h"
#include "tc05.cuh"

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

// ---- the 32 -> 32 convolutions on the tensor cores (implicit GEMM)
// BF16 operands in shared memory, FP32 accumulators in tensor memory, one elected thread issuing
// the MMAs.  Operands are K-major without swizzle: core matrices of 8 rows x 8 BF16 (16 bytes),
// core matrix (row / 8, k / 8) of an R-row operand at byte ((k / 8)(R / 8) + row / 8) 128, its row
// row % 8 at 16-byte steps, so the leading byte offset is (R / 8) 128 and one MMA (K = 16) spans
// two core-matrix columns.
//   conv:   D[pixel, o] = sum_{t, c} A[pixel, t 32 + c] Wop[o, t 32 + c], A the pixel's 9 taps x 32
//           channels (zero outside the image): M = 128 pixels, N = 32, K = 288 (18 MMAs).  The data
//           gradient is the same product over the output gradient with the taps mirrored.
//   wgrad:  D[t 32 + c, o] = sum_pixel A[t 32 + c, pixel] dz[o, pixel] over a chunk of 128 pixels:
//           rows padded to 384 (three M = 128 tiles), N = 32, K = 128 (8 MMAs per tile).
constexpr int kCvM = 128, kCvN = 32, kCvK = 9 * 32;
constexpr int kCvAbytes = kCvM * kCvK * 2;     // 73,728
constexpr int kCvBbytes = kCvN * kCvK * 2;     // 18,432: one layer's weight operand
constexpr int kCvSmem = kCvAbytes + kCvBbytes + 16;
constexpr uint32_t kCvIdesc = tc_idesc(1u, kCvM, kCvN);
constexpr int kWgRows = 384, kWgK = 128;        // weight-gradient rows (288 used), pixels per chunk
constexpr int kWgAbytes = kWgRows * kWgK * 2;  // 98,304
constexpr int kWgBbytes = kCvN * kWgK * 2;     // 8,192
constexpr int kWgSmem = kWgAbytes + kWgBbytes + 16;
constexpr int kWgStride = 32 * 32 * 9 + 32;    // one chunk's partial row: dW then db

// byte offset of element (row, k) in a K-major operand of R rows
__device__ __forceinline__ int cv_off(int row, int k, int R) {
    return ((k >> 3) * (R >> 3) + (row >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Weight operands of the three 32 -> 32 layers in the layout above, forward (Wop[o, t 32 + c] =
// W[o, c, t]) and mirrored for the data gradient (Wop'[c, t 32 + o] = W[o, c, 8 - t]); operand
// (layer l, mirrored f) at wop + (2 l + f) 32 288.
__global__ void conv_wop_kernel(const float *__restrict__ w, int64_t off1, int64_t off2, int64_t off3,
                                __nv_bfloat16 *__restrict__ wop) {
    const int per = kCvN * kCvK;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < 6 * per; q += gridDim.x * blockDim.x) {
        const int op = q / per, e = q % per, l = op >> 1, f = op & 1;
        const float *W = w + (l == 0 ? off1 : l == 1 ? off2 : off3);
        const int r = e / kCvK, k = e % kCvK, t = k >> 5, c = k & 31;
        const float v = f ? W[(c * 32 + r) * 9 + (8 - t)] : W[(r * 32 + c) * 9 + t];
        wop[(int64_t)op * per + cv_off(r, k, kCvN) / 2] = __float2bfloat16(v);
    }
}

// out[b, o, y, x] = bias[o] + sum_{c, t} Wop[o, t 32 + c] in[b, c, y + oy_t, x + ox_t] (zero
// padding, offsets (t / 3 - 1, t % 3 - 1) dil; bias may be NULL).  Persistent CTAs of 128
// threads take 128-pixel tiles gridDim.x apart: each thread gathers its pixel's 288 inputs into
// the A operand (16-byte stores), thread 0 issues the 18 MMAs and commits them to an mbarrier,
// and warp w reads accumulator lanes 32 w .. 32 w + 31 (its pixels) back.  The wait is bounded:
// a CTA in which it gives up records that in *err, waits once more for its MMAs and stops.
__global__ void __launch_bounds__(kCvM)
conv_tc_kernel(int B, int H, int Wd, int dil, const __nv_bfloat16 *__restrict__ in,
               const __nv_bfloat16 *__restrict__ wop, const float *__restrict__ bias, float *__restrict__ out,
               int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem, *sB = smem + kCvAbytes;
    uint64_t *mb = (uint64_t *)(sB + kCvBbytes);
    uint32_t *tslot = (uint32_t *)(mb + 1);
    const int HW = H * Wd;
    const int64_t P = (int64_t)B * HW, ntiles = (P + kCvM - 1) / kCvM;
    const int warp = threadIdx.x >> 5, p = threadIdx.x;
    for (int q = threadIdx.x; q < kCvBbytes / 16; q += blockDim.x) ((uint4 *)sB)[q] = ((const uint4 *)wop)[q];
    if (warp == 0) tc_alloc(tslot, kCvN);
    const uint32_t a0 = tc_smem_u32(sA), b0 = tc_smem_u32(sB), mbar = tc_smem_u32(mb);
    if (threadIdx.x == 0) {
        tc_mbar_init(mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const unsigned short *src16 = (const unsigned short *)in;
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int64_t pix = tile * kCvM + p;
        const bool valid = pix < P;
        const int b = valid ? (int)(pix / HW) : 0;
        const int yx = valid ? (int)(pix % HW) : 0, y = yx / Wd, x = yx % Wd;
        const unsigned short *src = src16 + (int64_t)b * 32 * HW;
#pragma unroll 1
        for (int t = 0; t < 9; ++t) {
            const int yy = y + (t / 3 - 1) * dil, xx = x + (t % 3 - 1) * dil;
            const bool ok = valid && yy >= 0 && yy < H && xx >= 0 && xx < Wd;
            const int off = ok ? yy * Wd + xx : 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t w4[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c = q * 8 + 2 * e;
                    const uint32_t lo = ok ? src[(int64_t)c * HW + off] : 0u;
                    const uint32_t hi = ok ? src[(int64_t)(c + 1) * HW + off] : 0u;
                    w4[e] = lo | (hi << 16);
                }
                *(uint4 *)(sA + cv_off(p, t * 32 + q * 8, kCvM)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
            }
        }
        // the generic-proxy stores above must be visible to the MMAs (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            const uint32_t lboA = (kCvM / 8) * 128, lboB = (kCvN / 8) * 128;
#pragma unroll
            for (int ks = 0; ks < kCvK / 16; ++ks)
                tc_mma<true>(tmem, tc_desc(a0 + ks * 2 * lboA, lboA), tc_desc(b0 + ks * 2 * lboB, lboB), kCvIdesc,
                             ks > 0);
            tc_commit(mbar);
        }
        const bool done = tc_wait(mbar, (uint32_t)(it & 1));
        if (__syncthreads_or(!done)) {
            if (threadIdx.x == 0) {
                atomicExch(err, 1);
                tc_wait(mbar, (uint32_t)(it & 1));   // its MMAs read this CTA's shared memory
            }
            break;
        }
        tc_fence_after();
        float v[32];
        tc_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
        if (valid) {
            float *dst = out + (int64_t)b * 32 * HW + yx;
#pragma unroll
            for (int o = 0; o < 32; ++o) dst[(int64_t)o * HW] = (bias ? bias[o] : 0.f) + v[o];
        }
        tc_fence_before();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tc_dealloc(tmem, kCvN);
}

// Partial weight and bias gradients of a 32 -> 32 convolution over chunk blockIdx.x of 128 pixels:
// part[chunk kWgStride + (o 32 + c) 9 + t] = sum_pixel dz[b, o, pixel] in[b, c, pixel + offset_t]
// and part[chunk kWgStride + 9216 + o] = sum_pixel dz[b, o, pixel] (FP32, a fixed order).  dz is
// rounded to BF16 for the MMAs.  The A operand is built in items of (row, 8 pixels), 32 items per
// warp pass: lanes 8 j + r take rows 8 R + r of one row octet R and pixel groups 4 G + j, so each
// phase of eight 16-byte stores covers eight distinct bank groups and each load instruction touches
// 8 channel planes in runs of 4 pixel groups.  Same waits and clean-up as conv_tc_kernel.
__global__ void __launch_bounds__(kCvM)
conv_wgrad_tc_kernel(int B, int H, int Wd, int dil, const __nv_bfloat16 *__restrict__ in,
                     const float *__restrict__ dz, float *__restrict__ part, int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ int sb[kWgK], sy[kWgK], sx[kWgK];
    __shared__ float sbias[kCvM];
    unsigned char *sA = smem, *sB = smem + kWgAbytes;
    uint64_t *mb = (uint64_t *)(sB + kWgBbytes);
    uint32_t *tslot = (uint32_t *)(mb + 1);
    const int HW = H * Wd;
    const int64_t P = (int64_t)B * HW, p0 = (int64_t)blockIdx.x * kWgK;
    const int np = (int)(P - p0 < kWgK ? P - p0 : kWgK);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) tc_alloc(tslot, 128);
    for (int i = threadIdx.x; i < kWgK; i += blockDim.x) {
        const int64_t pix = p0 + (i < np ? i : 0);
        const int yx = (int)(pix % HW);
        sb[i] = (int)(pix / HW);
        sy[i] = yx / Wd;
        sx[i] = yx % Wd;
    }
    if (threadIdx.x == 0) {
        tc_mbar_init(tc_smem_u32(mb), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // A: 192 warp passes of 32 items; rows 288.. are zero
    const unsigned short *in16 = (const unsigned short *)in;
    for (int qb = warp; qb < (kWgRows / 8) * (kWgK / 32); qb += kCvM / 32) {
        const int row = (qb % (kWgRows / 8)) * 8 + (lane & 7), kg = (qb / (kWgRows / 8)) * 4 + (lane >> 3);
        uint32_t w4[4] = {0u, 0u, 0u, 0u};
        if (row < kCvK) {
            const int t = row >> 5, c = row & 31;
            const int oy = (t / 3 - 1) * dil, ox = (t % 3 - 1) * dil;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int i = kg * 8 + e;
                uint32_t v = 0u;
                if (i < np) {
                    const int yy = sy[i] + oy, xx = sx[i] + ox;
                    if (yy >= 0 && yy < H && xx >= 0 && xx < Wd)
                        v = in16[((int64_t)sb[i] * 32 + c) * HW + yy * Wd + xx];
                }
                w4[e >> 1] |= v << ((e & 1) * 16);
            }
        }
        *(uint4 *)(sA + cv_off(row, kg * 8, kWgRows)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
    }
    // B: thread (o = tid % 32, pixel groups tid / 32 + 4 u), rounded to BF16; the FP32 sum of the
    // thread's 32 values (in pixel order) is its share of the bias gradient
    {
        const int o = threadIdx.x & 31;
        float bs = 0.f;
#pragma unroll 1
        for (int u = 0; u < 4; ++u) {
            const int kg = (threadIdx.x >> 5) + 4 * u;
            uint32_t w4[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int i = kg * 8 + e;
                const float v = i < np ? dz[((int64_t)sb[i] * 32 + o) * HW + sy[i] * Wd + sx[i]] : 0.f;
                bs += v;
                w4[e >> 1] |= (uint32_t)__bfloat16_as_ushort(__float2bfloat16(v)) << ((e & 1) * 16);
            }
            *(uint4 *)(sB + cv_off(o, kg * 8, kCvN)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
        sbias[threadIdx.x] = bs;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot, mbar = tc_smem_u32(mb);
    if (threadIdx.x == 0) {
        const uint32_t a0 = tc_smem_u32(sA), b0 = tc_smem_u32(sB);
        const uint32_t lboA = (kWgRows / 8) * 128, lboB = (kCvN / 8) * 128;
#pragma unroll
        for (int mt = 0; mt < kWgRows / 128; ++mt)
#pragma unroll
            for (int ks = 0; ks < kWgK / 16; ++ks)
                tc_mma<true>(tmem + (uint32_t)(mt * kCvN), tc_desc(a0 + mt * 16 * 128 + ks * 2 * lboA, lboA),
                             tc_desc(b0 + ks * 2 * lboB, lboB), kCvIdesc, ks > 0);
        tc_commit(mbar);
    }
    float *prow = part + (int64_t)blockIdx.x * kWgStride;
    if (warp == 0) prow[32 * 32 * 9 + lane] = ((sbias[lane] + sbias[lane + 32]) + sbias[lane + 64]) + sbias[lane + 96];
    const bool done = tc_wait(mbar, 0u);
    if (__syncthreads_or(!done)) {
        if (threadIdx.x == 0) {
            atomicExch(err, 1);
            tc_wait(mbar, 0u);
        }
    } else {
        tc_fence_after();
#pragma unroll 1
        for (int mt = 0; mt < kWgRows / 128; ++mt) {
            float v[32];
            tc_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mt * kCvN), v);
            const int row = mt * 128 + warp * 32 + lane;
            if (row < kCvK) {
                const int t = row >> 5, c = row & 31;
#pragma unroll
                for (int o = 0; o < 32; ++o) prow[(o * 32 + c) * 9 + t] = v[o];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tc_dealloc(tmem, 128);
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
    __nv_bfloat16 *wop = nullptr;   // tensor-core weight operands of layers 1-3 (forward, mirrored)
    int *derr = nullptr;            // set by a tensor-core kernel whose wait gave up
    int sms = 1;
    // activations of the last forward (B, k)
    int B = 0, k = 0;
    int64_t cap_pix = 0;
    __nv_bfloat16 *h[kLayers] = {};   // conv inputs: h[0] = the features
    float *z[kLayers] = {};           // conv outputs (z[4] = prediction)
    float *r[kLayers] = {};           // RMS of the normalised blocks
    float *g1 = nullptr, *g2 = nullptr;  // gradient ping-pong (B x C x HW)
    __nv_bfloat16 *gb = nullptr;         // BF16 copy of a gradient (the data gradient's operand)
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
    if (c->gb) cudaFree(c->gb);
    c->g1 = c->g2 = nullptr;
    c->gb = nullptr;
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
            cudaMalloc((void **)&c->g2, sizeof(float) * C * pix) != cudaSuccess ||
            cudaMalloc((void **)&c->gb, sizeof(__nv_bfloat16) * C * pix) != cudaSuccess)
            return cnn_fail(c, OT_ERR_OOM, "ot_cnn: gradient allocation failed");
        c->cap_pix = pix;
    }
    const int64_t nblk = (pix + kWgK - 1) / kWgK;   // chunk partials (128-pixel chunks, the most)
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
    conv_wop_kernel<<<blocks_for(6 * kCvN * kCvK, 256), 256, 0, c->st>>>(c->w, c->L[1].W, c->L[2].W, c->L[3].W, c->wop);
    if (cudaGetLastError() != cudaSuccess) return cnn_fail(c, OT_ERR_CUDA, "ot_cnn: launch failed");
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return OT_OK;
}

// tensor-core weight operand of 32 -> 32 layer l (1..3), forward or mirrored
const __nv_bfloat16 *wop_of(const ot_cnn *c, int l, int mirrored) {
    return c->wop + (int64_t)(2 * (l - 1) + mirrored) * kCvN * kCvK;
}

// a tensor-core kernel's wait that gave up (bounded waits; the flag is read after a synchronisation)
int check_tc(ot_cnn *c, const char *where) {
    int h = 0;
    if (cudaMemcpyAsync(&h, c->derr, sizeof(int), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        cudaStreamSynchronize(c->st) != cudaSuccess)
        return cnn_fail(c, OT_ERR_CUDA, std::string(where) + ": synchronisation failed");
    if (h) return cnn_fail(c, OT_ERR_TIMEOUT, std::string(where) + ": a tensor-core wait gave up");
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
        cudaMalloc((void **)&c->wb, sizeof(__nv_bfloat16) * c->nparam) != cudaSuccess ||
        cudaMalloc((void **)&c->wop, sizeof(__nv_bfloat16) * 6 * kCvN * kCvK) != cudaSuccess ||
        cudaMalloc((void **)&c->derr, sizeof(int)) != cudaSuccess) {
        ot_cnn_destroy(c);
        return cnn_fail(nullptr, OT_ERR_OOM, "ot_cnn_create: weight allocation failed");
    }
    cudaMemcpyAsync(c->w, params, nb, cudaMemcpyHostToDevice, c->st);
    cudaMemsetAsync(c->m, 0, nb, c->st);
    cudaMemsetAsync(c->v, 0, nb, c->st);
    cudaMemsetAsync(c->derr, 0, sizeof(int), c->st);
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaFuncSetAttribute(conv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kCvSmem) != cudaSuccess ||
            cudaFuncSetAttribute(conv_wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem) != cudaSuccess) {
            ot_cnn_destroy(c);
            return cnn_fail(nullptr, OT_ERR_CUDA, "ot_cnn_create: device query failed");
        }
    }
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
    const unsigned tc_grid = (unsigned)std::min<int64_t>((pix + kCvM - 1) / kCvM, 2LL * c->sms);
    for (int l = 0; l < kLayers; ++l) {
        const Layer &Ly = c->L[l];
        const __nv_bfloat16 *wl = c->wb + Ly.W;
        const float *bl = c->w + Ly.b;
        if (l == 0)
            conv_fwd_kernel<2, 32><<<gp, kPix, 0, st>>>(batch, k, k, Ly.dil, c->h[0], wl, bl, c->z[0]);
        else if (l < kLayers - 1)
            conv_tc_kernel<<<tc_grid, kCvM, kCvSmem, st>>>(batch, k, k, Ly.dil, c->h[l], wop_of(c, l, 0), bl, c->z[l],
                                                         c->derr);
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
    return check_tc(c, "ot_cnn_forward");
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
    const int nchunk_tc = (int)((pix + kWgK - 1) / kWgK);
    const unsigned tc_grid = (unsigned)std::min<int64_t>((pix + kCvM - 1) / kCvM, 2LL * c->sms);
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
            conv_wgrad_tc_kernel<<<nchunk_tc, kCvM, kWgSmem, st>>>(B, k, k, Ly.dil, c->h[l], dz, c->part, c->derr);
        else
            conv_bwd_weight_kernel<32, 2><<<nchunk, 256, 0, st>>>(B, k, k, Ly.dil, c->h[l], dz, c->part);
        CNN_LAUNCHED(c);
        // W and bias are contiguous in the flat layout: one pass over the partial rows
        const int nparts = (l > 0 && l < kLayers - 1) ? nchunk_tc : nchunk;
        reduce_rows_kernel<<<blocks_for(stride, 256), 256, 0, st>>>(stride, nparts, stride, c->part, grad + Ly.W);
        CNN_LAUNCHED(c);
        if (l > 0 || dx) {
            float *out = (l == 0) ? dx : bufs[flip];
            flip ^= 1;
            if (l == 0)
                conv_bwd_data_kernel<2, 32><<<gp, kPix, 0, st>>>(B, k, k, Ly.dil, dz, wl, out);
            else if (l < kLayers - 1) {
                to_bf16_kernel<<<blocks_for(32 * pix, 256), 256, 0, st>>>(32 * pix, dz, c->gb);
                CNN_LAUNCHED(c);
                conv_tc_kernel<<<tc_grid, kCvM, kCvSmem, st>>>(B, k, k, Ly.dil, c->gb, wop_of(c, l, 1), nullptr, out,
                                                             c->derr);
            } else
                conv_bwd_data_kernel<32, 2><<<gp, kPix, 0, st>>>(B, k, k, Ly.dil, dz, wl, out);
            CNN_LAUNCHED(c);
            gcur = out;
        }
    }
    return check_tc(c, "ot_cnn_backward");
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
    for (void *p : {(void *)c->w, (void *)c->m, (void *)c->v, (void *)c->wb, (void *)c->wop, (void *)c->derr,
                    (void *)c->part, (void *)c->lpart})
        if (p) cudaFree(p);
    delete c;
}

}  // extern "C"
