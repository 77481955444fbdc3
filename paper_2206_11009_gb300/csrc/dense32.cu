// FP32 dense LDL^T of S_M with the explicit inverse of its unit lower factor (dense32.cuh).
//
// Per 64-column panel k (column-major, leading dimension ld):
//   colsum  sums of the panel's columns below its diagonal block (the rows not yet eliminated);
//   diag    one CTA factors the 64x64 diagonal block in shared memory, each pivot being minus the
//           sum of its column's remaining off-diagonal entries (in the block, plus the below-block
//           sum updated as columns are eliminated), and writes the inverse of the unit block;
//   panel   L21 = A21 L11^-T D1^-1 through the inverse block (a product of non-positive entries
//           with non-negative ones: no cancellation), LD = L21 D1;
//   invrow  block row k of X = L^-1: X_kj = L11^-1 B_kj (B: the updates accumulated in X);
//   update  one launch over 128x128 tiles of both rank-64 updates: the trailing lower triangle
//           A22 -= LD L21^T and the rows of X below the panel, B -= L21 X_k.
// The sequence depends on n only, so it is captured once into a CUDA graph.
#include "dense32.cuh"
#include "primitives.cuh"
#include "tc05.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

namespace ot {
namespace {

constexpr int kP = 64;       // panel width
constexpr int kMaxN = 65536;  // largest n
constexpr int kSlice = 16384; // rows per assembly block (a column slice of 64-bit sums in shared memory)
constexpr int kTT = 256;     // threads per CTA
constexpr int kTile = 128;   // update tile (rows and columns)
constexpr int kKc = 16;      // depth of one staged slice of the update tiles

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}

// One CTA per column j: S_jj' = -sum_i theta_ij theta_ij' / M_i over the sources i shared by j and
// j', accumulated in fixed point (2^62 / N_j per unit: each |S_jj'| <= N_j, and so is their sum).
// Above kSlice rows, block (j, y) keeps only the rows [y kSlice, (y + 1) kSlice) of column j and
// adds its part of the diagonal's sum to tot[j] (an integer sum: the same in any order).
__global__ void __launch_bounds__(kTT)
d32_assemble_kernel(int n, int ld, const int32_t *__restrict__ col_ptr, const int32_t *__restrict__ col_row,
                    const double *__restrict__ theta_col, const int32_t *__restrict__ row_ptr,
                    const int32_t *__restrict__ sj, const double *__restrict__ theta,
                    const double *__restrict__ Minv, const double *__restrict__ Nc, float *__restrict__ A,
                    float *__restrict__ d0, unsigned long long *__restrict__ tot) {
    extern __shared__ unsigned long long acc[];
    __shared__ unsigned long long red[kTT / 32];
    const int j = blockIdx.x;
    const int lo = blockIdx.y * kSlice, hi = min(n, lo + kSlice), len = hi - lo;
    for (int t = threadIdx.x; t < len; t += blockDim.x) acc[t] = 0ull;
    __syncthreads();
    const double Nj = Nc[j];
    const double scale = Nj > 0 ? 4611686018427387904.0 / Nj : 0.0;  // 2^62 / N_j
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (scale > 0) {
        for (int k = col_ptr[j] + warp; k < col_ptr[j + 1]; k += nw) {
            const int i = col_row[k];
            const double f = theta_col[k] * Minv[i] * scale;
            for (int e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += 32) {
                const int jp = sj[e];
                if (jp != j && jp >= lo && jp < hi)
                    atomicAdd(&acc[jp - lo], (unsigned long long)__double2ull_rn(f * theta[e]));
            }
        }
    }
    __syncthreads();
    unsigned long long s = 0;
    for (int t = threadIdx.x; t < len; t += blockDim.x) s += acc[t];
    s = warp_sum_u64(s);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < nw; ++w) t += red[w];
        if (tot) atomicAdd(&tot[j], t);
        else d0[j] = scale > 0 ? (float)((double)t / scale) : 0.f;
    }
    const double inv = scale > 0 ? 1.0 / scale : 0.0;
    for (int r = max(j + 1, lo) + threadIdx.x; r < hi; r += blockDim.x)
        A[(size_t)j * ld + r] = -(float)((double)acc[r - lo] * inv);
}

// the diagonal from the slices' integer sums (the same scaling as the single-block case)
__global__ void d32_diag_total_kernel(int n, const double *__restrict__ Nc, const unsigned long long *__restrict__ tot,
                                      float *__restrict__ d0) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const double Nj = Nc[j];
        const double scale = Nj > 0 ? 4611686018427387904.0 / Nj : 0.0;
        d0[j] = scale > 0 ? (float)((double)tot[j] / scale) : 0.f;
    }
}

// csum[l] = sum of column l over the rows [bs, n) (first panel; later panels receive these sums
// from the previous update's epilogue)
__global__ void __launch_bounds__(kTT)
d32_colsum_kernel(int n, int ld, int bs, const float *__restrict__ A, float *__restrict__ csum) {
    __shared__ double sh[kTT / 32];
    const int l = blockIdx.x;
    const float *col = A + (size_t)l * ld;
    double s = 0.0;
    for (int r = bs + threadIdx.x; r < n; r += blockDim.x) s += (double)col[r];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) csum[l] = (float)s;
}

// One CTA factors the diagonal block in micro-panels of 8 columns.  Warp 0 eliminates a
// micro-panel with its 64 rows in registers (lane q: rows q and q+32; shuffles only): each pivot
// is minus the sum of the column's remaining entries plus its below-block sum (np fixed-order
// partials in csum[p * kP + l]), kept as sums of same-sign terms by a recurrence over the
// micro-panel's own 8 x 8 block (the warp-wide sums are taken once per micro-panel).  Then all warps apply the micro-panel's rank-8 update to the rest of
// the block (two barriers per micro-panel instead of one per column).  Columns stay unscaled until
// the end (l_ij = S_ij / d_j).  The inverse of the unit block is formed afterwards by 8x8 block
// rows: X_II = L_II^-1 by warp 0, X_IJ = -X_II sum_K L_IK X_KJ by all threads.
constexpr int kMp = 8;   // micro-panel width
static_assert(kTT / 32 == kP / kMp && kTT == 4 * kP, "one warp per 8x8 diagonal block, 8b threads per b-pair");

// Warp 0's elimination of one micro-panel (columns c0 .. c0 + nc - 1) with the block's 64 rows in
// registers (lane q: rows q and q + 32).  prev >= 0: the micro-panel's columns first receive the
// rank-8 update of the micro-panel starting at prev (eliminated by this warp just before), in the
// same order as the other warps apply it to the later columns.  kFull: nc == kMp known at compile
// time, so the whole micro-panel is one straight-line block.
template <bool kFull>
__device__ __forceinline__ void d32_micro_panel(int lane, int k, int c0, int nc, int prev, float (*S)[kP + 1],
                                                float *g, const float *thr, float *ids, float *D) {
    const unsigned full = 0xffffffffu;
    const int ncc = kFull ? kMp : nc;
    __syncwarp();
    float v0[kMp], v1[kMp], gm[kMp], tl[kMp], dv[kMp], iv[kMp];
#pragma unroll
    for (int jj = 0; jj < kMp; ++jj) {
        v0[jj] = jj < ncc ? S[lane][c0 + jj] : 0.f;
        v1[jj] = jj < ncc ? S[lane + 32][c0 + jj] : 0.f;
        gm[jj] = jj < ncc ? g[c0 + jj] : 0.f;
        tl[jj] = jj < ncc ? thr[c0 + jj] : 0.f;
    }
    if (prev >= 0) {
        float a0[kMp], a1[kMp], gp[kMp], ip[kMp];
#pragma unroll
        for (int q = 0; q < kMp; ++q) {
            a0[q] = S[lane][prev + q];
            a1[q] = S[lane + 32][prev + q];
            gp[q] = g[prev + q];
            ip[q] = ids[prev + q];
        }
#pragma unroll
        for (int jj = 0; jj < kMp; ++jj) {
            if (jj < ncc) {
                const int l = c0 + jj;
                float s0 = 0.f, s1 = 0.f, sg = 0.f;
#pragma unroll
                for (int q = 0; q < kMp; ++q) {
                    const float f = S[l][prev + q] * ip[q];
                    s0 += a0[q] * f;
                    s1 += a1[q] * f;
                    sg += f * gp[q];
                }
                if (lane > l) v0[jj] -= s0;
                if (lane + 32 > l) v1[jj] -= s1;
                gm[jj] -= sg;
            }
        }
    }
    // The pivots without a warp reduction on their chain.  With W_c the sum of column c's entries in
    // the rows from c0 + 8 on (in the block, and below it through g) and B the micro-panel's own
    // 8 x 8 lower part, eliminating column c changes, for every later column j of the micro-panel,
    //   B[r][j] -= B[r][c] l_jc  (r > j),   W_j -= W_c l_jc,   g_j -= g_c l_jc,   l_jc = B[j][c] / d_c,
    // and d_j = -(sum_{r > j} B[r][j] + W_j).  Every W and every B entry below the diagonal stays a
    // sum of non-positive terms (an M-matrix's Schur complements), so the pivots keep the
    // cancellation-free form.  The 8 initial W sums are reduced together, B is broadcast once,
    // and the 8-step recurrence runs on scalars in every lane.
    const bool lo_half = c0 < 32;   // the micro-panel's rows c0 .. c0 + 7 sit in one half
    float W[kMp], B[kMp][kMp];
#pragma unroll
    for (int jj = 0; jj < kMp; ++jj) {
        W[jj] = (lane >= c0 + kMp ? v0[jj] : 0.f) + (lane + 32 >= c0 + kMp ? v1[jj] : 0.f);
#pragma unroll
        for (int r = 0; r < kMp; ++r) B[r][jj] = 0.f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int jj = 0; jj < kMp; ++jj) W[jj] += __shfl_xor_sync(full, W[jj], o);
#pragma unroll
    for (int jj = 0; jj < kMp; ++jj) {
        W[jj] += gm[jj];
#pragma unroll
        for (int r = jj + 1; r < kMp; ++r) B[r][jj] = __shfl_sync(full, lo_half ? v0[jj] : v1[jj], (c0 + r) & 31);
    }
    float L[kMp][kMp];   // L[j][c] = l_jc of the micro-panel (j > c)
#pragma unroll
    for (int jj = 0; jj < kMp; ++jj)
#pragma unroll
        for (int c = 0; c < kMp; ++c) L[jj][c] = 0.f;
#pragma unroll
    for (int jj = 0; jj < kMp; ++jj) {
        dv[jj] = INFINITY;
        iv[jj] = 0.f;
        if (jj < ncc) {
            float sum = W[jj];
#pragma unroll
            for (int r = jj + 1; r < kMp; ++r) sum += B[r][jj];
            const float d = -sum;
            const bool inf = !(d > tl[jj]);
            const float id = inf ? 0.f : 1.f / d;
#pragma unroll
            for (int j2 = jj + 1; j2 < kMp; ++j2) {
                const float l = B[j2][jj] * id;
                L[j2][jj] = l;
#pragma unroll
                for (int r = j2 + 1; r < kMp; ++r) B[r][j2] -= B[r][jj] * l;
                W[j2] -= W[jj] * l;
                gm[j2] -= gm[jj] * l;
            }
            dv[jj] = inf ? INFINITY : d;
            iv[jj] = id;
        }
    }
    // each lane's own rows, in the same order: S_ij -= S_ic l_jc for c < j, rows below j only
#pragma unroll
    for (int jj = 1; jj < kMp; ++jj) {
        const int j = c0 + jj;
#pragma unroll
        for (int c = 0; c < jj; ++c) {
            if (lane > j) v0[jj] -= v0[c] * L[jj][c];
            if (lane + 32 > j) v1[jj] -= v1[c] * L[jj][c];
        }
    }
#pragma unroll
    for (int jj = 0; jj < kMp; ++jj) {
        if (dv[jj] == INFINITY) {   // a grounded column: its entries no longer enter anything
            v0[jj] = 0.f;
            v1[jj] = 0.f;
        }
    }
#pragma unroll
    for (int jj = 0; jj < kMp; ++jj) {
        if (jj < ncc) {
            S[lane][c0 + jj] = v0[jj];
            S[lane + 32][c0 + jj] = v1[jj];
            if (lane == jj) {
                g[c0 + jj] = gm[jj];
                D[k + c0 + jj] = dv[jj];
                ids[c0 + jj] = iv[jj];
            }
        }
    }
}

// shared memory of one diagonal-block factorisation (kDiagSmem bytes when carved from a buffer)
struct DiagSmem {
    float (*S)[kP + 1];
    float (*Xs)[kP + 1];
    float (*Ts)[kP / 2 + 1];
    float *g, *thr, *ids;
};
constexpr int kDiagSmem = (2 * kP * (kP + 1) + (kP / 2) * (kP / 2 + 1) + 3 * kP) * 4;

__device__ __forceinline__ DiagSmem diag_smem(float *buf) {
    DiagSmem m;
    m.S = (float (*)[kP + 1])buf;
    m.Xs = (float (*)[kP + 1])(buf + kP * (kP + 1));
    m.Ts = (float (*)[kP / 2 + 1])(buf + 2 * kP * (kP + 1));
    m.g = buf + 2 * kP * (kP + 1) + (kP / 2) * (kP / 2 + 1);
    m.thr = m.g + kP;
    m.ids = m.thr + kP;
    return m;
}

// The diagonal block at k (bs columns) by one CTA of kTT threads.  The block and the partial sums
// are read through L2 (__ldcg).  The partial column sums below the block come as np strips of
// `per` rows each (per = 2: the step kernel's two half-strip CTAs), added in a fixed order.
__device__ __forceinline__ void d32_diag_block(const DiagSmem &m, int ld, int k, int bs, float *__restrict__ A,
                                               float *__restrict__ D, const float *__restrict__ d0,
                                               const float *__restrict__ csum, int np, int per, float eps,
                                               float *__restrict__ Linv) {
    float (*S)[kP + 1] = m.S;
    float (*Xs)[kP + 1] = m.Xs;
    float (*Ts)[kP / 2 + 1] = m.Ts;
    float *g = m.g, *thr = m.thr, *ids = m.ids;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // every global load of the block, of the first kP rows of partial sums and of the diagonal
    // is issued before the first of them is used (kTT = 4 kP threads: 16 block entries each)
    constexpr int kPer = kP * kP / kTT;
    const int nq0 = min(kP, np);
    float sv[kPer], cv[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int t = (int)threadIdx.x + q * kTT, i = t % kP, j = t / kP;
        sv[q] = (i > j && i < bs) ? __ldcg(A + (size_t)(k + j) * ld + (k + i)) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        // strip t / kP's sum: its per (1 or 2) partial rows added in order
        const int t = (int)threadIdx.x + q * kTT, row = t / kP, col = t % kP;
        float v = 0.f;
        if (t < nq0 * kP) {
            v = __ldcg(csum + (size_t)(row * per) * kP + col);
            if (per == 2) v += __ldcg(csum + (size_t)(row * per + 1) * kP + col);
        }
        cv[q] = v;
    }
    const float d0v = (int)threadIdx.x < bs ? d0[k + threadIdx.x] : 0.f;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int t = (int)threadIdx.x + q * kTT;
        S[t % kP][t / kP] = sv[q];
        Xs[t / kP][t % kP] = cv[q];
    }
    __syncthreads();
    // each column's partials: four threads take every fourth row, then one adds the four in order
    // (further chunks of kP rows, for n above 4096, the same way)
    float gs = 0.f;
    {
        const int c = threadIdx.x % kP, h = threadIdx.x / kP;
        float part = 0.f;
        for (int q = h; q < nq0; q += kTT / kP) part += Xs[q][c];
        float *red = &Ts[0][0];   // free until the block inverse: [4][kP] here
        red[h * kP + c] = part;
        __syncthreads();
        if (threadIdx.x < kP && (int)threadIdx.x < bs) gs = red[c] + red[kP + c] + red[2 * kP + c] + red[3 * kP + c];
    }
    for (int q0 = kP; q0 < np; q0 += kP) {
        const int nq = min(kP, np - q0);
        for (int t = threadIdx.x; t < nq * kP; t += blockDim.x) {
            const int row = q0 + t / kP, col = t % kP;
            float v = __ldcg(csum + (size_t)(row * per) * kP + col);
            if (per == 2) v += __ldcg(csum + (size_t)(row * per + 1) * kP + col);
            Xs[t / kP][col] = v;
        }
        __syncthreads();
        if (threadIdx.x < kP && threadIdx.x < bs)
            for (int q = 0; q < nq; ++q) gs += Xs[q][threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x < kP) {
        g[threadIdx.x] = gs;
        thr[threadIdx.x] = eps * d0v;
    }
    __syncthreads();
    // micro-panel 0, then per step: warp 0 updates and eliminates the next micro-panel while the
    // other warps apply the current one's rank-8 update to the columns after it
    if (warp == 0) {
        if (bs >= kMp) d32_micro_panel<true>(lane, k, 0, kMp, -1, S, g, thr, ids, D);
        else d32_micro_panel<false>(lane, k, 0, bs, -1, S, g, thr, ids, D);
    }
    __syncthreads();
    for (int c0 = 0; c0 < bs; c0 += kMp) {
        const int c1 = c0 + kMp, nc1 = min(kMp, bs - c1);   // micro-panel c0 is full when c1 < bs
        if (warp == 0) {
            if (nc1 == kMp) d32_micro_panel<true>(lane, k, c1, kMp, c0, S, g, thr, ids, D);
            else if (nc1 > 0) d32_micro_panel<false>(lane, k, c1, nc1, c0, S, g, thr, ids, D);
        } else {
            // rank-8 update of the columns l >= lo: S[i][l] -= sum_jj S[i][c] S[l][c] / d_c (i > l),
            // and of their below-block sums: g[l] -= sum_jj (S[l][c] / d_c) g[c].  Thread (ty, tx):
            // the columns la = lo + tx and lb = la + 32 with their 8 factors in registers, the rows
            // lo + ty, +7, ... (each row's 8 entries read once for both columns)
            const int lo = c1 + max(nc1, 0);
            if (lo < bs) {
                const int tx = lane, ty = warp - 1;
                const int la = lo + tx, lb = la + 32;
                float fa[kMp], fb[kMp];
#pragma unroll
                for (int jj = 0; jj < kMp; ++jj) {
                    fa[jj] = (la < bs) ? S[la][c0 + jj] * ids[c0 + jj] : 0.f;
                    fb[jj] = (lb < bs) ? S[lb][c0 + jj] * ids[c0 + jj] : 0.f;
                }
                for (int i = lo + ty; i < bs; i += kTT / 32 - 1) {
                    if (i <= la) continue;
                    float sa = 0.f, sb = 0.f;
#pragma unroll
                    for (int jj = 0; jj < kMp; ++jj) {
                        const float x = S[i][c0 + jj];
                        sa += x * fa[jj];
                        sb += x * fb[jj];
                    }
                    S[i][la] -= sa;
                    if (i > lb) S[i][lb] -= sb;
                }
                if (ty == 0) {
                    float ga = 0.f, gb = 0.f;
#pragma unroll
                    for (int jj = 0; jj < kMp; ++jj) {
                        ga += fa[jj] * g[c0 + jj];
                        gb += fb[jj] * g[c0 + jj];
                    }
                    if (la < bs) g[la] -= ga;
                    if (lb < bs) g[lb] -= gb;
                }
            }
        }
        __syncthreads();
    }
    // scale the columns: L = S D^-1 (grounded columns are zero); back to A
    for (int t = threadIdx.x; t < kP * kP; t += blockDim.x) {
        const int i = t % kP, j = t / kP;
        const float l = (i > j && i < bs) ? S[i][j] * ids[j] : 0.f;
        S[i][j] = l;
        Xs[i][j] = 0.f;
        if (i > j && i < bs) A[(size_t)(k + j) * ld + (k + i)] = l;
    }
    __syncthreads();
    // X = L^-1 by recursive doubling.  Level 0: warp w inverts the diagonal 8x8 block w (lane c:
    // column c by forward substitution).  Level b = 8, 16, 32: for each pair of b-blocks on the
    // diagonal, X21 = -X22 (L21 X11), the product staged through Ts.  L <= 0 below the diagonal
    // and X >= 0, so every sum has terms of one sign.  Rows and columns >= bs hold the identity.
    if (lane < kMp) {
        const int o = warp * kMp;
        float x[kMp];
#pragma unroll
        for (int r = 0; r < kMp; ++r) {
            float v = (r == lane) ? 1.f : 0.f;
#pragma unroll
            for (int q = 0; q < r; ++q) v -= S[o + r][o + q] * x[q];
            x[r] = r < lane ? 0.f : v;
        }
#pragma unroll
        for (int r = 0; r < kMp; ++r) Xs[o + r][o + lane] = x[r];
    }
    __syncthreads();
#pragma unroll
    for (int b = kMp; b < kP; b *= 2) {
        // 8b threads per pair: column c, rows rg * (b / 8) .. + b / 8 of the pair's b x b product
        const int pair = threadIdx.x / (8 * b), loc = threadIdx.x % (8 * b);
        const int c = loc % b, q0 = (loc / b) * (b / 8);
        const int o = 2 * b * pair;
        float acc[kP / 16];
#pragma unroll
        for (int q = 0; q < b / 8; ++q) acc[q] = 0.f;
        for (int kk = c; kk < b; ++kk) {
            const float xk = Xs[o + kk][o + c];
#pragma unroll
            for (int q = 0; q < b / 8; ++q) acc[q] += S[o + b + q0 + q][o + kk] * xk;
        }
#pragma unroll
        for (int q = 0; q < b / 8; ++q) Ts[b * pair + q0 + q][c] = acc[q];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < b / 8; ++q) acc[q] = 0.f;
        for (int r = 0; r < q0 + b / 8; ++r) {
            const float t = Ts[b * pair + r][c];
#pragma unroll
            for (int q = 0; q < b / 8; ++q)
                if (r <= q0 + q) acc[q] += Xs[o + b + q0 + q][o + b + r] * t;
        }
#pragma unroll
        for (int q = 0; q < b / 8; ++q) Xs[o + b + q0 + q][o + c] = -acc[q];
        __syncthreads();
    }
    for (int t = threadIdx.x; t < bs * bs; t += blockDim.x) {
        const int i = t % bs, j = t / bs;
        Linv[(size_t)j * ld + (k + i)] = Xs[i][j];
    }
}

// L0 != NULL: first the rows [k, k + bs) of the previous panel's L21 (kept in L0 by the step
// kernel, whose other CTAs read those rows of A unscaled) go to A
__global__ void __launch_bounds__(kTT)
d32_diag_kernel(int ld, int k, int bs, float *__restrict__ A, float *__restrict__ D, const float *__restrict__ d0,
                const float *__restrict__ csum, int np, int per, float eps, float *__restrict__ Linv,
                const float *__restrict__ L0) {
    __shared__ __align__(16) float buf[kDiagSmem / 4];
    if (L0)
        for (int t = threadIdx.x; t < kP * kP; t += blockDim.x) {
            const int r = t % kP, j = t / kP;
            if (r < bs) A[(size_t)(k - kP + j) * ld + k + r] = L0[j * kP + r];
        }
    d32_diag_block(diag_smem(buf), ld, k, bs, A, D, d0, csum, np, per, eps, Linv);
}

// rows r in [k+64, n) of the panel (bs = 64 whenever rows remain below the block): 64 rows per
// CTA, 4 rows x 4 columns per thread, T = A21 L11^-T staged through shared memory
__global__ void __launch_bounds__(kTT)
d32_panel_kernel(int n, int ld, int k, float *__restrict__ A, const float *__restrict__ D,
                 const float *__restrict__ Linv, float *__restrict__ LD) {
    __shared__ __align__(16) float As[kP][kP];   // As[l][r] = A(r0 + r, k + l)
    __shared__ __align__(16) float Lt[kP][kP];   // Lt[l][j] = (L11^-1)_jl
    const int r0 = k + kP + blockIdx.x * kP;
    for (int t = threadIdx.x; t < kP * kP; t += blockDim.x) {
        const int j = t % kP, l = t / kP;
        Lt[l][j] = Linv[(size_t)l * ld + (k + j)];
        As[l][j] = r0 + j < n ? A[(size_t)(k + l) * ld + r0 + j] : 0.f;
    }
    __syncthreads();
    const int tr = threadIdx.x & 15, tc = threadIdx.x >> 4;  // rows tr*4.., columns tc*4..
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[u][w] = 0.f;
#pragma unroll 16
    for (int l = 0; l < kP; ++l) {
        const float4 a = *(const float4 *)&As[l][tr * 4];
        const float4 b = *(const float4 *)&Lt[l][tc * 4];
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[u][w] += av[u] * bv[w];
    }
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int j = tc * 4 + w;
        const float dj = D[k + j];
        const bool inf = isinf(dj);
        const float id = inf ? 0.f : 1.f / dj;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = r0 + tr * 4 + u;
            if (r < n) {
                LD[(size_t)j * ld + r] = inf ? 0.f : acc[u][w];
                A[(size_t)(k + j) * ld + r] = acc[u][w] * id;
            }
        }
    }
}

// block row k of X = L^-1 for the columns [c0, c0+64) of [0, k+bs); 4 rows x 4 columns per thread
__global__ void __launch_bounds__(kTT)
d32_invrow_kernel(int ld, int k, int bs, float *__restrict__ X, const float *__restrict__ Linv) {
    __shared__ __align__(16) float Lt[kP][kP];   // Lt[l][i] = (L11^-1)_il
    __shared__ __align__(16) float B[kP][kP];    // B[l][c] = X(k + l, c0 + c)
    const int c0 = blockIdx.x * kP;
    const int base = k + bs;
    for (int t = threadIdx.x; t < kP * kP; t += blockDim.x) {
        const int i = t % kP, l = t / kP;
        Lt[l][i] = (i < bs && l < bs) ? Linv[(size_t)l * ld + (k + i)] : 0.f;
    }
    for (int t = threadIdx.x; t < kP * kP; t += blockDim.x) {
        const int l = t % kP, c = t / kP;
        B[l][c] = (l < bs && c0 + c < k) ? X[(size_t)(c0 + c) * ld + (k + l)] : 0.f;
    }
    __syncthreads();
    const int ti = threadIdx.x & 15, tcc = threadIdx.x >> 4;  // rows ti*4.., columns tcc*4..
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[u][w] = 0.f;
    if (c0 < k) {
#pragma unroll 16
        for (int l = 0; l < kP; ++l) {
            const float4 a = *(const float4 *)&Lt[l][ti * 4];
            const float4 b = *(const float4 *)&B[l][tcc * 4];
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w] += av[u] * bv[w];
        }
    }
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int c = c0 + tcc * 4 + w;
        if (c >= base) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = ti * 4 + u;
            if (i >= bs) continue;
            X[(size_t)c * ld + (k + i)] = c < k ? acc[u][w] : Lt[c - k][i];
        }
    }
}

// The two rank-64 updates of panel k (trailing triangle A22 -= LD L21^T, rows of L^-1 below the
// panel B -= L21 X_k) are split in two launches: d32_update1_kernel covers what the next panel
// needs (its 64 columns of A22 and its 64 rows of B, 64x64 tiles) and d32_update_kernel the rest
// (rows and columns from base2 = k + 128 on, 128x128 tiles, 8x8 per thread).
__device__ __forceinline__ void tri_decode(int idx, int &ti, int &tj) {
    ti = (int)((sqrt(8.0 * idx + 1.0) - 1.0) * 0.5);
    while ((ti + 1) * (ti + 2) / 2 <= idx) ++ti;
    while (ti * (ti + 1) / 2 > idx) --ti;
    tj = idx - ti * (ti + 1) / 2;
}

// the next panel's part: blocks [0, ts) are the 64-column strip of A22 in 64-row tiles (with the
// strip's column sums below the next diagonal block, csum[s * 64 + c], fixed-order partials),
// blocks [ts, ts + tx) the next panel's 64 rows of B in 64-column tiles; all of K = 64 staged once
__global__ void __launch_bounds__(kTT)
d32_update1_kernel(int n, int ld, int k, float *__restrict__ A, float *__restrict__ X,
                   const float *__restrict__ LD, float *__restrict__ csum) {
    __shared__ __align__(16) float As[kP][kP];   // As[l][r] = A operand (row r0 + r, depth l)
    __shared__ __align__(16) float Bs[kP][kP];   // Bs[l][c] = B operand (column c0 + c, depth l)
    const int base = k + kP;
    const int ts = (n - base + kP - 1) / kP;
    const bool strip = (int)blockIdx.x < ts;
    const int r0 = strip ? base + (int)blockIdx.x * kP : base;
    const int c0 = strip ? base : ((int)blockIdx.x - ts) * kP;
    const int climit = strip ? n : base;
    const float *Pa = strip ? LD : A + (size_t)k * ld;
    const float *Pb = A + (size_t)k * ld;
    for (int t = threadIdx.x; t < kP * (kP / 4); t += kTT) {
        const int l = t / (kP / 4), q = (t % (kP / 4)) * 4;
        const float *src = Pa + (size_t)l * ld + r0 + q;
        float4 v;
        if (r0 + q + 4 <= n) v = *(const float4 *)src;
        else {
            v.x = r0 + q < n ? src[0] : 0.f;
            v.y = r0 + q + 1 < n ? src[1] : 0.f;
            v.z = r0 + q + 2 < n ? src[2] : 0.f;
            v.w = r0 + q + 3 < n ? src[3] : 0.f;
        }
        *(float4 *)&As[l][q] = v;
        if (strip) {
            const float *sb = Pb + (size_t)l * ld + c0 + q;
            float4 w;
            if (c0 + q + 4 <= climit) w = *(const float4 *)sb;
            else {
                w.x = c0 + q < climit ? sb[0] : 0.f;
                w.y = c0 + q + 1 < climit ? sb[1] : 0.f;
                w.z = c0 + q + 2 < climit ? sb[2] : 0.f;
                w.w = c0 + q + 3 < climit ? sb[3] : 0.f;
            }
            *(float4 *)&Bs[l][q] = w;
        } else {
            const int c = t % kP, lq = (t / kP) * 4;
            float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c0 + c < climit) w = *(const float4 *)(X + (size_t)(c0 + c) * ld + k + lq);
            Bs[lq][c] = w.x;
            Bs[lq + 1][c] = w.y;
            Bs[lq + 2][c] = w.z;
            Bs[lq + 3][c] = w.w;
        }
    }
    __syncthreads();
    const int tr = threadIdx.x & 15, tc = threadIdx.x >> 4;   // rows tr*4.., columns tc*4..
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[u][w] = 0.f;
#pragma unroll 16
    for (int l = 0; l < kP; ++l) {
        const float4 a = *(const float4 *)&As[l][tr * 4];
        const float4 b = *(const float4 *)&Bs[l][tc * 4];
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[u][w] += av[u] * bv[w];
    }
    float *C = strip ? A : X;
    float cs[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int c = c0 + tc * 4 + w;
        if (c >= climit) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = r0 + tr * 4 + u;
            if (r < n && (!strip || r > c)) {
                const float v = C[(size_t)c * ld + r] - acc[u][w];
                C[(size_t)c * ld + r] = v;
                if (r >= base + kP) cs[w] += v;
            }
        }
    }
    if (strip) {
        // the 16 threads with this tc are one half-warp (lanes tr = 0..15)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            float v = cs[w];
#pragma unroll
            for (int o = 1; o < 16; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (tr == 0) csum[(size_t)blockIdx.x * kP + tc * 4 + w] = v;
        }
    }
}

// the rest of the update from base2 = base + skip * 64 on (skip = 1, or 2 when the block after
// the next panel went to its own d32_update1_kernel launch)
__global__ void __launch_bounds__(kTT, 2)
d32_update_kernel(int n, int ld, int k, int skip, float *__restrict__ A, float *__restrict__ X,
                  const float *__restrict__ LD) {
    // two stages: slice s + 1 is fetched into registers while slice s is multiplied
    __shared__ __align__(16) float As[2][kKc][kTile];
    __shared__ __align__(16) float Bs[2][kKc][kTile];
    const int base = k + kP, base2 = base + skip * kP;
    const int t = (n - base2 + kTile - 1) / kTile;   // row / column tiles from base2 on
    const int tcn = (base + kTile - 1) / kTile;      // column tiles of the rows of L^-1
    const int idx = blockIdx.x;
    const int ntri = t * (t + 1) / 2;                // trailing tiles, diagonal ones included
    const bool tri = idx < ntri;
    int ti, tj;
    if (tri) {
        tri_decode(idx, ti, tj);
    } else {
        const int q = idx - ntri;
        ti = q / tcn;
        tj = q % tcn;
    }
    const int r0 = base2 + ti * kTile;
    const int c0 = tri ? base2 + tj * kTile : tj * kTile;
    const int climit = tri ? n : base;
    // A operand (l, r) = Pa[l * ld + r]; B operand (l, c) = Pb[l * ld + c] (trailing) or
    // X[c * ld + k + l] (inverse)
    const float *Pa = tri ? LD : A + (size_t)k * ld;
    const float *Pb = A + (size_t)k * ld;
    const int tr = threadIdx.x & 15, tc = threadIdx.x >> 4;
    float acc[8][8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int w = 0; w < 8; ++w) acc[u][w] = 0.f;
    float ra[8], rb[8];
    const int fl = threadIdx.x >> 4, fq = (threadIdx.x & 15) * 8;       // A (and trailing B) slot
    const int xc = threadIdx.x & (kTile - 1), xh = threadIdx.x >> 7;      // inverse B slot
    const float *pa0 = Pa + (size_t)fl * ld + r0 + fq, *pb0 = Pb + (size_t)fl * ld + c0 + fq;
    auto fetch = [&](int l0) {
        const float *src = pa0 + (size_t)l0 * ld;
        if (r0 + fq + 8 <= n) {
            const float4 v0 = *(const float4 *)src, v1 = *(const float4 *)(src + 4);
            ra[0] = v0.x; ra[1] = v0.y; ra[2] = v0.z; ra[3] = v0.w;
            ra[4] = v1.x; ra[5] = v1.y; ra[6] = v1.z; ra[7] = v1.w;
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) ra[u] = (r0 + fq + u < n) ? src[u] : 0.f;
        }
        if (tri) {
            const float *sb = pb0 + (size_t)l0 * ld;
            if (c0 + fq + 8 <= climit) {
                const float4 v0 = *(const float4 *)sb, v1 = *(const float4 *)(sb + 4);
                rb[0] = v0.x; rb[1] = v0.y; rb[2] = v0.z; rb[3] = v0.w;
                rb[4] = v1.x; rb[5] = v1.y; rb[6] = v1.z; rb[7] = v1.w;
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u) rb[u] = (c0 + fq + u < climit) ? sb[u] : 0.f;
            }
        } else if (c0 + xc < climit) {
            const float *sx = X + (size_t)(c0 + xc) * ld + k + l0 + xh * 8;
            const float4 v0 = *(const float4 *)sx, v1 = *(const float4 *)(sx + 4);
            rb[0] = v0.x; rb[1] = v0.y; rb[2] = v0.z; rb[3] = v0.w;
            rb[4] = v1.x; rb[5] = v1.y; rb[6] = v1.z; rb[7] = v1.w;
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) rb[u] = 0.f;
        }
    };
    auto stash = [&](int b) {
        *(float4 *)&As[b][fl][fq] = make_float4(ra[0], ra[1], ra[2], ra[3]);
        *(float4 *)&As[b][fl][fq + 4] = make_float4(ra[4], ra[5], ra[6], ra[7]);
        if (tri) {
            *(float4 *)&Bs[b][fl][fq] = make_float4(rb[0], rb[1], rb[2], rb[3]);
            *(float4 *)&Bs[b][fl][fq + 4] = make_float4(rb[4], rb[5], rb[6], rb[7]);
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) Bs[b][xh * 8 + u][xc] = rb[u];
        }
    };
    fetch(0);
    int buf = 0;
    for (int l0 = 0; l0 < kP; l0 += kKc) {
        stash(buf);
        __syncthreads();
        if (l0 + kKc < kP) fetch(l0 + kKc);
#pragma unroll
        for (int l = 0; l < kKc; ++l) {
            const float4 a0 = *(const float4 *)&As[buf][l][tr * 8], a1 = *(const float4 *)&As[buf][l][tr * 8 + 4];
            const float4 b0 = *(const float4 *)&Bs[buf][l][tc * 8], b1 = *(const float4 *)&Bs[buf][l][tc * 8 + 4];
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int w = 0; w < 8; ++w) acc[u][w] += a[u] * b[w];
        }
        buf ^= 1;
    }
    float *C = tri ? A : X;
    const bool full = r0 + kTile <= n && c0 + kTile <= climit && (!tri || r0 > c0);
    if (full) {
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            float *dst = C + (size_t)(c0 + tc * 8 + w) * ld + r0 + tr * 8;
            float4 v0 = *(float4 *)dst, v1 = *(float4 *)(dst + 4);
            v0.x -= acc[0][w]; v0.y -= acc[1][w]; v0.z -= acc[2][w]; v0.w -= acc[3][w];
            v1.x -= acc[4][w]; v1.y -= acc[5][w]; v1.z -= acc[6][w]; v1.w -= acc[7][w];
            *(float4 *)dst = v0;
            *(float4 *)(dst + 4) = v1;
        }
    } else {
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const int c = c0 + tc * 8 + w;
            if (c >= climit) continue;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int r = r0 + tr * 8 + u;
                if (r < n && (!tri || r > c)) C[(size_t)c * ld + r] -= acc[u][w];
            }
        }
    }
}

// ------------------------------------------------------------------ fused panel step (SIMT path)
// One launch per panel k (bs = 64, base = k + 64 < n) does what the next diagonal block waits for,
// so the panel-to-panel chain is two kernels (this one and the next diagonal block).  Its units are
// 64-row strips and 64-column blocks, each split over two CTAs (CTA 2 s + h takes half h of unit s),
// so that a CTA's dependent products are 2.5 instead of 4 64x64x64 ones and about 130 CTAs share the
// SMs instead of 65:
//   strip s (rows R = base + 64 s ..), half rows R_h = R[32 h, 32 h + 32): LD[R_h] = A21[R_h] L11^-T
//     and L21[R_h] = LD[R_h] D1^-1 (the panel), then the next panel's 64 columns A22[R_h, R0] -=
//     LD[R_h] L21[R0]^T (R0 = the next panel's rows; L21[R0] recomputed in every CTA from the
//     unscaled A21[R0]) together with the previous panel's update of the same columns, -= LD'[R_h]
//     L21'[R0]^T, and the fixed-order partial column sums below the next diagonal block (one row of
//     csum per half: row 2 s + h);
//   X block s - ts (columns C = 64 (s - ts) .. of block row k of L^-1), half columns C_h:
//     X[k, C_h] = L11^-1 B[k, C_h] (the block row), then X[R0, C_h] -= L21[R0] X[k, C_h] +
//     L21'[R0] X[k - 64, C_h] (the previous panel's part);
// L21[R0] goes to A with the next diagonal block's kernel (the other CTAs read A21[R0] unscaled).
// What remains of both updates (rows and columns from base + 128) is d32_update_kernel's (skip 2).
constexpr int kStepSmem = (5 * kP * kP + kP) * 4;
constexpr int kHalf = kP / 2;

// acc[u][w] += sum_l a[l][tr * 4 + u] b[l][tc * 4 + w] (64 x 64 operands, [depth][index])
__device__ __forceinline__ void mm64(const float *__restrict__ a, const float *__restrict__ b, float (&acc)[4][4],
                                     int tr, int tc) {
#pragma unroll 16
    for (int l = 0; l < kP; ++l) {
        const float4 x = *(const float4 *)(a + l * kP + tr * 4);
        const float4 y = *(const float4 *)(b + l * kP + tc * 4);
        const float av[4] = {x.x, x.y, x.z, x.w}, bv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[u][w] += av[u] * bv[w];
    }
}

// 32 x 64 outputs: acc[u][w] += sum_l a[l][tr * 2 + u] b[l][tc * 4 + w] (a's first 32 indices)
__device__ __forceinline__ void mm_r32(const float *__restrict__ a, const float *__restrict__ b, float (&acc)[2][4],
                                       int tr, int tc) {
#pragma unroll 16
    for (int l = 0; l < kP; ++l) {
        const float2 x = *(const float2 *)(a + l * kP + tr * 2);
        const float4 y = *(const float4 *)(b + l * kP + tc * 4);
        const float av[2] = {x.x, x.y}, bv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[u][w] += av[u] * bv[w];
    }
}

// 64 x 32 outputs: acc[u][w] += sum_l a[l][tr * 4 + u] b[l][tc * 2 + w] (b's first 32 indices)
__device__ __forceinline__ void mm_c32(const float *__restrict__ a, const float *__restrict__ b, float (&acc)[4][2],
                                       int tr, int tc) {
#pragma unroll 16
    for (int l = 0; l < kP; ++l) {
        const float4 x = *(const float4 *)(a + l * kP + tr * 4);
        const float2 y = *(const float2 *)(b + l * kP + tc * 2);
        const float av[4] = {x.x, x.y, x.z, x.w}, bv[2] = {y.x, y.y};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < 2; ++w) acc[u][w] += av[u] * bv[w];
    }
}

// tile[l][r] = G[(col0 + l) ld + row0 + r] for r < R and row0 + r < rlim, else 0 (row0 a multiple
// of 4; depth 64, tile stride 64)
template <int R>
__device__ __forceinline__ void load_cm(float *__restrict__ tile, const float *__restrict__ G, int ld, int col0,
                                        int row0, int rlim) {
    for (int t = threadIdx.x; t < kP * (R / 4); t += blockDim.x) {
        const int l = t / (R / 4), q = (t % (R / 4)) * 4;
        const float *src = G + (size_t)(col0 + l) * ld + row0 + q;
        float4 v;
        if (row0 + q + 4 <= rlim) v = *(const float4 *)src;
        else {
            v.x = row0 + q < rlim ? src[0] : 0.f;
            v.y = row0 + q + 1 < rlim ? src[1] : 0.f;
            v.z = row0 + q + 2 < rlim ? src[2] : 0.f;
            v.w = row0 + q + 3 < rlim ? src[3] : 0.f;
        }
        *(float4 *)(tile + l * kP + q) = v;
    }
}

// tile[l][c] = X(row0 + l, c0 + c) = X[(c0 + c) ld + row0 + l] for c < C and c0 + c < climit, else
// 0 (depth 64, tile stride 64)
template <int C>
__device__ __forceinline__ void load_rows_of_x(float *__restrict__ tile, const float *__restrict__ X, int ld,
                                               int row0, int c0, int climit) {
    for (int t = threadIdx.x; t < C * (kP / 4); t += blockDim.x) {
        const int c = t % C, lq = (t / C) * 4;
        float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c0 + c < climit) w = *(const float4 *)(X + (size_t)(c0 + c) * ld + row0 + lq);
        tile[(lq + 0) * kP + c] = w.x;
        tile[(lq + 1) * kP + c] = w.y;
        tile[(lq + 2) * kP + c] = w.z;
        tile[(lq + 3) * kP + c] = w.w;
    }
}

__global__ void __launch_bounds__(kTT)
d32_step_kernel(int n, int ld, int k, float *__restrict__ A, float *__restrict__ X,
                const float *__restrict__ D, const float *__restrict__ Linv, float *__restrict__ LDc,
                const float *__restrict__ LDprev, float *__restrict__ L0buf, float *__restrict__ csum) {
    extern __shared__ __align__(16) float sm[];
    float *Lt = sm, *T1 = sm + kP * kP, *T2 = sm + 2 * kP * kP, *T3 = sm + 3 * kP * kP, *T4 = sm + 4 * kP * kP;
    float *idv = sm + 5 * kP * kP;
    const int base = k + kP;
    const int ts = (n - base + kP - 1) / kP;
    const int unit = (int)blockIdx.x >> 1, h = (int)blockIdx.x & 1;
    const bool strip = unit < ts;
    const bool prev = k > 0;
    const int tr = threadIdx.x & 15, tc = threadIdx.x >> 4;
    // Lt[l][j] = (L11^-1)_jl; idv = D1^+ (0 for grounded pivots)
    for (int t = threadIdx.x; t < kP * kP; t += blockDim.x) {
        const int j = t % kP, l = t / kP;
        Lt[l * kP + j] = Linv[(size_t)l * ld + (k + j)];
    }
    if (threadIdx.x < kP) {
        const float dj = D[k + threadIdx.x];
        idv[threadIdx.x] = isinf(dj) ? 0.f : 1.f / dj;
    }
    if (strip) {
        const int rb = unit, rh = base + rb * kP + h * kHalf;   // this half's first row
        float acc[2][4], acc2[4][4], acc3[2][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                acc2[u][w] = 0.f;
                if (u < 2) acc[u][w] = acc3[u][w] = 0.f;
            }
        // the A22[R_h, R0] entries this thread updates, loaded with the operands (no other CTA of
        // this launch, and no rest-update running beside it, writes them)
        float cur[2][4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int c = base + tc * 4 + w;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int r = rh + tr * 2 + u;
                cur[u][w] = (c < n && r < n && r > c) ? A[(size_t)c * ld + r] : 0.f;
            }
        }
        if (rb > 0) load_cm<kHalf>(T1, A, ld, k, rh, n);       // A21[R_h]     [l][r], r < 32
        load_cm<kP>(T2, A, ld, k, base, n);                     // A21[R0]      [l][c]
        if (prev) {
            load_cm<kHalf>(T3, LDprev, ld, 0, rh, n);           // LD'[R_h]     [j][r]
            load_cm<kP>(T4, A, ld, k - kP, base, n);            // L21'[R0]     [j][c]
        }
        __syncthreads();
        // LD(R_h row tr*2+u, j = tc*4+w) (the first strip's rows are R0's: read from T2)
        mm_r32(rb > 0 ? T1 : T2 + h * kHalf, Lt, acc, tr, tc);
        mm64(T2, Lt, acc2, tr, tc);                             // LD(R0 row tr*4+u, j = tc*4+w)
        __syncthreads();
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int j = tc * 4 + w;
            const float id = idv[j];
            const bool inf = id == 0.f;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int rr = tr * 2 + u, r = rh + rr;
                const float ldv = inf ? 0.f : acc[u][w];
                if (r < n) {
                    LDc[(size_t)j * ld + r] = ldv;
                    if (rb == 0) L0buf[j * kP + h * kHalf + rr] = acc[u][w] * id;
                    else A[(size_t)(k + j) * ld + r] = acc[u][w] * id;
                }
                T1[j * kP + rr] = ldv;                                      // A operand [j][r]
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) T2[j * kP + tr * 4 + u] = acc2[u][w] * id;   // B operand [j][c]
        }
        __syncthreads();
        mm_r32(T1, T2, acc3, tr, tc);
        if (prev) mm_r32(T3, T4, acc3, tr, tc);
        // A22[R_h, R0] -= acc3 below the diagonal; column sums of the rows below the next block
        float cs[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int c = base + tc * 4 + w;
            if (c >= n) continue;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int r = rh + tr * 2 + u;
                if (r < n && r > c) {
                    const float v = cur[u][w] - acc3[u][w];
                    A[(size_t)c * ld + r] = v;
                    if (r >= base + kP) cs[w] += v;
                }
            }
        }
        // the 16 threads with this tc are one half-warp (lanes tr = 0..15)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            float v = cs[w];
#pragma unroll
            for (int o = 1; o < 16; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (tr == 0) csum[(size_t)(2 * rb + h) * kP + tc * 4 + w] = v;
        }
    } else {
        const int cb = unit - ts, c0 = cb * kP, ch = c0 + h * kHalf;   // this half's first column
        const bool before = c0 < k;                           // columns left of the diagonal block
        float acc[4][2], acc2[4][4], acc3[4][2];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                acc2[u][w] = 0.f;
                if (w < 2) acc[u][w] = acc3[u][w] = 0.f;
            }
        // the X[R0, C_h] entries this thread updates, loaded with the operands
        float cur[4][2];
#pragma unroll
        for (int w = 0; w < 2; ++w)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int r = base + tr * 4 + u;
                cur[u][w] = r < n ? X[(size_t)(ch + tc * 2 + w) * ld + r] : 0.f;
            }
        if (before) load_rows_of_x<kHalf>(T1, X, ld, k, ch, k);     // B[k, C_h]      [l][c], c < 32
        load_cm<kP>(T2, A, ld, k, base, n);                          // A21[R0]        [l][r]
        if (prev && before) {
            load_cm<kP>(T3, A, ld, k - kP, base, n);                 // L21'[R0]       [j][r]
            load_rows_of_x<kHalf>(T4, X, ld, k - kP, ch, k);         // X[k - 64, C_h] [j][c]
        }
        __syncthreads();
        if (before) mm_c32(Lt, T1, acc, tr, tc);              // X(k + i, c), i = tr*4+u, c = tc*2+w
        mm64(T2, Lt, acc2, tr, tc);                           // LD(R0_r, j), r = tr*4+u, j = tc*4+w
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int w = 0; w < 2; ++w) {
                const int i = tr * 4 + u, c = tc * 2 + w;
                const float x = before ? acc[u][w] : Lt[(h * kHalf + c) * kP + i];
                X[(size_t)(ch + c) * ld + (k + i)] = x;
                T1[i * kP + c] = x;                                          // B operand [i][c]
            }
#pragma unroll
            for (int w = 0; w < 4; ++w)
                T2[(tc * 4 + w) * kP + tr * 4 + u] = acc2[u][w] * idv[tc * 4 + w];  // A operand [j][r]
        }
        __syncthreads();
        mm_c32(T2, T1, acc3, tr, tc);
        if (prev && before) mm_c32(T3, T4, acc3, tr, tc);
#pragma unroll
        for (int w = 0; w < 2; ++w) {
            const int c = ch + tc * 2 + w;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int r = base + tr * 4 + u;
                if (r < n) X[(size_t)c * ld + r] = cur[u][w] - acc3[u][w];
            }
        }
    }
}

// ------------------------------------------------------------------ tensor-core bulk update
// The bulk update C -= A_op B_op^T (depth 64, one panel) on the fifth-generation tensor cores in
// split TF32: a = a_hi + a_lo with a_hi the TF32 rounding of a, and C -= a_hi b_hi + a_hi b_lo +
// a_lo b_hi (the a_lo b_lo term is below FP32 rounding), accumulated in FP32 in tensor memory.
// Once per panel the operands are split and written in the MMA's shared-memory layout (K-major,
// no swizzle: 8-row x 16-byte core matrices; core matrix (row / 8, k / 4) of an R-row block at
// byte ((k / 4) (R / 8) + row / 8) 128, its row (row % 8) at 16-byte steps), so a tile fetches its
// operands with four bulk copies completing on one mbarrier, one thread issues 3 x 8 MMAs
// (M = 128, N = 64, K = 8 each), and all four warps read the accumulator back (each warp its 32
// lanes) and subtract it from C.  Every wait is bounded: a wait that gives up records the failure
// in *err, waits once more for its own copies or MMAs, releases the tensor memory and returns.
constexpr int kTcM = 128, kTcN = 256;                 // tile rows, tile columns
constexpr int kTcApiece = kTcM * kP * 4;              // one A piece (hi or lo): 32 KB
constexpr int kTcBpiece = kTcN * kP * 4;              // one B piece: 64 KB
constexpr int kTcSmem = 2 * kTcApiece + 2 * kTcBpiece + 64;
constexpr int kTcThreads = 160;   // four epilogue warps and one producer warp
constexpr int kTcAutoN = 8192;    // tc_mode 0: the tensor-core update from this n on
__device__ __forceinline__ float tc_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// kind::tf32 instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = 256
constexpr uint32_t kTcIdesc = tc_idesc(2u, kTcM, kTcN);

// Rows [row0 + b RB, +RB) of an operand, depth 64, split into TF32 hi / lo pieces in the layout
// above: piece (b, hi) at out + 2 b P, (b, lo) at out + (2 b + 1) P (P = RB * 64 floats).  The
// element (row r, depth l) is src[l * ld + r] (a column-major panel) or, kmaj, src[r * ld + l]
// (rows of L^-1 held by column); rows at or beyond `rows` are zero.
template <int RB, bool KMAJ>
__global__ void __launch_bounds__(kTT)
d32_tc_split_kernel(int rows, int ld, const float *__restrict__ src, int row0, float *__restrict__ out) {
    const int b = blockIdx.x;
    float *hi = out + (size_t)(2 * b) * RB * kP, *lo = hi + (size_t)RB * kP;
    for (int t = threadIdx.x; t < RB * (kP / 4); t += blockDim.x) {
        const int r = t % RB, kq = t / RB;
        const int row = row0 + b * RB + r;
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int l = kq * 4 + q;
            v[q] = row < rows ? (KMAJ ? src[(size_t)row * ld + l] : src[(size_t)l * ld + row]) : 0.f;
        }
        float h[4], w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            h[q] = tc_tf32(v[q]);
            w[q] = v[q] - h[q];
        }
        const size_t off = ((size_t)kq * (RB / 8) + (r >> 3)) * 32 + (size_t)(r & 7) * 4;  // in floats
        *(float4 *)(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
        *(float4 *)(lo + off) = make_float4(w[0], w[1], w[2], w[3]);
    }
}

// Tile t of one panel's bulk update: tiles [0, T TJ) are the trailing triangle from base2 (row
// tile ti of 128, column tile tj of 256; only those that start left of the row tile's last row),
// then T x tcx tiles of the rows of L^-1 (C = X, columns below base).  False: nothing to do.
__device__ __forceinline__ bool tc_tile(int t, int n, int base, int base2, int T, int TJ, int tcx, bool &tri, int &ti,
                                        int &tj, int &r0, int &c0, int &climit) {
    const int ntri = T * TJ;
    tri = t < ntri;
    if (tri) {
        ti = t / TJ;
        tj = t % TJ;
        if (tj * kTcN >= (ti + 1) * kTcM) return false;
    } else {
        ti = (t - ntri) / tcx;
        tj = (t - ntri) % tcx;
    }
    r0 = base2 + ti * kTcM;
    c0 = tri ? base2 + tj * kTcN : tj * kTcN;
    climit = tri ? n : base;
    return r0 < n && c0 < climit;
}

__device__ __forceinline__ int tc_next(int t, int step, int ntiles, int n, int base, int base2, int T, int TJ,
                                       int tcx) {
    bool tri;
    int ti, tj, r0, c0, cl;
    while (t < ntiles && !tc_tile(t, n, base, base2, T, TJ, tcx, tri, ti, tj, r0, c0, cl)) t += step;
    return t;
}

// Persistent CTAs (one per SM), each taking tiles gridDim.x apart, warp-specialised: warp 4 (one
// lane) brings each tile's four operand pieces with two bulk copies on an mbarrier and issues its
// 3 x 8 MMAs into one of two tensor-memory accumulators, committing them to that accumulator's
// "full" mbarrier; warps 0-3 (tensor-memory lanes 0-127) wait for it, subtract the accumulator
// from C and arrive on its "empty" mbarrier.  So tile i + 1's copies and MMAs run while tile i's
// epilogue does; the single operand stage is refilled once tile i's MMAs are done.  Every wait
// is bounded: one that gives up records the failure in *err and the CTA winds down (its own
// copies and MMAs waited for once more) before it releases the tensor memory.  Operand pieces:
// trailing A = split L D rows, B = split panel rows (256-row blocks); inverse A = split panel rows
// (128-row blocks), B = split rows of L^-1.
constexpr int kTcWarps = 5;

__global__ void __launch_bounds__(kTcWarps * 32, 1)
d32_tc_update_kernel(int n, int ld, int base, int base2, int T, const float *__restrict__ LDs,
                     const float *__restrict__ PBs, const float *__restrict__ PAs, const float *__restrict__ XBs,
                     float *__restrict__ A, float *__restrict__ X, int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int TJ = (int)ceil_div(T * kTcM, kTcN), tcx = (int)ceil_div(base, kTcN);
    const int ntiles = T * TJ + T * tcx, step = (int)gridDim.x;
    const int first = tc_next((int)blockIdx.x, step, ntiles, n, base, base2, T, TJ, tcx);
    if (first >= ntiles) return;   // no tile for this CTA: uniform, nothing started
    uint64_t *mbs = (uint64_t *)(smem + 2 * kTcApiece + 2 * kTcBpiece);
    // [0] load, [1..2] full (per accumulator), [3..4] empty (per accumulator)
    uint32_t *tslot = (uint32_t *)(mbs + 5);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(tc_smem_u32(tslot)), "r"(2 * kTcN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    const uint32_t mbl = tc_smem_u32(mbs), sbase = tc_smem_u32(smem);
    const uint32_t mfull[2] = {tc_smem_u32(mbs + 1), tc_smem_u32(mbs + 2)};
    const uint32_t mempty[2] = {tc_smem_u32(mbs + 3), tc_smem_u32(mbs + 4)};
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbl) : "memory");
        for (int q = 0; q < 2; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mfull[q]) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" :: "r"(mempty[q]) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    if (warp == 4) {
        if (lane == 0) {
            int i = 0, failed = 0;
            for (int t = first; t < ntiles && !failed; t = tc_next(t + step, step, ntiles, n, base, base2, T, TJ, tcx), ++i) {
                const int bsel = i & 1;
                // the stage is free once the previous tile's MMAs are done
                if (i >= 1 && !tc_wait(mfull[(i - 1) & 1], (uint32_t)(((i - 1) >> 1) & 1))) { failed = 1; break; }
                bool tri;
                int ti, tj, r0, c0, cl;
                tc_tile(t, n, base, base2, T, TJ, tcx, tri, ti, tj, r0, c0, cl);
                const float *pa = (tri ? LDs : PAs) + (size_t)(2 * ti) * kTcM * kP;
                const float *pb = (tri ? PBs : XBs) + (size_t)(2 * tj) * kTcN * kP;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                             :: "r"(mbl), "r"((uint32_t)(2 * kTcApiece + 2 * kTcBpiece)) : "memory");
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             :: "r"(sbase), "l"(pa), "r"((uint32_t)(2 * kTcApiece)), "r"(mbl) : "memory");
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             :: "r"(sbase + 2 * kTcApiece), "l"(pb), "r"((uint32_t)(2 * kTcBpiece)), "r"(mbl) : "memory");
                if (!tc_wait(mbl, (uint32_t)(i & 1))) {
                    failed = 1;
                    tc_wait(mbl, (uint32_t)(i & 1));   // the copies target this CTA's shared memory
                    break;
                }
                // the accumulator is free once the epilogue of tile i - 2 is done
                if (i >= 2 && !tc_wait(mempty[bsel], (uint32_t)(((i - 2) >> 1) & 1))) { failed = 1; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc = tmem + (uint32_t)(bsel * kTcN);
                const uint32_t ah = sbase, al = sbase + kTcApiece;
                const uint32_t bh = sbase + 2 * kTcApiece, bl = bh + kTcBpiece;
                const uint32_t lboA = (kTcM / 8) * 128, lboB = (kTcN / 8) * 128;
#pragma unroll
                for (int ks = 0; ks < kP / 8; ++ks) {
                    const uint32_t ka = (uint32_t)ks * 2 * lboA, kb = (uint32_t)ks * 2 * lboB;
                    const uint64_t dah = tc_desc(ah + ka, lboA), dal = tc_desc(al + ka, lboA);
                    const uint64_t dbh = tc_desc(bh + kb, lboB), dbl = tc_desc(bl + kb, lboB);
                    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                                 :: "r"(acc), "l"(dah), "l"(dbh), "r"(kTcIdesc), "r"(ks > 0 ? 1u : 0u) : "memory");
                    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                                 :: "r"(acc), "l"(dah), "l"(dbl), "r"(kTcIdesc), "r"(1u) : "memory");
                    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                                 :: "r"(acc), "l"(dal), "l"(dbh), "r"(kTcIdesc), "r"(1u) : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(mfull[bsel]) : "memory");
            }
            if (failed) atomicExch(err, 1);
            // before the CTA ends: the last MMAs issued must be complete (bounded)
            if (i >= 1) tc_wait(mfull[(i - 1) & 1], (uint32_t)(((i - 1) >> 1) & 1));
        }
    } else {
        // epilogue warps: warp w owns tensor-memory lanes (tile rows) 32 w .. 32 w + 31
        int i = 0;
        for (int t = first; t < ntiles; t = tc_next(t + step, step, ntiles, n, base, base2, T, TJ, tcx), ++i) {
            const int bsel = i & 1;
            bool tri;
            int ti, tj, r0, c0, climit;
            tc_tile(t, n, base, base2, T, TJ, tcx, tri, ti, tj, r0, c0, climit);
            float *C = tri ? A : X;
            const int r = r0 + warp * 32 + lane;
            float cv[2][32];
            auto load_part = [&](float (&dst)[32], int part) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int c = c0 + part * 32 + j;
                    dst[j] = (r < n && c < climit && (!tri || r > c)) ? C[(size_t)c * ld + r] : 0.f;
                }
            };
            load_part(cv[0], 0);   // while the MMAs run
            if (!tc_wait(mfull[bsel], (uint32_t)((i >> 1) & 1))) {
                if (lane == 0) atomicExch(err, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t accrow = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(bsel * kTcN);
#pragma unroll 2
            for (int part = 0; part < kTcN / 32; ++part) {
                if (part + 1 < kTcN / 32) load_part(cv[(part + 1) & 1], part + 1);
                uint32_t v[32];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                    "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                    "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                      "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                      "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(accrow + (uint32_t)(part * 32)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (r < n) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int c = c0 + part * 32 + j;
                        if (c < climit && (!tri || r > c)) C[(size_t)c * ld + r] = cv[part & 1][j] - __uint_as_float(v[j]);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) tc_arrive(mempty[bsel]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(2 * kTcN) : "memory");
}

// partial sums of y = X r: CTA (rb, cb) covers rows [rb*256, +256) (four per thread, float4 loads)
// and columns [cb*64, +64) for the lower-triangle tiles only (rows beyond n read the zero padding);
// the tile's 64 columns are split over four thread groups of 16 columns, reduced in shared memory
constexpr int kFr = 256, kFc = 64;
__global__ void __launch_bounds__(kFr)
d32_fwd_kernel(int n, int ld, int ncb, const float *__restrict__ X, const double *__restrict__ r,
               float *__restrict__ part) {
    __shared__ float rs[kFc];
    __shared__ float4 red[3][kFr / 4];
    // tile index -> (rb, cb) with cb*kFc < (rb+1)*kFr
    const int per = kFr / kFc;
    int idx = blockIdx.x, rb = 0;
    while (idx >= min(ncb, (rb + 1) * per)) { idx -= min(ncb, (rb + 1) * per); ++rb; }
    const int cb = idx;
    const int rq = threadIdx.x & (kFr / 4 - 1), cg = threadIdx.x / (kFr / 4);
    const int c0 = cb * kFc, i = rb * kFr + rq * 4;
    if (threadIdx.x < kFc) rs[threadIdx.x] = c0 + (int)threadIdx.x < n ? (float)r[c0 + threadIdx.x] : 0.f;
    __syncthreads();
    const bool live = i < n && i + 3 >= c0;
    const int jn = min(kFc, n - c0);
    const int jlo = cg * (kFc / 4), jhi = min(jlo + kFc / 4, jn);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (live) {
        const float *col = X + (size_t)c0 * ld + i;
        if (i >= c0 + kFc - 1) {
#pragma unroll 16
            for (int jj = jlo; jj < jhi; ++jj) {
                const float4 v = *(const float4 *)(col + (size_t)jj * ld);
                const float rj = rs[jj];
                acc.x += v.x * rj; acc.y += v.y * rj; acc.z += v.z * rj; acc.w += v.w * rj;
            }
        } else {
            for (int jj = jlo; jj < jhi; ++jj) {
                const int j = c0 + jj;
                const float4 v = *(const float4 *)(col + (size_t)jj * ld);
                const float rj = rs[jj];
                if (j <= i) acc.x += v.x * rj;
                if (j <= i + 1) acc.y += v.y * rj;
                if (j <= i + 2) acc.z += v.z * rj;
                if (j <= i + 3) acc.w += v.w * rj;
            }
        }
    }
    if (cg > 0) red[cg - 1][rq] = acc;
    __syncthreads();
    if (cg == 0 && live) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float4 o = red[q][rq];
            acc.x += o.x; acc.y += o.y; acc.z += o.z; acc.w += o.w;
        }
        *(float4 *)(part + (size_t)cb * ld + i) = acc;
    }
}

// w = D^+ y, y_i = sum of the partials of row i (fixed order)
__global__ void d32_mid_kernel(int n, int ld, const float *__restrict__ part, const float *__restrict__ D,
                               float *__restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int last = i / kFc;
    float y = 0.f;
    for (int cb = 0; cb <= last; ++cb) y += part[(size_t)cb * ld + i];
    const float d = D[i];
    w[i] = isinf(d) ? 0.f : y / d;
}

// z_j = sum_{i >= j} X_ij w_i, one warp per column, float4 per lane
__global__ void __launch_bounds__(kTT)
d32_bwd_kernel(int n, int ld, const float *__restrict__ X, const float *__restrict__ w, double *__restrict__ z) {
    const int j = blockIdx.x * (kTT / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j >= n) return;
    const float *col = X + (size_t)j * ld;
    float acc = 0.f;
    const int i0 = j & ~3;
#pragma unroll 4
    for (int i = i0 + lane * 4; i < n; i += 128) {
        const float4 v = *(const float4 *)(col + i);
        if (i >= j && i + 3 < n) {
            acc += v.x * w[i] + v.y * w[i + 1] + v.z * w[i + 2] + v.w * w[i + 3];
        } else {
            if (i >= j && i < n) acc += v.x * w[i];
            if (i + 1 >= j && i + 1 < n) acc += v.y * w[i + 1];
            if (i + 2 >= j && i + 2 < n) acc += v.z * w[i + 2];
            if (i + 3 >= j && i + 3 < n) acc += v.w * w[i + 3];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) z[j] = (double)acc;
}

}  // namespace

Error d32_alloc(Dense32 &F, int32_t n) {
    F.n = n;
    F.ld = (n + 31) / 32 * 32;
    const size_t big = sizeof(float) * (size_t)F.ld * n;
    OT_CUDA(cudaMalloc((void **)&F.A, big));
    OT_CUDA(cudaMalloc((void **)&F.X, big));
    OT_CUDA(cudaMalloc((void **)&F.LD, 3 * sizeof(float) * (size_t)F.ld * kP));
    OT_CUDA(cudaMalloc((void **)&F.Linv, sizeof(float) * (size_t)F.ld * kP));
    OT_CUDA(cudaMalloc((void **)&F.D, sizeof(float) * n));
    OT_CUDA(cudaMalloc((void **)&F.d0, sizeof(float) * n));
    // partial column sums: up to two rows (one per half strip) per 64-row strip
    OT_CUDA(cudaMalloc((void **)&F.csum, sizeof(float) * 2 * kP * (size_t)ceil_div(n, kP)));
    OT_CUDA(cudaMalloc((void **)&F.L0, sizeof(float) * kP * kP));
    OT_CUDA(cudaMalloc((void **)&F.w, sizeof(float) * n));
    OT_CUDA(cudaMalloc((void **)&F.part, sizeof(float) * (size_t)F.ld * (size_t)ceil_div(n, kFc)));
    // lower bound of the unwritten upper parts, so that nothing uninitialised is ever read
    OT_CUDA(cudaMemset(F.A, 0, big));
    OT_CUDA(cudaMemset(F.LD, 0, 3 * sizeof(float) * (size_t)F.ld * kP));
    OT_CUDA(cudaMemset(F.Linv, 0, sizeof(float) * (size_t)F.ld * kP));
    // one process-wide limit, the largest any n of this path needs (a per-n value set by one
    // handle could undercut another handle's launch on another thread)
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(d32_assemble_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(sizeof(unsigned long long) * kSlice));
        if (attr_err == cudaSuccess)
            attr_err = cudaFuncSetAttribute(d32_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kStepSmem);
    });
    if (attr_err != cudaSuccess) return fail(OT_ERR_CUDA, cudaGetErrorString(attr_err));
    if (n > kMaxN) return fail(OT_ERR_ARG, "dense32: n above the supported size");
    return ok();
}

void d32_free(Dense32 &F) {
    if (F.graph) cudaGraphExecDestroy(F.graph);
    for (void *p : {(void *)F.A, (void *)F.X, (void *)F.LD, (void *)F.Linv, (void *)F.D, (void *)F.d0, (void *)F.csum,
                    (void *)F.L0, (void *)F.w, (void *)F.part, (void *)F.tc, (void *)F.tc_err})
        if (p) cudaFree(p);
    if (F.tc_err_host) cudaFreeHost(F.tc_err_host);
    F = Dense32();
}

Error d32_assemble(Dense32 &F, const Newton &W, const Support &S, cudaStream_t st) {
    const int n = F.n;
    const int slices = (int)ceil_div(n, kSlice);
    const size_t smem = sizeof(unsigned long long) * std::min(n, kSlice);
    if (slices == 1) {
        d32_assemble_kernel<<<n, kTT, smem, st>>>(n, F.ld, S.col_ptr, S.col_row, W.theta_col, S.row_ptr, S.j,
                                                   W.theta, W.Minv, W.N, F.A, F.d0, nullptr);
        OT_LAUNCHED();
        return ok();
    }
    DevTemp<unsigned long long> tot;
    OT_TRY(tot.alloc(n, st));
    OT_CUDA(cudaMemsetAsync(tot.p, 0, sizeof(unsigned long long) * n, st));
    d32_assemble_kernel<<<dim3(n, slices), kTT, smem, st>>>(n, F.ld, S.col_ptr, S.col_row, W.theta_col, S.row_ptr,
                                                             S.j, W.theta, W.Minv, W.N, F.A, F.d0, tot.p);
    OT_LAUNCHED();
    d32_diag_total_kernel<<<(unsigned)ceil_div(n, kTT), kTT, 0, st>>>(n, W.N, tot.p, F.d0);
    OT_LAUNCHED();
    return ok();
}

// The factorisation's launch sequence for this n as an explicit CUDA graph: a chain of kernel
// nodes built with the graph API (no stream capture, so nothing another host thread does, such as
// a device-synchronising cudaFree, can invalidate it).
namespace {
struct Dag {
    cudaGraph_t g = nullptr;
    int64_t nodes = 0;
    cudaError_t err = cudaSuccess;
    template <typename... Args>
    cudaGraphNode_t kernel(std::vector<cudaGraphNode_t> deps, void (*fn)(Args...), unsigned grid, unsigned block,
                           Args... args) {
        cudaGraphNode_t node = nullptr;
        if (err != cudaSuccess) return node;
        void *ptrs[] = {(void *)&args...};
        cudaKernelNodeParams kp = {};
        kp.func = (void *)fn;
        kp.gridDim = dim3(grid);
        kp.blockDim = dim3(block);
        kp.sharedMemBytes = 0;
        kp.kernelParams = ptrs;
        kp.extra = nullptr;
        deps.erase(std::remove(deps.begin(), deps.end(), nullptr), deps.end());
        err = cudaGraphAddKernelNode(&node, g, deps.data(), deps.size(), &kp);
        if (err == cudaSuccess) ++nodes;
        return node;
    }
    // launch priority of a kernel node (stream-priority scale: lower values run first)
    void priority(cudaGraphNode_t node, int value) {
        if (err != cudaSuccess || !node) return;
        cudaKernelNodeAttrValue v = {};
        v.priority = value;
        err = cudaGraphKernelNodeSetAttribute(node, cudaKernelNodeAttributePriority, &v);
    }
    template <typename... Args>
    cudaGraphNode_t kernel_smem(std::vector<cudaGraphNode_t> deps, void (*fn)(Args...), unsigned grid,
                                unsigned block, unsigned smem, Args... args) {
        cudaGraphNode_t node = nullptr;
        if (err != cudaSuccess) return node;
        void *ptrs[] = {(void *)&args...};
        cudaKernelNodeParams kp = {};
        kp.func = (void *)fn;
        kp.gridDim = dim3(grid);
        kp.blockDim = dim3(block);
        kp.sharedMemBytes = smem;
        kp.kernelParams = ptrs;
        kp.extra = nullptr;
        deps.erase(std::remove(deps.begin(), deps.end(), nullptr), deps.end());
        err = cudaGraphAddKernelNode(&node, g, deps.data(), deps.size(), &kp);
        if (err == cudaSuccess) ++nodes;
        return node;
    }
    cudaGraphNode_t memset0(float *dst, size_t count, std::vector<cudaGraphNode_t> deps) {
        cudaGraphNode_t node = nullptr;
        if (err != cudaSuccess) return node;
        cudaMemsetParams mp = {};
        mp.dst = dst;
        mp.value = 0;
        mp.elementSize = sizeof(float);
        mp.width = count;
        mp.height = 1;
        mp.pitch = 0;
        err = cudaGraphAddMemsetNode(&node, g, deps.data(), deps.size(), &mp);
        if (err == cudaSuccess) ++nodes;
        return node;
    }
    cudaGraphNode_t join(std::vector<cudaGraphNode_t> deps) {
        cudaGraphNode_t node = nullptr;
        if (err != cudaSuccess) return node;
        deps.erase(std::remove(deps.begin(), deps.end(), nullptr), deps.end());
        err = cudaGraphAddEmptyNode(&node, g, deps.data(), deps.size());
        return node;
    }
};
}  // namespace

// split operand storage for one panel parity: two 128-row-block operands and two 64-row-block ones
static size_t tc_a_floats(int n) { return (size_t)ceil_div(n, kTcM) * 2 * kTcM * kP; }
static size_t tc_b_floats(int n) { return (size_t)ceil_div(n, kTcN) * 2 * kTcN * kP; }
static size_t tc_per_parity(int n) { return 2 * tc_a_floats(n) + 2 * tc_b_floats(n); }
static Error d32_build(Dense32 &F, float eps, cudaGraph_t g, int64_t *nodes) {
    const int n = F.n, ld = F.ld;
    Dag c;
    c.g = g;
    cudaGraphNode_t prev = c.memset0(F.X, (size_t)ld * n, {});
    int lo_prio = 0, hi_prio = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio) != cudaSuccess) lo_prio = hi_prio = 0;
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 1;
    if (!F.use_tc) {
        // SIMT: the first diagonal block, then one fused step per panel (which also factors the next
        // diagonal block) on the chain, the rest of each panel's update (from base + 128) beside
        // it.  The step of panel p waits for the rest-update of panel p - 2 (which covered its
        // columns); the rest-updates run in order.  Three LD buffers: the rest-update of panel p
        // still reads its own while the steps of p + 1 and p + 2 write theirs.
        const int bs0 = std::min(kP, n);
        prev = c.kernel({prev}, d32_colsum_kernel, (unsigned)bs0, kTT, n, ld, bs0, (const float *)F.A, F.csum);
        cudaGraphNode_t chain = c.kernel({prev}, d32_diag_kernel, 1u, kTT, ld, 0, bs0, F.A, F.D, (const float *)F.d0,
                                         (const float *)F.csum, 1, 1, eps, F.Linv, (const float *)nullptr);
        c.priority(chain, hi_prio);
        cudaGraphNode_t rest1 = nullptr, rest2 = nullptr;   // rest-updates of panels p - 1 and p - 2
        int k = 0, p = 0;
        for (; k + kP < n; k += kP, ++p) {
            const int base = k + kP;
            const int ts = (int)ceil_div(n - base, kP), tx = (int)ceil_div(base, kP);
            float *LDc = F.LD + (size_t)(p % 3) * ld * kP;
            const float *LDprev = F.LD + (size_t)((p + 2) % 3) * ld * kP;
            const cudaGraphNode_t sn =
                c.kernel_smem({chain, rest2}, d32_step_kernel, (unsigned)(2 * (ts + tx)), kTT, (unsigned)kStepSmem, n, ld,
                              k, F.A, F.X, (const float *)F.D, (const float *)F.Linv, LDc, LDprev, F.L0, F.csum);
            c.priority(sn, hi_prio);
            const cudaGraphNode_t dn =
                c.kernel({sn}, d32_diag_kernel, 1u, kTT, ld, base, std::min(kP, n - base), F.A, F.D,
                         (const float *)F.d0, (const float *)F.csum, ts, 2, eps, F.Linv, (const float *)F.L0);
            c.priority(dn, hi_prio);
            const int b2 = base + 2 * kP;
            const int t2 = b2 < n ? (int)ceil_div(n - b2, kTile) : 0, tcn = (int)ceil_div(base, kTile);
            const int n2 = t2 * (t2 + 1) / 2 + t2 * tcn;
            cudaGraphNode_t rest = nullptr;
            if (n2 > 0) {
                rest = c.kernel({sn, rest1}, d32_update_kernel, (unsigned)n2, kTT, n, ld, k, 2, F.A, F.X,
                                (const float *)LDc);
                c.priority(rest, lo_prio);
            } else {
                rest = c.join({sn, rest1});
            }
            rest2 = rest1;
            rest1 = rest;
            chain = dn;
        }
        // the last panel: its diagonal block came with the last step (or is the first block); its
        // block row of L^-1, then the end of the graph after all writes
        const int bs = n - k;
        const cudaGraphNode_t ir = c.kernel({chain}, d32_invrow_kernel, (unsigned)ceil_div(n, kP), kTT, ld, k, bs,
                                            F.X, (const float *)F.Linv);
        c.priority(ir, hi_prio);
        prev = c.join({ir, rest1, rest2});
    } else {
    // tensor cores: per panel diag -> panel / invrow -> first update part (the next panel's block) on
    // the chain, the bulk update of the rest beside it (the next panel's first part waits for it)
    cudaGraphNode_t u1 = nullptr, u2 = nullptr;
    int np = 1;  // partial column sums feeding the next diagonal block
    for (int k = 0, p = 0; k < n; k += kP, ++p) {
        const int bs = std::min(kP, n - k), base = k + bs;
        float *LDp = F.LD + (size_t)(p % 3) * ld * kP;
        if (k == 0) prev = c.kernel({prev}, d32_colsum_kernel, (unsigned)bs, kTT, n, ld, bs, (const float *)F.A, F.csum);
        const cudaGraphNode_t dg = c.kernel({k == 0 ? prev : u1}, d32_diag_kernel, 1u, kTT, ld, k, bs, F.A, F.D,
                                            (const float *)F.d0, (const float *)F.csum, np, 1, eps, F.Linv,
                                            (const float *)nullptr);
        c.priority(dg, hi_prio);
        std::vector<cudaGraphNode_t> ready;
        if (base < n)
            ready.push_back(c.kernel({dg}, d32_panel_kernel, (unsigned)ceil_div(n - base, kP), kTT, n, ld, k, F.A,
                                     (const float *)F.D, (const float *)F.Linv, LDp));
        ready.push_back(c.kernel({dg}, d32_invrow_kernel, (unsigned)ceil_div(base, kP), kTT, ld, k, bs, F.X,
                                 (const float *)F.Linv));
        for (cudaGraphNode_t r : ready) c.priority(r, hi_prio);
        if (u2) ready.push_back(u2);
        if (base >= n) {
            // the last panel: join everything so the graph ends after all writes
            prev = c.join(ready);
            break;
        }
        const int ts = (int)ceil_div(n - base, kP), tx = (int)ceil_div(base, kP);
        np = ts;
        u1 = c.kernel(ready, d32_update1_kernel, (unsigned)(ts + tx), kTT, n, ld, k, F.A, F.X, (const float *)LDp,
                      F.csum);
        c.priority(u1, hi_prio);
        const int base2 = base + kP;
        u2 = nullptr;
        if (base2 < n) {
            // the operands of this panel's bulk update split for the tensor cores (buffers by panel
            // parity: the previous panel's update may still read the other half)
            const int T = (int)ceil_div(n - base2, kTcM), nb = (int)ceil_div(n - base2, kTcN);
            const int nx = (int)ceil_div(base, kTcN);
            float *LDs = F.tc + (size_t)(p & 1) * tc_per_parity(n);
            float *PAs = LDs + tc_a_floats(n), *PBs = PAs + tc_a_floats(n), *XBs = PBs + tc_b_floats(n);
            const float *panel = F.A + (size_t)k * ld;
            std::vector<cudaGraphNode_t> sp;
            sp.push_back(c.kernel(ready, d32_tc_split_kernel<kTcM, false>, (unsigned)T, kTT, n, ld, (const float *)LDp,
                                  base2, LDs));
            sp.push_back(c.kernel(ready, d32_tc_split_kernel<kTcN, false>, (unsigned)nb, kTT, n, ld, panel, base2, PBs));
            sp.push_back(c.kernel(ready, d32_tc_split_kernel<kTcM, false>, (unsigned)T, kTT, n, ld, panel, base2, PAs));
            sp.push_back(c.kernel(ready, d32_tc_split_kernel<kTcN, true>, (unsigned)nx, kTT, base, ld,
                                  (const float *)(F.X + k), 0, XBs));
            for (cudaGraphNode_t q : sp) c.priority(q, lo_prio);
            const int TJ = (int)ceil_div(T * kTcM, kTcN);
            const int tiles = T * TJ + T * nx;   // persistent CTAs: one per SM at most
            u2 = c.kernel_smem(sp, d32_tc_update_kernel, (unsigned)std::max(1, std::min(tiles, sms)), kTcThreads,
                               (unsigned)kTcSmem, n, ld, base, base2, T, (const float *)LDs, (const float *)PBs,
                               (const float *)PAs, (const float *)XBs, F.A, F.X, F.tc_err);
            c.priority(u2, lo_prio);
        }
    }
    }
    if (c.err != cudaSuccess) return fail(OT_ERR_CUDA, cudaGetErrorString(c.err));
    *nodes = c.nodes;
    return ok();
}

Error d32_factor(Dense32 &F, float eps, cudaStream_t st) {
    if (F.tc_err_host && *F.tc_err_host)
        return fail(OT_ERR_TIMEOUT, "dense32: a bounded wait of the tensor-core update gave up");
    if (!F.graph || F.eps != eps) {
        const bool want_tc = F.tc_mode > 0 || (F.tc_mode == 0 && F.n >= kTcAutoN);
        if (want_tc && !F.tc) {
            OT_CUDA(cudaMalloc((void **)&F.tc, sizeof(float) * 2 * tc_per_parity(F.n)));
            OT_CUDA(cudaMalloc((void **)&F.tc_err, sizeof(int)));
            OT_CUDA(cudaMemset(F.tc_err, 0, sizeof(int)));
            OT_CUDA(cudaMallocHost((void **)&F.tc_err_host, sizeof(int)));
            *F.tc_err_host = 0;
            static std::once_flag once;
            static cudaError_t attr = cudaSuccess;
            std::call_once(once, [] {
                attr = cudaFuncSetAttribute(d32_tc_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
            });
            if (attr != cudaSuccess) return fail(OT_ERR_CUDA, cudaGetErrorString(attr));
        }
        F.use_tc = want_tc;
        if (F.graph) {
            cudaGraphExecDestroy(F.graph);
            F.graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        OT_CUDA(cudaGraphCreate(&g, 0));
        int64_t nodes = 0;
        Error e = d32_build(F, eps, g, &nodes);
        if (e.code == OT_OK && cudaGraphInstantiate(&F.graph, g, 0) != cudaSuccess) {
            F.graph = nullptr;
            e = fail(OT_ERR_CUDA, "dense32: graph instantiation failed");
        }
        cudaGraphDestroy(g);
        cudaGetLastError();
        OT_TRY(e);
        F.graph_nodes = nodes;
        F.eps = eps;
    }
    ktimer_begin(KT_D32_FACTOR, st);
    OT_CUDA(cudaGraphLaunch(F.graph, st));
    g_launches.fetch_add(F.graph_nodes, std::memory_order_relaxed);
    ktimer_end(KT_D32_FACTOR, st);
    if (F.use_tc) OT_CUDA(cudaMemcpyAsync(F.tc_err_host, F.tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    // FP32 flops: n^3/3 for L D L^T (n^3/6 multiply-adds) plus n^3/3 for the unit triangular inverse
    ktimer_add_work(KT_D32_FACTOR, 2.0 * (double)F.n * F.n * F.n / 3.0);
    return ok();
}

Error d32_apply(Dense32 &F, const double *r, double *z, cudaStream_t st) {
    const int n = F.n, ld = F.ld;
    const int ncb = (int)ceil_div(n, kFc), nrb = (int)ceil_div(n, kFr);
    int tiles = 0;
    for (int rb = 0; rb < nrb; ++rb) tiles += std::min(ncb, (rb + 1) * (kFr / kFc));
    ktimer_begin(KT_D32_APPLY, st);
    d32_fwd_kernel<<<(unsigned)tiles, kFr, 0, st>>>(n, ld, ncb, F.X, r, F.part);
    OT_LAUNCHED();
    d32_mid_kernel<<<(unsigned)ceil_div(n, kTT), kTT, 0, st>>>(n, ld, F.part, F.D, F.w);
    OT_LAUNCHED();
    d32_bwd_kernel<<<(unsigned)ceil_div(n, kTT / 32), kTT, 0, st>>>(n, ld, F.X, F.w, z);
    OT_LAUNCHED();
    ktimer_end(KT_D32_APPLY, st);
    // bytes: the lower triangle of L^-1 read twice
    ktimer_add_work(KT_D32_APPLY, 4.0 * (double)n * n);
    return ok();
}

}  // namespace ot
