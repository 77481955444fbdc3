// Pricing: reduced costs d_ij = c_ij - u_i - v_j over all m*n pairs (Section 3.4), costs
// evaluated on the fly from integer point coordinates (never stored) -- the squared Euclidean
// distance, or the L1, Euclidean and L-infinity distances of Section 5.1 -- or read from an
// explicit matrix, and the exact selection of the at most kmax most negative pairs outside the
// support (Section 3.2).  Optionally the scan covers only the listed pairs of the heuristic set
// J = {(i, j) : c_ij < C_max} of Section 3.4.
//
// Pipeline (one host synchronisation):
//   prep     squared cost: rows -> float4 (A_i, X_i, Y_i), cols -> float4 (B_j, x_j, y_j) with
//            A_i = |x_i|^2 - u_i, X_i = -2 x_i (coordinates shifted to a common origin);
//            other distances: rows -> (u_i, x_i, y_i), cols -> (v_j, x_j, y_j) in FP32;
//            plus the magnitudes that bound the FP32 rounding error;
//   bound    E >= |d_fp32 - d| for every pair (a priori rounding analysis, 1 thread);
//   pass 1   register-blocked scan (or a pass over the J list), histogram of d < E over 4096
//            magnitude bins + [0, E], minimum per tile;
//   support  the support pairs' own contributions are subtracted from the histogram;
//   thresh   T = edge of the bin holding the kmax-th smallest key; gather threshold
//            Tg = min(T + 2E, E): every pair of the exact selection has d_fp32 <= Tg;
//   pass 2   rescan only tiles whose minimum is <= Tg, append (i, j) with d_fp32 <= Tg;
//   recheck  FP64 d = (c - u) - v (no fusion), support membership by binary search in the
//            CSR rows; sort by (d, jlin) with a stable LSD radix sort; keep the first kmax.
// In the FP64 variant the scan computes d exactly, keys are float(d) (monotone), E = 0.  An
// explicit cost matrix always takes the FP64 variant.
#include "pricing.cuh"
#include "primitives.cuh"

#include <cfloat>
#include <cmath>
#include <type_traits>

namespace ot {
namespace {

constexpr int kBins = 4097;       // bins 0..4095: d < 0 by magnitude (large first); 4096: [0, E]
constexpr int kPT = 256;          // threads per scan CTA
constexpr int kRJ = 8;            // columns held in registers per thread
constexpr int kTJ = kPT * kRJ;    // columns per tile
// above this many pairs inside the FP32 gather window the selection is redone with the FP64 scan
constexpr unsigned long long kMaxWindowPairs = 1ull << 27;

struct Geo {
    unsigned long long umax_bits, vmax_bits;     // max |u|, max |v| (nonneg double bit patterns)
    int xs_max, ys_max, xt_max, yt_max;          // max |shifted coordinate|
    unsigned long long x2s_max, x2t_max;         // max |x|^2 (integers)
    float E;                                     // FP32 error window
    float Tg;                                    // gather threshold (inclusive)
    unsigned long long gather_bound;             // upper bound of pairs with key <= Tg
    unsigned int ncand;                          // gathered pairs
    unsigned int nvalid;                         // rechecked candidates
};

__device__ __forceinline__ int bin_of_neg(float d) {  // d <= 0
    unsigned b = __float_as_uint(-d) >> 19;             // exponent + 4 mantissa bits
    return 4095 - (int)b;                               // larger magnitude -> smaller bin
}

// ------------------------------------------------------------------------ cost evaluation
// Kinds are the ot_cost_kind values.  FP64 costs follow the oracle's definitions exactly: the
// coordinate differences are integers, the squared distance is an exact integer, and the
// Euclidean distance is its correctly rounded square root.
enum : int { K_SQ = OT_COST_SQEUCLID, K_EU = OT_COST_EUCLID, K_L1 = OT_COST_L1, K_LI = OT_COST_LINF,
             K_DN = OT_COST_DENSE };

template <int K>
__device__ __forceinline__ double cost64(int dx, int dy) {
    if (K == K_SQ) return (double)(dx * dx + dy * dy);
    if (K == K_EU) return __dsqrt_rn((double)(dx * dx + dy * dy));
    if (K == K_L1) return (double)(abs(dx) + abs(dy));
    return (double)max(abs(dx), abs(dy));
}

__device__ __forceinline__ double cost64_rt(int kind, int dx, int dy) {
    switch (kind) {
    case K_SQ: return cost64<K_SQ>(dx, dy);
    case K_EU: return cost64<K_EU>(dx, dy);
    case K_L1: return cost64<K_L1>(dx, dy);
    default: return cost64<K_LI>(dx, dy);
    }
}

// Integer key ordered like the cost (the J test c_ij < C_max is key < jlim, exact).
__device__ __forceinline__ long long cost_key(int kind, int dx, int dy) {
    if (kind == K_L1) return (long long)abs(dx) + abs(dy);
    if (kind == K_LI) return (long long)max(abs(dx), abs(dy));
    return (long long)dx * dx + (long long)dy * dy;  // squared and Euclidean distances
}

// FP32 key of one pair.  Squared cost: the alpha/beta form (2 FMA + 1 add) on the packed rows
// (A_i, X_i, Y_i) and columns (B_j, x_j, y_j).  Other distances, direct form on (u_i, x_i, y_i)
// and (v_j, x_j, y_j): dx, dy exact; L1 / L-infinity exact; Euclidean sqrt(fma(dx, dx, dy*dy));
// then d = (c - u_i) - v_j.
template <int K>
__device__ __forceinline__ float key32(const float4 &R, float cB, float cx, float cy) {
    if (K == K_SQ) {
        const float t1 = __fadd_rn(R.x, cB);
        const float t2 = __fmaf_rn(R.z, cy, t1);
        return __fmaf_rn(R.y, cx, t2);
    }
    const float dx = __fsub_rn(R.y, cx), dy = __fsub_rn(R.z, cy);
    float c;
    if (K == K_L1) c = __fadd_rn(fabsf(dx), fabsf(dy));
    else if (K == K_LI) c = fmaxf(fabsf(dx), fabsf(dy));
    else c = __fsqrt_rn(__fmaf_rn(dx, dx, __fmul_rn(dy, dy)));
    return __fsub_rn(__fsub_rn(c, R.x), cB);
}

// --------------------------------------------------------------------------------- prep
template <bool SQ>
__global__ void prep_kernel(int m, int n, const int32_t *__restrict__ sx, const int32_t *__restrict__ sy,
                            const int32_t *__restrict__ tx, const int32_t *__restrict__ ty,
                            const double *__restrict__ u, const double *__restrict__ v, int ox, int oy,
                            float4 *__restrict__ rows, float4 *__restrict__ cols, Geo *geo) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double umax = 0, vmax = 0;
    int xsm = 0, ysm = 0, xtm = 0, ytm = 0;
    long long x2s = 0, x2t = 0;
    for (int64_t i = tid; i < m; i += stride) {
        int x = sx[i] - ox, y = sy[i] - oy;
        long long x2 = (long long)x * x + (long long)y * y;
        float uf = __double2float_rn(u[i]);
        if (rows) {
            if (SQ) rows[i] = make_float4(__fsub_rn(__ll2float_rn(x2), uf), -2.0f * (float)x, -2.0f * (float)y, 0.f);
            else rows[i] = make_float4(uf, (float)x, (float)y, 0.f);
        }
        umax = fmax(umax, fabs(u[i]));
        xsm = max(xsm, abs(x)); ysm = max(ysm, abs(y)); x2s = max(x2s, x2);
    }
    for (int64_t j = tid; j < n; j += stride) {
        int x = tx[j] - ox, y = ty[j] - oy;
        long long x2 = (long long)x * x + (long long)y * y;
        float vf = __double2float_rn(v[j]);
        if (cols) {
            if (SQ) cols[j] = make_float4(__fsub_rn(__ll2float_rn(x2), vf), (float)x, (float)y, 0.f);
            else cols[j] = make_float4(vf, (float)x, (float)y, 0.f);
        }
        vmax = fmax(vmax, fabs(v[j]));
        xtm = max(xtm, abs(x)); ytm = max(ytm, abs(y)); x2t = max(x2t, x2);
    }
    // NaN duals poison the bound: force it to +inf so the window covers everything
    if (umax != umax) umax = INFINITY;
    if (vmax != vmax) vmax = INFINITY;
    atomicMax(&geo->umax_bits, (unsigned long long)__double_as_longlong(umax));
    atomicMax(&geo->vmax_bits, (unsigned long long)__double_as_longlong(vmax));
    atomicMax(&geo->xs_max, xsm); atomicMax(&geo->ys_max, ysm);
    atomicMax(&geo->xt_max, xtm); atomicMax(&geo->yt_max, ytm);
    atomicMax(&geo->x2s_max, (unsigned long long)x2s);
    atomicMax(&geo->x2t_max, (unsigned long long)x2t);
}

// A priori bound of |d_fp32 - d|.  Every rounding contributes at most 2^-24 times the magnitude
// of the value it rounds; each magnitude is bounded from the maxima gathered by prep.
//  squared cost, evaluation order
//    A = fl(fl(|x_i|^2) - fl(u_i)), B = fl(fl(|x_j|^2) - fl(v_j)),
//    t1 = fl(A + B), t2 = fma(Y_i, y_j, t1), d~ = fma(X_i, x_j, t2)
//  (products of integers are exact inside the FMA);
//  other distances, d~ = fl(fl(c~ - fl(u_i)) - fl(v_j)) with c~ exact for L1 and L-infinity and
//  |c~ - c| <= 2.001 * 2^-24 * c for the Euclidean distance (one rounding of dy*dy, one of the
//  FMA, one of the square root; the first two enter the root halved).
__global__ void bound_kernel(Geo *geo, int fp64, int kind) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (fp64) { geo->E = 0.f; return; }
    const double uu = 5.9604644775390625e-08;  // 2^-24
    double umax = __longlong_as_double((long long)geo->umax_bits);
    double vmax = __longlong_as_double((long long)geo->vmax_bits);
    double E;
    if (kind == K_SQ) {
        double x2s = (double)geo->x2s_max, x2t = (double)geo->x2t_max;
        double cross = 2.0 * ((double)geo->xs_max * geo->xt_max + (double)geo->ys_max * geo->yt_max);
        double A = (x2s + umax) * (1 + 2 * uu), B = (x2t + vmax) * (1 + 2 * uu);
        double T1 = (A + B) * (1 + uu), T2 = (T1 + cross) * (1 + uu), D = (T2 + cross) * (1 + uu);
        E = uu * (x2s + umax + A + x2t + vmax + B + T1 + T2 + D) * 1.0001 + 1e-30;
    } else {
        const double xs = (double)geo->xs_max + geo->xt_max, ys = (double)geo->ys_max + geo->yt_max;
        double cmax, epsc = 0.0;
        if (kind == K_L1) cmax = xs + ys;
        else if (kind == K_LI) cmax = fmax(xs, ys);
        else { cmax = sqrt(xs * xs + ys * ys) * (1 + 1e-15); epsc = 2.001 * uu * cmax; }
        const double Cp = cmax + epsc, Up = umax * (1 + uu), Vp = vmax * (1 + uu);
        const double T = Cp + Up;            // |c~ - u~|
        const double Dd = T * (1 + uu) + Vp; // |fl(c~ - u~) - v~|
        E = (epsc + uu * (umax + vmax + T + Dd)) * 1.0001 + 1e-30;
    }
    float Ef = __double2float_ru(E);
    geo->E = isfinite(Ef) ? Ef : FLT_MAX;
}

// One key into the histogram (pass 1) or the candidate list (pass 2).
// Padding columns (j >= n) carry key +inf and never qualify; the gather also checks j < n.
template <bool FP64, bool GATHER>
__device__ __forceinline__ void take_key(float d, bool neg64, float E, float Tg, unsigned *sh_hist, int i, int j,
                                         int n, int32_t *ci, int32_t *cj, unsigned long long cap, unsigned *ncand) {
    const bool neg = FP64 ? neg64 : (d < 0.f);
    if (!GATHER) {
        if (neg) atomicAdd(&sh_hist[bin_of_neg(d)], 1u);
        else if (!FP64 && d <= E) atomicAdd(&sh_hist[4096], 1u);
    } else {
        const bool take = (FP64 ? (neg && d <= Tg) : (d <= Tg)) && j < n;
        if (take) {
            const unsigned pos = atomicAdd(ncand, 1u);
            if (pos < cap) { ci[pos] = i; cj[pos] = j; }
        }
    }
}

// ---------------------------------------------------------------------------------- scan
// Tiles of TI source rows x kTJ target columns; kRJ columns per thread in registers, rows from
// shared memory.  The FP32 variants evaluate keys in groups of 4 rows x kRJ columns with one
// minimum and one branch per group.
template <int K, bool FP64, bool GATHER>
__global__ void __launch_bounds__(kPT)
scan_kernel(int m, int n, int TI, int ncb, int64_t ntiles,
            const float4 *__restrict__ rows, const float4 *__restrict__ cols,
            const int32_t *__restrict__ sx, const int32_t *__restrict__ sy,
            const int32_t *__restrict__ tx, const int32_t *__restrict__ ty,
            const double *__restrict__ u, const double *__restrict__ v, const double *__restrict__ C,
            const Geo *__restrict__ geo, float *__restrict__ tile_min,
            unsigned long long *__restrict__ hist, int32_t *__restrict__ ci,
            int32_t *__restrict__ cj, unsigned long long cap, unsigned int *__restrict__ ncand) {
    __shared__ float4 srow[FP64 ? 1 : 256];
    __shared__ int2 srowi[FP64 ? 256 : 1];
    __shared__ double srowu[FP64 ? 256 : 1];
    __shared__ unsigned sh_hist[GATHER ? 1 : kBins];
    __shared__ float sred[kPT / 32];
    if (!GATHER) {
        for (int b = threadIdx.x; b < kBins; b += kPT) sh_hist[b] = 0;
    }
    const float E = geo->E;
    const float Tg = geo->Tg;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int rb = (int)(t / ncb), cb = (int)(t % ncb);
        if (GATHER && tile_min[t] > Tg) continue;  // uniform over the block
        const int i0 = rb * TI;
        const int nrows = min(TI, m - i0);
        __syncthreads();
        if (threadIdx.x < nrows) {
            const int i = i0 + threadIdx.x;
            if (FP64) {
                if (K != K_DN) srowi[threadIdx.x] = make_int2(sx[i], sy[i]);
                srowu[threadIdx.x] = u[i];
            } else {
                srow[threadIdx.x] = rows[i];
            }
        }
        // columns into registers
        float cB[kRJ], cx[kRJ], cy[kRJ];
        int ix[kRJ], iy[kRJ];
        double dv[kRJ];
#pragma unroll
        for (int c = 0; c < kRJ; ++c) {
            const int j = cb * kTJ + c * kPT + threadIdx.x;
            if (FP64) {
                if (j < n) { if (K != K_DN) { ix[c] = tx[j]; iy[c] = ty[j]; } dv[c] = v[j]; }
                else { ix[c] = 0; iy[c] = 0; dv[c] = -INFINITY; }  // d = +inf
            } else {
                // padding columns get key +inf: cB = +inf in the squared form (d = ... + B_j),
                // -inf in the direct form (d = ... - v_j)
                float4 q = j < n ? cols[j] : make_float4(K == K_SQ ? INFINITY : -INFINITY, 0.f, 0.f, 0.f);
                cB[c] = q.x; cx[c] = q.y; cy[c] = q.z;
            }
        }
        __syncthreads();
        float tmin = INFINITY;
        const float thr = GATHER ? Tg : E;
        int r0 = 0;
        if (!FP64) {
            for (; r0 + 4 <= nrows; r0 += 4) {
                float d[4][kRJ], mq[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 R = srow[r0 + q];
                    mq[q] = INFINITY;
#pragma unroll
                    for (int c = 0; c < kRJ; ++c) {
                        d[q][c] = key32<K>(R, cB[c], cx[c], cy[c]);
                        mq[q] = fminf(mq[q], d[q][c]);
                    }
                }
                const float dmin = fminf(fminf(mq[0], mq[1]), fminf(mq[2], mq[3]));
                tmin = fminf(tmin, dmin);
                if (dmin <= thr) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (mq[q] > thr) continue;
#pragma unroll
                        for (int c = 0; c < kRJ; ++c)
                            take_key<false, GATHER>(d[q][c], false, E, Tg, sh_hist, i0 + r0 + q,
                                                    cb * kTJ + c * kPT + threadIdx.x, n, ci, cj, cap, ncand);
                    }
                }
            }
        }
        for (int r = r0; r < nrows; ++r) {
            float d[kRJ];
            double dd[kRJ];
            float dmin = INFINITY;
            if (FP64) {
                const double ur = srowu[r];
#pragma unroll
                for (int c = 0; c < kRJ; ++c) {
                    double cc;
                    if (K == K_DN) {
                        const int j = cb * kTJ + c * kPT + threadIdx.x;
                        cc = j < n ? C[(int64_t)(i0 + r) * n + j] : 0.0;
                    } else {
                        const int2 R = srowi[r];
                        cc = cost64<K>(R.x - ix[c], R.y - iy[c]);
                    }
                    dd[c] = __dsub_rn(__dsub_rn(cc, ur), dv[c]);
                    d[c] = __double2float_rn(dd[c]);
                    dmin = fminf(dmin, d[c]);
                }
            } else {
                const float4 R = srow[r];
#pragma unroll
                for (int c = 0; c < kRJ; ++c) {
                    d[c] = key32<K>(R, cB[c], cx[c], cy[c]);
                    dmin = fminf(dmin, d[c]);
                }
            }
            tmin = fminf(tmin, dmin);
            if (dmin <= thr) {
#pragma unroll
                for (int c = 0; c < kRJ; ++c)
                    take_key<FP64, GATHER>(d[c], FP64 ? (dd[c] < 0.0) : false, E, Tg, sh_hist, i0 + r,
                                           cb * kTJ + c * kPT + threadIdx.x, n, ci, cj, cap, ncand);
            }
        }
        if (!GATHER) {
            // tile minimum (for skipping tiles in pass 2)
            float w = tmin;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w = fminf(w, __shfl_down_sync(0xffffffffu, w, o));
            if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = w;
            __syncthreads();
            if (threadIdx.x == 0) {
                float b = sred[0];
                for (int k = 1; k < kPT / 32; ++k) b = fminf(b, sred[k]);
                tile_min[t] = b;
            }
        }
    }
    if (!GATHER) {
        __syncthreads();
        for (int b = threadIdx.x; b < kBins; b += kPT)
            if (sh_hist[b]) atomicAdd(&hist[b], (unsigned long long)sh_hist[b]);
    }
}

// ------------------------------------------------------------------------ J-list scan
// Section 3.4's heuristic: only the pairs of J (listed, sorted by (i, j)) are priced.  Tiles of
// kJT consecutive list entries; each thread takes kJE entries kPT apart (coalesced list reads;
// the row and column data come from L2).
constexpr int kJE = 16;
constexpr int kJT = kPT * kJE;

template <int K, bool FP64, bool GATHER>
__global__ void __launch_bounds__(kPT)
jscan_kernel(int n, int64_t jn, int64_t ntiles, const int32_t *__restrict__ ji, const int32_t *__restrict__ jj,
             const float4 *__restrict__ rows, const float4 *__restrict__ cols,
             const int32_t *__restrict__ sx, const int32_t *__restrict__ sy,
             const int32_t *__restrict__ tx, const int32_t *__restrict__ ty,
             const double *__restrict__ u, const double *__restrict__ v, const double *__restrict__ C,
             const Geo *__restrict__ geo, float *__restrict__ tile_min,
             unsigned long long *__restrict__ hist, int32_t *__restrict__ ci,
             int32_t *__restrict__ cj, unsigned long long cap, unsigned int *__restrict__ ncand) {
    __shared__ unsigned sh_hist[GATHER ? 1 : kBins];
    __shared__ float sred[kPT / 32];
    if (!GATHER) {
        for (int b = threadIdx.x; b < kBins; b += kPT) sh_hist[b] = 0;
        __syncthreads();
    }
    const float E = geo->E;
    const float Tg = geo->Tg;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (GATHER && tile_min[t] > Tg) continue;  // uniform over the block
        float tmin = INFINITY;
#pragma unroll 4
        for (int k = 0; k < kJE; ++k) {
            const int64_t e = t * kJT + (int64_t)k * kPT + threadIdx.x;
            if (e >= jn) break;
            const int i = ji[e], j = jj[e];
            float d;
            bool neg64 = false;
            if (FP64) {
                double cc;
                if (K == K_DN) cc = C[(int64_t)i * n + j];
                else cc = cost64<K>(sx[i] - tx[j], sy[i] - ty[j]);
                const double dd = __dsub_rn(__dsub_rn(cc, u[i]), v[j]);
                d = __double2float_rn(dd);
                neg64 = dd < 0.0;
            } else {
                const float4 R = rows[i], Q = cols[j];
                d = key32<K>(R, Q.x, Q.y, Q.z);
            }
            tmin = fminf(tmin, d);
            if (d <= (GATHER ? Tg : E))
                take_key<FP64, GATHER>(d, neg64, E, Tg, sh_hist, i, j, n, ci, cj, cap, ncand);
        }
        if (!GATHER) {
            float w = tmin;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w = fminf(w, __shfl_down_sync(0xffffffffu, w, o));
            __syncthreads();
            if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = w;
            __syncthreads();
            if (threadIdx.x == 0) {
                float b = sred[0];
                for (int q = 1; q < kPT / 32; ++q) b = fminf(b, sred[q]);
                tile_min[t] = b;
            }
        }
    }
    if (!GATHER) {
        __syncthreads();
        for (int b = threadIdx.x; b < kBins; b += kPT)
            if (sh_hist[b]) atomicAdd(&hist[b], (unsigned long long)sh_hist[b]);
    }
}

// The support pairs entered the histogram too (the scan does not test membership); take their
// keys out again.  Same arithmetic as the scan, so every key lands in the same bin.  With a J
// list only the support pairs inside J were scanned: jlim > 0 (integer cost key < jlim) or, for
// an explicit matrix, jcmax > 0 (c_ij < jcmax) selects them.
template <int K, bool FP64>
__global__ void support_hist_kernel(int n, int64_t psi, const int32_t *__restrict__ si, const int32_t *__restrict__ sj,
                                    const float4 *__restrict__ rows, const float4 *__restrict__ cols,
                                    const int32_t *__restrict__ sx, const int32_t *__restrict__ sy,
                                    const int32_t *__restrict__ tx, const int32_t *__restrict__ ty,
                                    const double *__restrict__ u, const double *__restrict__ v,
                                    const double *__restrict__ C, long long jlim, double jcmax,
                                    const Geo *__restrict__ geo, unsigned long long *__restrict__ hist) {
    const float E = geo->E;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < psi;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = si[e], j = sj[e];
        if (K == K_DN) {
            if (jcmax > 0.0 && !(C[(int64_t)i * n + j] < jcmax)) continue;
        } else if (jlim > 0 && cost_key(K, sx[i] - tx[j], sy[i] - ty[j]) >= jlim) {
            continue;
        }
        int bin = -1;
        if (FP64) {
            const double cc = K == K_DN ? C[(int64_t)i * n + j] : cost64<K>(sx[i] - tx[j], sy[i] - ty[j]);
            const double d = __dsub_rn(__dsub_rn(cc, u[i]), v[j]);
            if (d < 0.0) bin = bin_of_neg(__double2float_rn(d));
        } else {
            const float4 R = rows[i], Q = cols[j];
            const float d = key32<K>(R, Q.x, Q.y, Q.z);
            if (d < 0.f) bin = bin_of_neg(d);
            else if (d <= E) bin = 4096;
        }
        if (bin >= 0) atomicAdd(&hist[bin], ~0ull);  // -1
    }
}

// One block: find the bin holding the kmax-th smallest key, the gather threshold Tg and an
// upper bound on the number of pairs (support included) the gather pass will append.
__global__ void __launch_bounds__(1024)
threshold_kernel(const unsigned long long *__restrict__ hist_ns,   // support removed
                 const unsigned long long *__restrict__ hist_all,  // support included
                 int kmax, int fp64, Geo *geo) {
    __shared__ unsigned long long part[1024];
    __shared__ int s_bstar;
    const int t = threadIdx.x;
    unsigned long long loc = 0;
    for (int k = 0; k < 4; ++k) {
        int b = 4 * t + k;
        if (b < kBins) loc += hist_ns[b];
    }
    if (t == 1023) loc += hist_ns[4096];  // 4*1023+3 = 4095; bin 4096 joins the last group
    part[t] = loc;
    if (t == 0) s_bstar = -1;
    __syncthreads();
    // inclusive scan (Hillis-Steele; 1024 entries)
    for (int o = 1; o < 1024; o <<= 1) {
        unsigned long long y = t >= o ? part[t - o] : 0ull;
        __syncthreads();
        part[t] += y;
        __syncthreads();
    }
    unsigned long long before = t > 0 ? part[t - 1] : 0ull;
    if (part[t] >= (unsigned long long)kmax && before < (unsigned long long)kmax) {
        unsigned long long acc = before;
        int lim = (t == 1023) ? 5 : 4;
        for (int k = 0; k < lim; ++k) {
            acc += hist_ns[4 * t + k];
            if (acc >= (unsigned long long)kmax) { s_bstar = 4 * t + k; break; }
        }
    }
    __shared__ int s_bg;
    __syncthreads();
    if (t == 0) {
        const int bstar = s_bstar;
        const float E = geo->E;
        float Tg;
        if (bstar < 0 || bstar == 4096) {
            Tg = fp64 ? 0.0f : E;                 // take every candidate
        } else {
            const float lo = __uint_as_float((unsigned)(4095 - bstar) << 19);
            const float T = -lo;                  // every key in bins <= bstar is <= T
            if (fp64) Tg = T;
            else Tg = fminf(__fadd_ru(T, __fmul_ru(2.0f, E)), E);
        }
        geo->Tg = Tg;
        // bins that can hold keys <= Tg
        s_bg = Tg < 0.f ? bin_of_neg(Tg) : (fp64 ? 4095 : 4096);
    }
    __syncthreads();
    // the gather bound: the pairs (support included) in bins 0 .. bg, summed by the whole block
    const int bg = s_bg;
    unsigned long long loc2 = 0;
    for (int b = t; b <= bg; b += 1024) loc2 += hist_all[b];
    part[t] = loc2;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (t < o) part[t] += part[t + o];
        __syncthreads();
    }
    if (t == 0) geo->gather_bound = part[0];
}

__global__ void recheck_kernel(int m, int n, int kind, unsigned long long count, const int32_t *__restrict__ ci,
                               const int32_t *__restrict__ cj, const int32_t *__restrict__ sx,
                               const int32_t *__restrict__ sy, const int32_t *__restrict__ tx,
                               const int32_t *__restrict__ ty, const double *__restrict__ u,
                               const double *__restrict__ v, const double *__restrict__ C,
                               const int32_t *__restrict__ row_ptr,
                               const int32_t *__restrict__ sup_j, Geo *geo,
                               uint64_t *__restrict__ key, uint32_t *__restrict__ val,
                               uint64_t *__restrict__ dkey, double *__restrict__ dval) {
    const unsigned ncand = geo->ncand;
    for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < count;
         g += (unsigned long long)gridDim.x * blockDim.x) {
        uint64_t kj = ~0ull, kd = ~0ull;
        double d = 0.0;
        if (g < ncand) {
            const int i = ci[g], j = cj[g];
            int lo = row_ptr[i], hi = row_ptr[i + 1];
            while (lo < hi) {  // lower_bound of j in the sorted columns of row i
                int mid = (lo + hi) >> 1;
                if (sup_j[mid] < j) lo = mid + 1; else hi = mid;
            }
            const bool member = lo < row_ptr[i + 1] && sup_j[lo] == j;
            const double cc = kind == K_DN ? C[(int64_t)i * n + j] : cost64_rt(kind, sx[i] - tx[j], sy[i] - ty[j]);
            d = __dsub_rn(__dsub_rn(cc, u[i]), v[j]);
            kj = (uint64_t)i + (uint64_t)j * (uint64_t)m;
            if (!member && d < 0.0) {
                kd = f64_key(d);
                atomicAdd(&geo->nvalid, 1u);
            }
        }
        key[g] = kj;
        val[g] = (uint32_t)g;
        dkey[g] = kd;
        dval[g] = d;
    }
}

__global__ void rekey_kernel(unsigned long long count, const uint32_t *__restrict__ val,
                             const uint64_t *__restrict__ dkey, uint64_t *__restrict__ key) {
    for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < count;
         g += (unsigned long long)gridDim.x * blockDim.x)
        key[g] = dkey[val[g]];
}

__global__ void finalize_kernel(int kmax, const uint32_t *__restrict__ val, const int32_t *__restrict__ ci,
                                const int32_t *__restrict__ cj, const double *__restrict__ dval,
                                const Geo *__restrict__ geo, int32_t *__restrict__ out_i,
                                int32_t *__restrict__ out_j, double *__restrict__ out_d,
                                int32_t *__restrict__ out_count) {
    const int cnt = (int)min((unsigned)kmax, geo->nvalid);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
        const uint32_t g = val[k];
        out_i[k] = ci[g];
        out_j[k] = cj[g];
        if (out_d) out_d[k] = dval[g];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *out_count = cnt;
}

__global__ void row_ptr_kernel(const int32_t *__restrict__ sup_i, int64_t psi, int m, int32_t *__restrict__ rp) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= m; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = psi;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (sup_i[mid] < i) lo = mid + 1; else hi = mid;
        }
        rp[i] = (int32_t)lo;
    }
}

__global__ void minmax_kernel(int m, int n, const int32_t *sx, const int32_t *sy, const int32_t *tx,
                              const int32_t *ty, int *mm /* xmin, ymin, -xmax, -ymax */) {
    int xmin = INT_MAX, ymin = INT_MAX, xmax = INT_MIN, ymax = INT_MIN;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)m + n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int x = i < m ? sx[i] : tx[i - m];
        int y = i < m ? sy[i] : ty[i - m];
        xmin = min(xmin, x); ymin = min(ymin, y); xmax = max(xmax, x); ymax = max(ymax, y);
    }
    atomicMin(&mm[0], xmin); atomicMin(&mm[1], ymin);
    atomicMin(&mm[2], -xmax); atomicMin(&mm[3], -ymax);
}

// J list (Section 3.4): the pairs with c_ij < C_max, sorted by (i, j).  One block per (row,
// chunk of kJC columns): count, then (after an exclusive scan over the counts) fill in order.
constexpr int kJC = 2048;

__device__ __forceinline__ bool in_jset(int kind, int i, int j, int n, const int32_t *sx, const int32_t *sy,
                                        const int32_t *tx, const int32_t *ty, const double *C, long long jlim,
                                        double jcmax) {
    if (kind == K_DN) return C[(int64_t)i * n + j] < jcmax;
    return cost_key(kind, sx[i] - tx[j], sy[i] - ty[j]) < jlim;
}

__global__ void jcount_kernel(int m, int n, int kind, const int32_t *__restrict__ sx, const int32_t *__restrict__ sy,
                              const int32_t *__restrict__ tx, const int32_t *__restrict__ ty,
                              const double *__restrict__ C, long long jlim, double jcmax,
                              uint32_t *__restrict__ counts, unsigned long long *__restrict__ total) {
    __shared__ int sh[kPT / 32];
    const int nch = (int)ceil_div(n, kJC);
    const int64_t blk = blockIdx.x;
    const int i = (int)(blk / nch), c0 = (int)(blk % nch) * kJC;
    int cnt = 0;
    for (int j = c0 + threadIdx.x; j < min(n, c0 + kJC); j += kPT)
        cnt += in_jset(kind, i, j, n, sx, sy, tx, ty, C, jlim, jcmax) ? 1 : 0;
    cnt = warp_sum(cnt);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < kPT / 32; ++w) s += sh[w];
        counts[blk] = (uint32_t)s;
        atomicAdd(total, (unsigned long long)s);
    }
}

__global__ void jfill_kernel(int m, int n, int kind, const int32_t *__restrict__ sx, const int32_t *__restrict__ sy,
                             const int32_t *__restrict__ tx, const int32_t *__restrict__ ty,
                             const double *__restrict__ C, long long jlim, double jcmax,
                             const uint32_t *__restrict__ offs, int32_t *__restrict__ ji, int32_t *__restrict__ jj) {
    __shared__ int wtot[kPT / 32];
    const int nch = (int)ceil_div(n, kJC);
    const int64_t blk = blockIdx.x;
    const int i = (int)(blk / nch), c0 = (int)(blk % nch) * kJC;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t base = offs[blk];
    for (int r = 0; r < kJC / kPT; ++r) {
        const int j = c0 + r * kPT + threadIdx.x;
        const bool f = j < n && in_jset(kind, i, j, n, sx, sy, tx, ty, C, jlim, jcmax);
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wtot[wid] = __popc(bal);
        __syncthreads();
        int before = 0, all = 0;
        for (int w = 0; w < kPT / 32; ++w) { if (w < wid) before += wtot[w]; all += wtot[w]; }
        if (f) {
            const int64_t pos = base + before + __popc(bal & ((1u << lane) - 1u));
            ji[pos] = i;
            jj[pos] = j;
        }
        base += all;
        __syncthreads();
    }
}

}  // namespace

Error build_row_ptr(const int32_t *sup_i, int64_t psi, int32_t m, int32_t *row_ptr, cudaStream_t st) {
    row_ptr_kernel<<<(unsigned)ceil_div((int64_t)m + 1, 256), 256, 0, st>>>(sup_i, psi, m, row_ptr);
    OT_LAUNCHED();
    return ok();
}

Error coord_origin(int32_t m, int32_t n, const int32_t *sx, const int32_t *sy, const int32_t *tx,
                   const int32_t *ty, int32_t *ox, int32_t *oy, cudaStream_t st) {
    DevTemp<int> mm;
    OT_TRY(mm.alloc(4, st));
    int init[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX};
    OT_CUDA(cudaMemcpyAsync(mm.p, init, sizeof(init), cudaMemcpyHostToDevice, st));
    minmax_kernel<<<(unsigned)std::min<int64_t>(1024, ceil_div((int64_t)m + n, 256)), 256, 0, st>>>(
        m, n, sx, sy, tx, ty, mm.p);
    OT_LAUNCHED();
    int h[4];
    OT_CUDA(cudaMemcpyAsync(h, mm.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    OT_CUDA(cudaStreamSynchronize(st));
    *ox = (int32_t)(((int64_t)h[0] + (int64_t)(-h[2])) / 2);
    *oy = (int32_t)(((int64_t)h[1] + (int64_t)(-h[3])) / 2);
    return ok();
}


long long jset_limit(int kind, double cmax) {
    if (!(cmax > 0)) return 0;
    // smallest integer key D whose cost is >= cmax (costs are nondecreasing in the key)
    long long lo = 0, hi = 1LL << 33;
    while (lo < hi) {
        const long long mid = lo + (hi - lo) / 2;
        const double c = kind == K_EU ? std::sqrt((double)mid) : (double)mid;
        if (c >= cmax) hi = mid; else lo = mid + 1;
    }
    return lo;
}

void jset_free(JSet &J) {
    if (J.i) cudaFree(J.i);
    if (J.j) cudaFree(J.j);
    J = JSet();
}

Error jset_build(int kind, int32_t m, int32_t n, const int32_t *sx, const int32_t *sy, const int32_t *tx,
                 const int32_t *ty, const double *C, double cmax, JSet *out, cudaStream_t st) {
    jset_free(*out);
    if (m <= 0 || n <= 0 || !(cmax > 0)) return fail(OT_ERR_ARG, "J set: sizes or C_max out of range");
    if (kind == K_DN ? !C : (!sx || !sy || !tx || !ty)) return fail(OT_ERR_ARG, "J set: missing cost data");
    const long long lim = kind == K_DN ? 0 : jset_limit(kind, cmax);
    const int64_t nch = ceil_div(n, kJC), nblk = (int64_t)m * nch;
    if (nblk > 0x7fffffffLL) return fail(OT_ERR_ARG, "J set: too many row chunks");
    DevTemp<uint32_t> counts;
    DevTemp<unsigned long long> total;
    OT_TRY(counts.alloc(nblk, st));
    OT_TRY(total.alloc(1, st));
    OT_CUDA(cudaMemsetAsync(total.p, 0, sizeof(unsigned long long), st));
    jcount_kernel<<<(unsigned)nblk, kPT, 0, st>>>(m, n, kind, sx, sy, tx, ty, C, lim, cmax, counts.p, total.p);
    OT_LAUNCHED();
    unsigned long long tot = 0;
    OT_CUDA(cudaMemcpyAsync(&tot, total.p, sizeof(tot), cudaMemcpyDeviceToHost, st));
    OT_CUDA(cudaStreamSynchronize(st));
    if (tot > 0x7fffffffull) return fail(OT_ERR_ARG, "J set: more than 2^31 pairs (lower C_max)");
    JSet J;
    J.n = (int64_t)tot;
    J.lim = lim;
    J.cmax = cmax;
    OT_CUDA(cudaMalloc((void **)&J.i, sizeof(int32_t) * std::max<int64_t>(J.n, 1)));
    Error e = [&]() -> Error {
        OT_CUDA(cudaMalloc((void **)&J.j, sizeof(int32_t) * std::max<int64_t>(J.n, 1)));
        OT_TRY(scan_exclusive_u32(counts.p, counts.p, nblk, nullptr, st));
        jfill_kernel<<<(unsigned)nblk, kPT, 0, st>>>(m, n, kind, sx, sy, tx, ty, C, lim, cmax, counts.p, J.i, J.j);
        OT_LAUNCHED();
        OT_CUDA(cudaStreamSynchronize(st));
        return ok();
    }();
    if (e.code != OT_OK) { jset_free(J); return e; }
    *out = J;
    return ok();
}

namespace {

// One scan pass (full tiles or the J list) for cost kind K.
template <int K>
Error scan_pass(const PriceInput &in, bool fp64, bool gather, int TI, int ncb, int64_t ntiles, int grid,
                const float4 *rows, const float4 *cols, const Geo *geo, float *tmin, unsigned long long *hist,
                int32_t *ci, int32_t *cj, unsigned long long cap, unsigned *ncand, cudaStream_t st) {
    const bool jmode = in.jn >= 0;
#define OT_SCAN_ARGS in.m, in.n, TI, ncb, ntiles, rows, cols, in.sx, in.sy, in.tx, in.ty, in.u, in.v, in.C, geo, tmin, \
                     hist, ci, cj, cap, ncand
#define OT_JSCAN_ARGS in.n, in.jn, ntiles, in.ji, in.jj, rows, cols, in.sx, in.sy, in.tx, in.ty, in.u, in.v, in.C, geo, \
                      tmin, hist, ci, cj, cap, ncand
    if constexpr (K == K_DN) {
        if (jmode) {
            if (gather) jscan_kernel<K, true, true><<<grid, kPT, 0, st>>>(OT_JSCAN_ARGS);
            else jscan_kernel<K, true, false><<<grid, kPT, 0, st>>>(OT_JSCAN_ARGS);
        } else {
            if (gather) scan_kernel<K, true, true><<<grid, kPT, 0, st>>>(OT_SCAN_ARGS);
            else scan_kernel<K, true, false><<<grid, kPT, 0, st>>>(OT_SCAN_ARGS);
        }
    } else {
        if (jmode) {
            if (fp64) {
                if (gather) jscan_kernel<K, true, true><<<grid, kPT, 0, st>>>(OT_JSCAN_ARGS);
                else jscan_kernel<K, true, false><<<grid, kPT, 0, st>>>(OT_JSCAN_ARGS);
            } else {
                if (gather) jscan_kernel<K, false, true><<<grid, kPT, 0, st>>>(OT_JSCAN_ARGS);
                else jscan_kernel<K, false, false><<<grid, kPT, 0, st>>>(OT_JSCAN_ARGS);
            }
        } else {
            if (fp64) {
                if (gather) scan_kernel<K, true, true><<<grid, kPT, 0, st>>>(OT_SCAN_ARGS);
                else scan_kernel<K, true, false><<<grid, kPT, 0, st>>>(OT_SCAN_ARGS);
            } else {
                if (gather) scan_kernel<K, false, true><<<grid, kPT, 0, st>>>(OT_SCAN_ARGS);
                else scan_kernel<K, false, false><<<grid, kPT, 0, st>>>(OT_SCAN_ARGS);
            }
        }
    }
#undef OT_SCAN_ARGS
#undef OT_JSCAN_ARGS
    OT_LAUNCHED();
    return ok();
}

template <int K>
Error support_pass(const PriceInput &in, bool fp64, int blocks, const float4 *rows, const float4 *cols,
                   const Geo *geo, unsigned long long *hist, cudaStream_t st) {
    const bool jmode = in.jn >= 0;
    const long long jlim = jmode ? in.jlim : 0;
    const double jcmax = jmode ? in.jcmax : 0.0;
    if (fp64 || K == K_DN)
        support_hist_kernel<K, true><<<blocks, 256, 0, st>>>(in.n, in.psi, in.sup_i, in.sup_j, rows, cols, in.sx,
                                                             in.sy, in.tx, in.ty, in.u, in.v, in.C, jlim, jcmax,
                                                             geo, hist);
    else
        support_hist_kernel<K, false><<<blocks, 256, 0, st>>>(in.n, in.psi, in.sup_i, in.sup_j, rows, cols, in.sx,
                                                              in.sy, in.tx, in.ty, in.u, in.v, in.C, jlim, jcmax,
                                                              geo, hist);
    OT_LAUNCHED();
    return ok();
}

template <typename F>
Error by_kind(int kind, F &&f) {
    switch (kind) {
    case K_SQ: return f(std::integral_constant<int, K_SQ>());
    case K_EU: return f(std::integral_constant<int, K_EU>());
    case K_L1: return f(std::integral_constant<int, K_L1>());
    case K_LI: return f(std::integral_constant<int, K_LI>());
    case K_DN: return f(std::integral_constant<int, K_DN>());
    default: return fail(OT_ERR_ARG, "price_topk: unknown cost kind");
    }
}

}  // namespace

Error price_topk(const PriceInput &in, int32_t *out_i, int32_t *out_j, double *out_d,
                 int32_t *out_count, PriceStats *stats, cudaStream_t st) {
    const int m = in.m, n = in.n;
    if (m <= 0 || n <= 0 || in.kmax < 0) return fail(OT_ERR_ARG, "price_topk: bad sizes");
    if ((uint64_t)m * (uint64_t)n > (1ull << 32)) return fail(OT_ERR_ARG, "price_topk: m*n > 2^32");
    const int kind = in.kind;
    if (kind < K_SQ || kind > K_DN) return fail(OT_ERR_ARG, "price_topk: unknown cost kind");
    if (kind == K_DN ? !in.C : (!in.sx || !in.sy || !in.tx || !in.ty))
        return fail(OT_ERR_ARG, "price_topk: missing coordinates or cost matrix");
    const bool jmode = in.jn >= 0;
    if (jmode && in.jn > 0 && (!in.ji || !in.jj)) return fail(OT_ERR_ARG, "price_topk: J list missing");
    const bool fp64 = in.precision == 0 || kind == K_DN;
    int sms = in.num_sms;
    if (sms <= 0) {
        int dev;
        OT_CUDA(cudaGetDevice(&dev));
        OT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    // tiles: TI rows x 2048 columns (aim for >= 4 tiles per SM), or kJT entries of the J list
    const int ncb = (int)ceil_div(n, kTJ);
    int TI = kPT;
    while (TI > 8 && ceil_div(m, TI) * (int64_t)ncb < 4LL * sms) TI >>= 1;
    if (in.rows > 0) TI = std::max(8, std::min(kPT, in.rows));
    const int64_t ntiles = jmode ? ceil_div(in.jn, kJT) : (int64_t)ceil_div(m, TI) * ncb;

    DevTemp<Geo> geo;
    DevTemp<float4> rows, cols;
    DevTemp<float> tmin;
    DevTemp<unsigned long long> hist;  // [2][kBins]: support removed / support included
    OT_TRY(geo.alloc(1, st));
    if (!fp64) {
        OT_TRY(rows.alloc(m, st));
        OT_TRY(cols.alloc(n, st));
    }
    OT_TRY(tmin.alloc(ntiles, st));
    OT_TRY(hist.alloc(2 * kBins, st));
    OT_CUDA(cudaMemsetAsync(geo.p, 0, sizeof(Geo), st));
    OT_CUDA(cudaMemsetAsync(hist.p, 0, sizeof(unsigned long long) * 2 * kBins, st));

    if (kind != K_DN) {
        const int prep_blocks = (int)std::min<int64_t>(4 * sms, ceil_div(std::max(m, n), 256));
        if (kind == K_SQ)
            prep_kernel<true><<<prep_blocks, 256, 0, st>>>(m, n, in.sx, in.sy, in.tx, in.ty, in.u, in.v, in.origin_x,
                                                           in.origin_y, rows.p, cols.p, geo.p);
        else
            prep_kernel<false><<<prep_blocks, 256, 0, st>>>(m, n, in.sx, in.sy, in.tx, in.ty, in.u, in.v, in.origin_x,
                                                            in.origin_y, rows.p, cols.p, geo.p);
        OT_LAUNCHED();
    }
    bound_kernel<<<1, 32, 0, st>>>(geo.p, fp64 ? 1 : 0, kind);
    OT_LAUNCHED();

    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, 8LL * sms));
    if (ntiles > 0) {
        ktimer_begin(KT_SCAN_HIST, st);
        OT_TRY(by_kind(kind, [&](auto kc) {
            return scan_pass<decltype(kc)::value>(in, fp64, false, TI, ncb, ntiles, grid, rows.p, cols.p, geo.p,
                                                  tmin.p, hist.p, nullptr, nullptr, 0, nullptr, st);
        }));
        ktimer_end(KT_SCAN_HIST, st);
        const double per_pair = kind == K_SQ ? 4.0 : (kind == K_EU ? 8.0 : 6.0);
        ktimer_add_work(KT_SCAN_HIST, per_pair * (jmode ? (double)in.jn : (double)m * (double)n));
    }
    OT_CUDA(cudaMemcpyAsync(hist.p + kBins, hist.p, sizeof(unsigned long long) * kBins,
                            cudaMemcpyDeviceToDevice, st));
    if (in.psi > 0) {
        const int sb = (int)std::min<int64_t>(4 * sms, ceil_div(in.psi, 256));
        OT_TRY(by_kind(kind, [&](auto kc) {
            return support_pass<decltype(kc)::value>(in, fp64, sb, rows.p, cols.p, geo.p, hist.p, st);
        }));
    }
    threshold_kernel<<<1, 1024, 0, st>>>(hist.p, hist.p + kBins, std::max(in.kmax, 1), fp64 ? 1 : 0, geo.p);
    OT_LAUNCHED();
    Geo hg;
    OT_CUDA(cudaMemcpyAsync(&hg, geo.p, sizeof(Geo), cudaMemcpyDeviceToHost, st));
    OT_CUDA(cudaStreamSynchronize(st));
    const unsigned long long cap = hg.gather_bound;
    if (!fp64 && cap > kMaxWindowPairs) {
        // fewer negative keys than kmax and a flood of pairs inside the FP32 window [0, E] (duals
        // near a degenerate optimum): the exact FP64 scan gathers only the pairs with d < 0
        PriceInput in64 = in;
        in64.precision = 0;
        return price_topk(in64, out_i, out_j, out_d, out_count, stats, st);
    }
    if (cap > 0x7fffffffull) return fail(OT_ERR_OOM, "price_topk: candidate set exceeds 2^31 pairs");

    DevTemp<int32_t> ci, cj;
    OT_TRY(ci.alloc((int64_t)cap, st));
    OT_TRY(cj.alloc((int64_t)cap, st));
    if (cap > 0 && ntiles > 0) {
        ktimer_begin(KT_SCAN_GATHER, st);
        OT_TRY(by_kind(kind, [&](auto kc) {
            return scan_pass<decltype(kc)::value>(in, fp64, true, TI, ncb, ntiles, grid, rows.p, cols.p, geo.p,
                                                  tmin.p, nullptr, ci.p, cj.p, cap, &geo.p->ncand, st);
        }));
        ktimer_end(KT_SCAN_GATHER, st);
    }
    // support membership needs CSR rows
    DevTemp<int32_t> rp_tmp;
    const int32_t *rp = in.row_ptr;
    if (!rp) {
        OT_TRY(rp_tmp.alloc((int64_t)m + 1, st));
        OT_TRY(build_row_ptr(in.sup_i, in.psi, m, rp_tmp.p, st));
        rp = rp_tmp.p;
    }
    DevTemp<uint64_t> key, dkey;
    DevTemp<uint32_t> val;
    DevTemp<double> dval;
    const int64_t cnt = (int64_t)cap;
    OT_TRY(key.alloc(cnt, st));
    OT_TRY(dkey.alloc(cnt, st));
    OT_TRY(val.alloc(cnt, st));
    OT_TRY(dval.alloc(cnt, st));
    if (cnt > 0) {
        const int rb = (int)std::min<int64_t>(8 * sms, ceil_div(cnt, 256));
        ktimer_begin(KT_RECHECK, st);
        recheck_kernel<<<rb, 256, 0, st>>>(m, n, kind, (unsigned long long)cnt, ci.p, cj.p, in.sx, in.sy, in.tx,
                                           in.ty, in.u, in.v, in.C, rp, in.sup_j, geo.p, key.p, val.p, dkey.p, dval.p);
        OT_LAUNCHED();
        ktimer_end(KT_RECHECK, st);
        int jbits = 1;
        while (jbits < 64 && ((uint64_t)m * (uint64_t)n - 1) >> jbits) ++jbits;
        OT_TRY(radix_sort_pairs(key.p, val.p, cnt, jbits, st));
        rekey_kernel<<<rb, 256, 0, st>>>((unsigned long long)cnt, val.p, dkey.p, key.p);
        OT_LAUNCHED();
        OT_TRY(radix_sort_pairs(key.p, val.p, cnt, 64, st));
    }
    finalize_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(in.kmax, 256), 4 * sms)), 256, 0, st>>>(
        in.kmax, val.p, ci.p, cj.p, dval.p, geo.p, out_i, out_j, out_d, out_count);
    OT_LAUNCHED();
    if (stats) {
        OT_CUDA(cudaMemcpyAsync(&hg, geo.p, sizeof(Geo), cudaMemcpyDeviceToHost, st));
        OT_CUDA(cudaStreamSynchronize(st));
        stats->gathered = hg.ncand;
        stats->valid = hg.nvalid;
        stats->selected = std::min<uint32_t>((uint32_t)in.kmax, hg.nvalid);
        stats->err_bound = hg.E;
    }
    return ok();
}

}  // namespace ot
