// Pricing: reduced costs d_ij = c_ij - u_i - v_j over all m*n pairs of a squared-Euclidean
// point set (Section 3.4), costs evaluated on the fly (never stored), and the exact selection
// of the at most kmax most negative pairs outside the support (Section 3.2).
//
// Pipeline (one host synchronisation):
//   prep     rows -> float4 (A_i, X_i, Y_i), cols -> float4 (B_j, x_j, y_j) with
//            A_i = |x_i|^2 - u_i, X_i = -2 x_i (coordinates shifted to a common origin),
//            plus the magnitudes that bound the FP32 rounding error;
//   bound    E >= |d_fp32 - d| for every pair (a priori rounding analysis, 1 thread);
//   pass 1   register-blocked scan, histogram of d < E over 4096 magnitude bins + [0, E],
//            minimum per tile;
//   support  the support pairs' own contributions are subtracted from the histogram;
//   thresh   T = edge of the bin holding the kmax-th smallest key; gather threshold
//            Tg = min(T + 2E, E): every pair of the exact selection has d_fp32 <= Tg;
//   pass 2   rescan only tiles whose minimum is <= Tg, append (i, j) with d_fp32 <= Tg;
//   recheck  FP64 d = (c - u) - v (no fusion), support membership by binary search in the
//            CSR rows; sort by (d, jlin) with a stable LSD radix sort; keep the first kmax.
// In the FP64 variant the scan computes d exactly, keys are float(d) (monotone), E = 0.
#include "pricing.cuh"
#include "primitives.cuh"

#include <cfloat>
#include <cmath>

namespace ot {
namespace {

constexpr int kBins = 4097;       // bins 0..4095: d < 0 by magnitude (large first); 4096: [0, E]
constexpr int kPT = 256;          // threads per scan CTA
constexpr int kRJ = 8;            // columns held in registers per thread
constexpr int kTJ = kPT * kRJ;    // columns per tile

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

// --------------------------------------------------------------------------------- prep
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
        float a = __fsub_rn(__ll2float_rn(x2), uf);
        if (rows) rows[i] = make_float4(a, -2.0f * (float)x, -2.0f * (float)y, 0.f);
        umax = fmax(umax, fabs(u[i]));
        xsm = max(xsm, abs(x)); ysm = max(ysm, abs(y)); x2s = max(x2s, x2);
    }
    for (int64_t j = tid; j < n; j += stride) {
        int x = tx[j] - ox, y = ty[j] - oy;
        long long x2 = (long long)x * x + (long long)y * y;
        float vf = __double2float_rn(v[j]);
        float b = __fsub_rn(__ll2float_rn(x2), vf);
        if (cols) cols[j] = make_float4(b, (float)x, (float)y, 0.f);
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

// A priori bound of |d_fp32 - d| for the evaluation order
//   A = fl(fl(|x_i|^2) - fl(u_i)), B = fl(fl(|x_j|^2) - fl(v_j)),
//   t1 = fl(A + B), t2 = fma(Y_i, y_j, t1), d~ = fma(X_i, x_j, t2)
// (products of integers are exact inside the FMA).  Every rounding contributes at most
// 2^-24 times the magnitude of the value it rounds; each magnitude is bounded below.
__global__ void bound_kernel(Geo *geo, int fp64) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (fp64) { geo->E = 0.f; return; }
    const double uu = 5.9604644775390625e-08;  // 2^-24
    double umax = __longlong_as_double((long long)geo->umax_bits);
    double vmax = __longlong_as_double((long long)geo->vmax_bits);
    double x2s = (double)geo->x2s_max, x2t = (double)geo->x2t_max;
    double cross = 2.0 * ((double)geo->xs_max * geo->xt_max + (double)geo->ys_max * geo->yt_max);
    double A = (x2s + umax) * (1 + 2 * uu), B = (x2t + vmax) * (1 + 2 * uu);
    double T1 = (A + B) * (1 + uu), T2 = (T1 + cross) * (1 + uu), D = (T2 + cross) * (1 + uu);
    double E = uu * (x2s + umax + A + x2t + vmax + B + T1 + T2 + D) * 1.0001 + 1e-30;
    float Ef = __double2float_ru(E);
    geo->E = isfinite(Ef) ? Ef : FLT_MAX;
}

// ---------------------------------------------------------------------------------- scan
template <bool FP64, bool GATHER>
__global__ void __launch_bounds__(kPT)
scan_kernel(int m, int n, int TI, int ncb, int64_t ntiles,
            const float4 *__restrict__ rows, const float4 *__restrict__ cols,
            const int32_t *__restrict__ sx, const int32_t *__restrict__ sy,
            const int32_t *__restrict__ tx, const int32_t *__restrict__ ty,
            const double *__restrict__ u, const double *__restrict__ v,
            const Geo *__restrict__ geo, float *__restrict__ tile_min,
            unsigned long long *__restrict__ hist, int32_t *__restrict__ ci,
            int32_t *__restrict__ cj, unsigned long long cap, unsigned int *__restrict__ ncand) {
    __shared__ float4 srow[256];
    __shared__ int2 srowi[256];
    __shared__ double srowu[256];
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
                srowi[threadIdx.x] = make_int2(sx[i], sy[i]);
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
                if (j < n) { ix[c] = tx[j]; iy[c] = ty[j]; dv[c] = v[j]; }
                else { ix[c] = 0; iy[c] = 0; dv[c] = -INFINITY; }  // d = +inf
            } else {
                float4 q = j < n ? cols[j] : make_float4(INFINITY, 0.f, 0.f, 0.f);
                cB[c] = q.x; cx[c] = q.y; cy[c] = q.z;
            }
        }
        __syncthreads();
        float tmin = INFINITY;
        const float thr = GATHER ? Tg : E;
        int r0 = 0;
        if (!FP64) {
            // FP32 scan in groups of 4 rows: 32 independent keys, one minimum and one branch per group
            for (; r0 + 4 <= nrows; r0 += 4) {
                float d[4][kRJ], mq[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 R = srow[r0 + q];
                    mq[q] = INFINITY;
#pragma unroll
                    for (int c = 0; c < kRJ; ++c) {
                        const float t1 = __fadd_rn(R.x, cB[c]);
                        const float t2 = __fmaf_rn(R.z, cy[c], t1);
                        d[q][c] = __fmaf_rn(R.y, cx[c], t2);
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
                        for (int c = 0; c < kRJ; ++c) {
                            if (!GATHER) {
                                if (d[q][c] < 0.f) atomicAdd(&sh_hist[bin_of_neg(d[q][c])], 1u);
                                else if (d[q][c] <= E) atomicAdd(&sh_hist[4096], 1u);
                            } else if (d[q][c] <= Tg) {
                                const unsigned pos = atomicAdd(ncand, 1u);
                                if (pos < cap) {
                                    ci[pos] = i0 + r0 + q;
                                    cj[pos] = cb * kTJ + c * kPT + threadIdx.x;
                                }
                            }
                        }
                    }
                }
            }
        }
        for (int r = r0; r < nrows; ++r) {
            float d[kRJ];
            double dd[kRJ];
            float dmin = INFINITY;
            if (FP64) {
                const int2 R = srowi[r];
                const double ur = srowu[r];
#pragma unroll
                for (int c = 0; c < kRJ; ++c) {
                    const int dx = R.x - ix[c], dy = R.y - iy[c];
                    const double cc = (double)(dx * dx + dy * dy);
                    dd[c] = __dsub_rn(__dsub_rn(cc, ur), dv[c]);
                    d[c] = __double2float_rn(dd[c]);
                    dmin = fminf(dmin, d[c]);
                }
            } else {
                const float4 R = srow[r];
#pragma unroll
                for (int c = 0; c < kRJ; ++c) {
                    float t1 = __fadd_rn(R.x, cB[c]);
                    float t2 = __fmaf_rn(R.z, cy[c], t1);
                    d[c] = __fmaf_rn(R.y, cx[c], t2);
                    dmin = fminf(dmin, d[c]);
                }
            }
            tmin = fminf(tmin, dmin);
            if (dmin <= thr) {
#pragma unroll
                for (int c = 0; c < kRJ; ++c) {
                    const bool neg = FP64 ? (dd[c] < 0.0) : (d[c] < 0.f);
                    if (!GATHER) {
                        if (neg) atomicAdd(&sh_hist[bin_of_neg(d[c])], 1u);
                        else if (!FP64 && d[c] <= E) atomicAdd(&sh_hist[4096], 1u);
                    } else {
                        const bool take = FP64 ? (neg && d[c] <= Tg) : (d[c] <= Tg);
                        if (take) {
                            unsigned pos = atomicAdd(ncand, 1u);
                            if (pos < cap) {
                                ci[pos] = i0 + r;
                                cj[pos] = cb * kTJ + c * kPT + threadIdx.x;
                            }
                        }
                    }
                }
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

// The support pairs entered the histogram too (the scan does not test membership); take their
// keys out again.  Same arithmetic as the scan, so every key lands in the same bin.
template <bool FP64>
__global__ void support_hist_kernel(int64_t psi, const int32_t *__restrict__ si, const int32_t *__restrict__ sj,
                                    const float4 *__restrict__ rows, const float4 *__restrict__ cols,
                                    const int32_t *__restrict__ sx, const int32_t *__restrict__ sy,
                                    const int32_t *__restrict__ tx, const int32_t *__restrict__ ty,
                                    const double *__restrict__ u, const double *__restrict__ v,
                                    const Geo *__restrict__ geo, unsigned long long *__restrict__ hist) {
    const float E = geo->E;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < psi;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = si[e], j = sj[e];
        int bin = -1;
        if (FP64) {
            const int dx = sx[i] - tx[j], dy = sy[i] - ty[j];
            const double d = __dsub_rn(__dsub_rn((double)(dx * dx + dy * dy), u[i]), v[j]);
            if (d < 0.0) bin = bin_of_neg(__double2float_rn(d));
        } else {
            const float4 R = rows[i], Q = cols[j];
            float t1 = __fadd_rn(R.x, Q.x);
            float t2 = __fmaf_rn(R.z, Q.z, t1);
            float d = __fmaf_rn(R.y, Q.y, t2);
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
        int bg;                                   // bins that can hold keys <= Tg
        if (Tg < 0.f) bg = bin_of_neg(Tg);
        else bg = fp64 ? 4095 : 4096;
        unsigned long long tot = 0;
        for (int b = 0; b <= bg; ++b) tot += hist_all[b];
        geo->gather_bound = tot;
    }
}

__global__ void recheck_kernel(int m, unsigned long long count, const int32_t *__restrict__ ci,
                               const int32_t *__restrict__ cj, const int32_t *__restrict__ sx,
                               const int32_t *__restrict__ sy, const int32_t *__restrict__ tx,
                               const int32_t *__restrict__ ty, const double *__restrict__ u,
                               const double *__restrict__ v, const int32_t *__restrict__ row_ptr,
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
            const int dx = sx[i] - tx[j], dy = sy[i] - ty[j];
            d = __dsub_rn(__dsub_rn((double)(dx * dx + dy * dy), u[i]), v[j]);
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

Error price_topk(const PriceInput &in, int32_t *out_i, int32_t *out_j, double *out_d,
                 int32_t *out_count, PriceStats *stats, cudaStream_t st) {
    const int m = in.m, n = in.n;
    if (m <= 0 || n <= 0 || in.kmax < 0) return fail(OT_ERR_ARG, "price_topk: bad sizes");
    if ((uint64_t)m * (uint64_t)n > (1ull << 32)) return fail(OT_ERR_ARG, "price_topk: m*n > 2^32");
    const bool fp64 = in.precision == 0;
    int sms = in.num_sms;
    if (sms <= 0) {
        int dev;
        OT_CUDA(cudaGetDevice(&dev));
        OT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    // tiles: TI rows x 2048 columns; aim for >= 4 tiles per SM
    const int ncb = (int)ceil_div(n, kTJ);
    int TI = kPT;
    while (TI > 8 && ceil_div(m, TI) * (int64_t)ncb < 4LL * sms) TI >>= 1;
    if (in.rows > 0) TI = std::max(8, std::min(kPT, in.rows));
    const int nrb = (int)ceil_div(m, TI);
    const int64_t ntiles = (int64_t)nrb * ncb;

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

    const int prep_blocks = (int)std::min<int64_t>(4 * sms, ceil_div(std::max(m, n), 256));
    prep_kernel<<<prep_blocks, 256, 0, st>>>(m, n, in.sx, in.sy, in.tx, in.ty, in.u, in.v, in.origin_x,
                                             in.origin_y, rows.p, cols.p, geo.p);
    OT_LAUNCHED();
    bound_kernel<<<1, 32, 0, st>>>(geo.p, fp64 ? 1 : 0);
    OT_LAUNCHED();

    const int grid = (int)std::min<int64_t>(ntiles, 8LL * sms);
    ktimer_begin(KT_SCAN_HIST, st);
    if (fp64)
        scan_kernel<true, false><<<grid, kPT, 0, st>>>(m, n, TI, ncb, ntiles, rows.p, cols.p, in.sx, in.sy,
                                                       in.tx, in.ty, in.u, in.v, geo.p, tmin.p, hist.p,
                                                       nullptr, nullptr, 0, nullptr);
    else
        scan_kernel<false, false><<<grid, kPT, 0, st>>>(m, n, TI, ncb, ntiles, rows.p, cols.p, in.sx, in.sy,
                                                        in.tx, in.ty, in.u, in.v, geo.p, tmin.p, hist.p,
                                                        nullptr, nullptr, 0, nullptr);
    OT_LAUNCHED();
    ktimer_end(KT_SCAN_HIST, st);
    ktimer_add_work(KT_SCAN_HIST, 4.0 * (double)m * (double)n);
    OT_CUDA(cudaMemcpyAsync(hist.p + kBins, hist.p, sizeof(unsigned long long) * kBins,
                            cudaMemcpyDeviceToDevice, st));
    if (in.psi > 0) {
        const int sb = (int)std::min<int64_t>(4 * sms, ceil_div(in.psi, 256));
        if (fp64)
            support_hist_kernel<true><<<sb, 256, 0, st>>>(in.psi, in.sup_i, in.sup_j, rows.p, cols.p, in.sx,
                                                         in.sy, in.tx, in.ty, in.u, in.v, geo.p, hist.p);
        else
            support_hist_kernel<false><<<sb, 256, 0, st>>>(in.psi, in.sup_i, in.sup_j, rows.p, cols.p, in.sx,
                                                          in.sy, in.tx, in.ty, in.u, in.v, geo.p, hist.p);
        OT_LAUNCHED();
    }
    threshold_kernel<<<1, 1024, 0, st>>>(hist.p, hist.p + kBins, std::max(in.kmax, 1), fp64 ? 1 : 0, geo.p);
    OT_LAUNCHED();
    Geo hg;
    OT_CUDA(cudaMemcpyAsync(&hg, geo.p, sizeof(Geo), cudaMemcpyDeviceToHost, st));
    OT_CUDA(cudaStreamSynchronize(st));
    const unsigned long long cap = hg.gather_bound;
    if (cap > 0x7fffffffull) return fail(OT_ERR_OOM, "price_topk: candidate set exceeds 2^31 pairs");

    DevTemp<int32_t> ci, cj;
    OT_TRY(ci.alloc((int64_t)cap, st));
    OT_TRY(cj.alloc((int64_t)cap, st));
    if (cap > 0) {
        ktimer_begin(KT_SCAN_GATHER, st);
        if (fp64)
            scan_kernel<true, true><<<grid, kPT, 0, st>>>(m, n, TI, ncb, ntiles, rows.p, cols.p, in.sx, in.sy,
                                                          in.tx, in.ty, in.u, in.v, geo.p, tmin.p, nullptr,
                                                          ci.p, cj.p, cap, &geo.p->ncand);
        else
            scan_kernel<false, true><<<grid, kPT, 0, st>>>(m, n, TI, ncb, ntiles, rows.p, cols.p, in.sx, in.sy,
                                                           in.tx, in.ty, in.u, in.v, geo.p, tmin.p, nullptr,
                                                           ci.p, cj.p, cap, &geo.p->ncand);
        OT_LAUNCHED();
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
        recheck_kernel<<<rb, 256, 0, st>>>(m, (unsigned long long)cnt, ci.p, cj.p, in.sx, in.sy, in.tx, in.ty,
                                           in.u, in.v, rp, in.sup_j, geo.p, key.p, val.p, dkey.p, dval.p);
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
