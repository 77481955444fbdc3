// Newton direction of the restricted IPM (eq. redsystem) through the normal equations
// (eq. normalequationsipm) and the Schur complement S_M = N - V^T M^-1 V (Section 4), solved
// matrix-free by PCG.  All reductions are deterministic (fixed-order two-stage sums).
#include "newton.cuh"
#include "ic.cuh"
#include "tree.cuh"
#include "dense32.cuh"
#include "chol.cuh"
#include "primitives.cuh"

#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

namespace ot {
namespace {

constexpr int kT = 256;

inline unsigned grid_of(int64_t work, int sms) {
    int64_t g = ceil_div(work, kT);
    int64_t cap = std::min<int64_t>(kMaxPartBlocks, 4LL * std::max(sms, 1));
    return (unsigned)std::max<int64_t>(1, std::min(g, cap));
}

#define GRID_STRIDE(var, count) \
    for (int64_t var = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; var < (count); var += (int64_t)gridDim.x * blockDim.x)

// stage-1 partial: thread 0 of each block writes part[slot*kMaxPartBlocks + blockIdx.x]
__device__ __forceinline__ void put_sum(double x, double *part, int slot, double *sh) {
    double r = block_sum(x, sh);
    if (threadIdx.x == 0) part[(int64_t)slot * kMaxPartBlocks + blockIdx.x] = r;
}
__device__ __forceinline__ void put_min(double x, double *part, int slot, double *sh) {
    double r = block_min(x, sh);
    if (threadIdx.x == 0) part[(int64_t)slot * kMaxPartBlocks + blockIdx.x] = r;
}
__device__ __forceinline__ void put_max(double x, double *part, int slot, double *sh) {
    double r = -block_min(-x, sh);
    if (threadIdx.x == 0) part[(int64_t)slot * kMaxPartBlocks + blockIdx.x] = r;
}

// stage 2: block b reduces slot slots[b] over nblk[b] partials with op ops[b] (0 sum, 1 min, 2 max)
struct Finish {
    int count;
    int slot[8];
    int nblk[8];
    int op[8];
};

__global__ void finish_kernel(Finish f, const double *__restrict__ part, double *__restrict__ scal) {
    __shared__ double sh[kT / 32];
    const int b = blockIdx.x;
    if (b >= f.count) return;
    const int slot = f.slot[b], nb = f.nblk[b], op = f.op[b];
    double acc = op == 0 ? 0.0 : (op == 1 ? INFINITY : -INFINITY);
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        double x = part[(int64_t)slot * kMaxPartBlocks + k];
        acc = op == 0 ? acc + x : (op == 1 ? fmin(acc, x) : fmax(acc, x));
    }
    double r;
    if (op == 0) r = block_sum(acc, sh);
    else if (op == 1) r = block_min(acc, sh);
    else r = -block_min(-acc, sh);
    if (threadIdx.x == 0) scal[slot] = r;
}

Error finish(const Finish &f, Newton &W, cudaStream_t st) {
    finish_kernel<<<f.count, kT, 0, st>>>(f, W.part, W.scal);
    OT_LAUNCHED();
    return ok();
}

// ------------------------------------------------------------------------ support costs
__global__ void support_cost_kernel(CostDev cd, int64_t psi, const int32_t *__restrict__ si,
                                    const int32_t *__restrict__ sj, double *__restrict__ c) {
    GRID_STRIDE(e, psi) c[e] = cost_at(cd, si[e], sj[e]);
}

// ------------------------------------------------------------------------ residuals
__global__ void res_rows_kernel(int m, const int32_t *__restrict__ rp, const double *__restrict__ p,
                                const double *__restrict__ a, double *__restrict__ r1a, double *part) {
    __shared__ double sh[kT / 32];
    double sq = 0, l1 = 0;
    GRID_STRIDE(i, m) {
        double acc = 0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) acc += p[e];
        const double r = a[i] - acc;
        r1a[i] = r;
        sq += r * r;
        l1 += fabs(r);
    }
    put_sum(sq, part, SC_R1A_SQ, sh);
    put_sum(l1, part, SC_R1A_L1, sh);
}

__global__ void res_entries_kernel(int64_t psi, const int32_t *__restrict__ si, const int32_t *__restrict__ sj,
                                   const double *__restrict__ c, const double *__restrict__ p,
                                   const double *__restrict__ s, const double *__restrict__ u,
                                   const double *__restrict__ v, double *__restrict__ r2, double *part) {
    __shared__ double sh[kT / 32];
    double r2sq = 0, ps = 0, cp = 0, csq = 0, cmax = 0;
    GRID_STRIDE(e, psi) {
        const double ce = c[e];
        const double r = ((ce - u[si[e]]) - v[sj[e]]) - s[e];
        r2[e] = r;
        r2sq += r * r;
        ps += p[e] * s[e];
        cp += ce * p[e];
        csq += ce * ce;
        cmax = fmax(cmax, fabs(ce));
    }
    put_sum(r2sq, part, SC_R2SQ, sh);
    put_sum(ps, part, SC_PS, sh);
    put_sum(cp, part, SC_CP, sh);
    put_sum(csq, part, SC_CSQ, sh);
    put_max(cmax, part, SC_CMAX, sh);
}

// ------------------------------------------------------------------------ Schur setup
__global__ void theta_kernel(int64_t psi, const double *__restrict__ p, const double *__restrict__ s,
                             double *__restrict__ th, float *__restrict__ th32) {
    GRID_STRIDE(e, psi) {
        const double t = p[e] / s[e];
        th[e] = t;
        th32[e] = (float)t;
    }
}

// Connected components of the bipartite support graph (nodes: rows 0..m-1, columns m..m+n-1)
// by lock-free union-find: hooking always points the larger root at the smaller, so every
// root is the smallest node id of its component.
__device__ __forceinline__ int uf_find(int32_t *parent, int x) {
    int p = parent[x];
    while (p != x) {
        const int gp = parent[p];
        if (gp != p) parent[x] = gp;  // path halving (benign race: only moves to an ancestor)
        x = p;
        p = gp;
    }
    return x;
}

__global__ void uf_init_kernel(int nn, int32_t *parent) {
    GRID_STRIDE(v, nn) parent[v] = (int32_t)v;
}

__global__ void uf_hook_kernel(int64_t psi, int m, const int32_t *__restrict__ si, const int32_t *__restrict__ sj,
                               int32_t *parent) {
    GRID_STRIDE(e, psi) {
        int a = si[e], b = m + sj[e];
        for (int guard = 0; guard < (1 << 20); ++guard) {
            a = uf_find(parent, a);
            b = uf_find(parent, b);
            if (a == b) break;
            if (a < b) { int t = a; a = b; b = t; }
            if (atomicCAS(&parent[a], a, b) == a) break;
        }
    }
}

__global__ void uf_final_kernel(int nn, int32_t *parent) {
    GRID_STRIDE(v, nn) parent[v] = uf_find(parent, (int)v);
}

// SC_ONECOMP <- number of columns whose label differs from column 0's (0: one component)
__global__ void onecomp_kernel(int m, int n, const int32_t *__restrict__ parent, double *part) {
    __shared__ double sh[kT / 32];
    double diff = 0;
    const int l0 = parent[m];
    GRID_STRIDE(j, n) diff += parent[m + j] != l0 ? 1.0 : 0.0;
    put_sum(diff, part, SC_ONECOMP, sh);
}

// ------------------------------------------------------------------------ right-hand side
__global__ void g_kernel(int64_t psi, const double *__restrict__ th, const double *__restrict__ p,
                         const double *__restrict__ r2, const double *__restrict__ r3, double *__restrict__ g) {
    GRID_STRIDE(e, psi) {
        const double a = r2 ? r2[e] : 0.0;
        const double b = r3 ? r3[e] / p[e] : 0.0;
        g[e] = th[e] * (a - b);
    }
}

__global__ void sum_kernel(int n, const double *__restrict__ x, double *part, int slot) {
    __shared__ double sh[kT / 32];
    double t = 0;
    GRID_STRIDE(j, n) t += x[j];
    put_sum(t, part, slot, sh);
}

// one component: subtract the mean (scal[slot] / n)
__global__ void center_kernel(int n, double *__restrict__ x, const double *__restrict__ scal, int slot) {
    const double mean = scal[slot] / (double)n;
    GRID_STRIDE(j, n) x[j] -= mean;
}

// several components: per-label sums by atomics, then subtract the label mean
__global__ void comp_accum_kernel(int m, int n, const int32_t *__restrict__ parent, const double *__restrict__ x,
                                  double *comp_sum, double *comp_cnt) {
    GRID_STRIDE(j, n) {
        const int l = parent[m + j];
        atomicAdd(&comp_sum[l], x[j]);
        atomicAdd(&comp_cnt[l], 1.0);
    }
}
__global__ void comp_center_kernel(int m, int n, const int32_t *__restrict__ parent, double *__restrict__ x,
                                   const double *__restrict__ comp_sum, const double *__restrict__ comp_cnt) {
    GRID_STRIDE(j, n) {
        const int l = parent[m + j];
        x[j] -= comp_sum[l] / comp_cnt[l];
    }
}

// ------------------------------------------------------------------------ PCG on S_M
template <typename T>
struct PcgArgs {
    int m, n;
    const int32_t *rp, *sj, *cp, *crow;
    const T *th, *thc, *Minv, *Dinv;
    const T *b;
    T *x, *r, *z, *pa, *pb, *q, *w;   // pa / pb: double-buffered search direction
    double *part;  // 3 slots x gridDim
    unsigned *bar;
    int *err;
    double tol;
    int maxit;
    double *scal;  // SC_PCG_ITERS, SC_PCG_RELRES
    int *bnd;      // lane-group boundaries: rows at bnd[0 ..], columns at bnd[bnd_cap ..]
    int64_t bnd_cap;
};

constexpr int kPcgT = 512;   // threads per PCG block

// sum of `x` over the g lanes of an aligned lane group (g a power of two <= 32)
template <typename T>
__device__ __forceinline__ T group_sum(T x, int g) {
    for (int o = g >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// beta2_j = r1b_j + sum_i g_ij and rhs_j = beta2_j - sum_i theta_ij M_i^-1 beta1_i over the
// column's pairs, G lanes per column (warp-uniform trip counts: groups past the end contribute
// nothing but take part in the shuffles)
template <int G>
__global__ void rhs_group_kernel(int n, const int32_t *__restrict__ cp, const int32_t *__restrict__ perm,
                                 const int32_t *__restrict__ crow, const double *__restrict__ g,
                                 const double *__restrict__ thc, const double *__restrict__ Minv,
                                 const double *__restrict__ beta1, const double *__restrict__ r1b,
                                 double *__restrict__ beta2, double *__restrict__ rhs) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lg = threadIdx.x & (G - 1);
    const int64_t grp = tid / G, ngrp = stride / G, wgrp0 = (tid & ~(int64_t)31) / G;
    for (int64_t j0 = wgrp0; j0 < n; j0 += ngrp) {
        const int64_t j = j0 + (grp - wgrp0);
        double b2 = 0.0, vt = 0.0;
        if (j < n) {
            for (int k = cp[j] + lg; k < cp[j + 1]; k += G) {
                b2 += g[perm[k]];
                const int i = crow[k];
                vt += thc[k] * (Minv[i] * beta1[i]);
            }
        }
        b2 = group_sum(b2, G);
        vt = group_sum(vt, G);
        if (lg == 0 && j < n) {
            if (r1b) b2 += r1b[j];
            beta2[j] = b2;
            rhs[j] = b2 - vt;
        }
    }
}

// du_i = M_i^-1 (beta1_i - sum_j theta_ij dv_j), G lanes per row
template <int G>
__global__ void du_group_kernel(int m, const int32_t *__restrict__ rp, const int32_t *__restrict__ sj,
                                const double *__restrict__ th, const double *__restrict__ Minv,
                                const double *__restrict__ beta1, const double *__restrict__ dv,
                                double *__restrict__ du) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lg = threadIdx.x & (G - 1);
    const int64_t grp = tid / G, ngrp = stride / G, wgrp0 = (tid & ~(int64_t)31) / G;
    for (int64_t i0 = wgrp0; i0 < m; i0 += ngrp) {
        const int64_t i = i0 + (grp - wgrp0);
        double acc = 0.0;
        if (i < m)
            for (int e = rp[i] + lg; e < rp[i + 1]; e += G) acc += th[e] * dv[sj[e]];
        acc = group_sum(acc, G);
        if (lg == 0 && i < m) du[i] = Minv[i] * (beta1[i] - acc);
    }
}

// Lane-group forms (G lanes per row or column, warp-uniform trip counts; groups past the end take
// part in the shuffles with nothing) of the per-row / per-column loops of the residuals, of Theta's
// row and column sums and of beta1: one thread per row or column walked long rows serially.

// r1b_j = b_j - sum_i p_ij over the column, with the block partials of |r1b|^2 and |r1b|_1
template <int G>
__global__ void res_cols_group_kernel(int n, const int32_t *__restrict__ cp, const int32_t *__restrict__ perm,
                                      const double *__restrict__ p, const double *__restrict__ b,
                                      double *__restrict__ r1b, double *part) {
    __shared__ double sh[kT / 32];
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lg = threadIdx.x & (G - 1);
    const int64_t grp = tid / G, ngrp = stride / G, wgrp0 = (tid & ~(int64_t)31) / G;
    double sq = 0, l1 = 0;
    for (int64_t j0 = wgrp0; j0 < n; j0 += ngrp) {
        const int64_t j = j0 + (grp - wgrp0);
        double acc = 0.0;
        if (j < n)
            for (int k = cp[j] + lg; k < cp[j + 1]; k += G) acc += p[perm[k]];
        acc = group_sum(acc, G);
        if (lg == 0 && j < n) {
            const double r = b[j] - acc;
            r1b[j] = r;
            sq += r * r;
            l1 += fabs(r);
        }
    }
    put_sum(sq, part, SC_R1B_SQ, sh);
    put_sum(l1, part, SC_R1B_L1, sh);
}

// M_i = sum_j theta_ij, Minv; excl_ij = the sum of the OTHER entries of row i (a forward exclusive
// scan plus a backward one, never a subtraction, so a dominant theta does not cancel:
// S_jj = sum_i theta_ij excl_ij / M_i)
template <int G>
__global__ void theta_rows_group_kernel(int m, const int32_t *__restrict__ rp, const double *__restrict__ th,
                                        double *__restrict__ excl, double *__restrict__ M,
                                        double *__restrict__ Minv, float *__restrict__ Minv32) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lg = threadIdx.x & (G - 1);
    const int64_t grp = tid / G, ngrp = stride / G, wgrp0 = (tid & ~(int64_t)31) / G;
    const unsigned full = 0xffffffffu;
    for (int64_t i0 = wgrp0; i0 < m; i0 += ngrp) {
        const int64_t i = i0 + (grp - wgrp0);
        const int lo = i < m ? rp[i] : 0, hi = i < m ? rp[i + 1] : 0;
        // trips of the longest row among the warp's groups (every lane takes part in the shuffles)
        int trips = (hi - lo + G - 1) / G;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) trips = max(trips, __shfl_xor_sync(full, trips, o));
        double carry = 0.0;
        for (int c = 0; c < trips; ++c) {
            const int e = lo + c * G + lg;
            const double t = e < hi ? th[e] : 0.0;
            double x = t;
#pragma unroll
            for (int o = 1; o < G; o <<= 1) {
                const double y = __shfl_up_sync(full, x, o, G);
                if (lg >= o) x += y;
            }
            double ex = __shfl_up_sync(full, x, 1, G);
            ex = lg == 0 ? 0.0 : ex;
            if (e < hi) excl[e] = carry + ex;
            carry += __shfl_sync(full, x, G - 1, G);
        }
        __syncwarp();
        double suf = 0.0;
        for (int c = trips - 1; c >= 0; --c) {
            const int e = lo + c * G + lg;
            const double t = e < hi ? th[e] : 0.0;
            double x = t;
#pragma unroll
            for (int o = 1; o < G; o <<= 1) {
                const double y = __shfl_down_sync(full, x, o, G);
                if (lg + o < G) x += y;
            }
            double ex = __shfl_down_sync(full, x, 1, G);
            ex = lg == G - 1 ? 0.0 : ex;
            if (e < hi) excl[e] += suf + ex;
            suf += __shfl_sync(full, x, 0, G);
        }
        if (lg == 0 && i < m) {
            M[i] = carry;
            const double mi = carry > 0 ? 1.0 / carry : 0.0;
            Minv[i] = mi;
            Minv32[i] = (float)mi;
        }
    }
}

// theta in column order, N_j = the column's sum, the Jacobi diagonal of S_M
template <int G>
__global__ void theta_cols_group_kernel(int n, const int32_t *__restrict__ cp, const int32_t *__restrict__ perm,
                                        const int32_t *__restrict__ crow, const double *__restrict__ th,
                                        const double *__restrict__ excl, const double *__restrict__ Minv,
                                        double *__restrict__ thc, float *__restrict__ thc32, double *__restrict__ N,
                                        double *__restrict__ Dinv, float *__restrict__ Dinv32,
                                        double *__restrict__ Sdiag) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lg = threadIdx.x & (G - 1);
    const int64_t grp = tid / G, ngrp = stride / G, wgrp0 = (tid & ~(int64_t)31) / G;
    for (int64_t j0 = wgrp0; j0 < n; j0 += ngrp) {
        const int64_t j = j0 + (grp - wgrp0);
        double nsum = 0, d = 0;
        if (j < n)
            for (int k = cp[j] + lg; k < cp[j + 1]; k += G) {
                const int e = perm[k];
                const double t = th[e];
                thc[k] = t;
                thc32[k] = (float)t;
                nsum += t;
                d += t * excl[e] * Minv[crow[k]];
            }
        nsum = group_sum(nsum, G);
        d = group_sum(d, G);
        if (lg == 0 && j < n) {
            N[j] = nsum;
            Sdiag[j] = d;
            const double di = d > 0 ? 1.0 / d : 0.0;  // columns with D = 0 are private stars: masked
            Dinv[j] = di;
            Dinv32[j] = (float)di;
        }
    }
}

// beta1_i = r1a_i + sum_j g_ij over the row
template <int G>
__global__ void beta1_group_kernel(int m, const int32_t *__restrict__ rp, const double *__restrict__ g,
                                   const double *__restrict__ r1a, double *__restrict__ beta1) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lg = threadIdx.x & (G - 1);
    const int64_t grp = tid / G, ngrp = stride / G, wgrp0 = (tid & ~(int64_t)31) / G;
    for (int64_t i0 = wgrp0; i0 < m; i0 += ngrp) {
        const int64_t i = i0 + (grp - wgrp0);
        double acc = 0.0;
        if (i < m)
            for (int e = rp[i] + lg; e < rp[i + 1]; e += G) acc += g[e];
        acc = group_sum(acc, G);
        if (lg == 0 && i < m) beta1[i] = acc + (r1a ? r1a[i] : 0.0);
    }
}

// every block sums the gridDim partials of `slots` (fixed order: deterministic, identical in
// all blocks); warp 0 does it, lanes taking strided partials
__device__ __forceinline__ void sum_partials(const double *part, unsigned G, int nslots, double *out_sh) {
    if (threadIdx.x < 32) {
        for (int s = 0; s < nslots; ++s) {
            double a = 0;
            for (unsigned k = threadIdx.x; k < G; k += 32) a += part[(int64_t)s * G + k];
            a = warp_sum(a);
            if (threadIdx.x == 0) out_sh[s] = a;
        }
    }
    __syncthreads();
}

// Jacobi-preconditioned CG on S_M, persistent cooperative kernel.  Rows and columns are handled
// by lane groups of g threads (g ~ the average row/column length), each group a contiguous range
// of rows (and one of columns) of equal weight, pairs + g per row (the per-row reduction costs
// about one trip): group q starts at the first row i with rp[i] + g i >= q (psi + g m) / ngrp.
// Contiguous ranges keep neighbouring pixels together (the gathers stay local) and bound a group's
// excess over the mean by one row.  With p_k = z_k + beta_k p_{k-1}
// formed on the fly from z and the previous direction (double buffer), one iteration is
//   row pass:    w_i = M_i^-1 sum_j theta_ij p_j                                   | barrier
//   column pass: p_j stored; q_j = sum_i theta_ij (p_j - w_i); partial p.q           | barrier
//   update:      alpha = rz/pq; x += alpha p; r -= alpha q; z = D^-1 r; partial r.z, r.r | barrier
// Dot products are accumulated in double in every precision.
template <typename T>
__global__ void __launch_bounds__(kPcgT) pcg_kernel(PcgArgs<T> A, int g) {
    __shared__ double sh[kPcgT / 32];
    __shared__ double s_val[3];
    const unsigned G = gridDim.x;
    const int n = A.n, m = A.m;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)G * blockDim.x;
    const int lg = threadIdx.x & (g - 1);                 // lane within its group
    const int64_t grp = tid / g, ngrp = stride / g;
    double *P0 = A.part, *P1 = A.part + G, *P2 = A.part + 2 * G;

    // the group boundaries (lane 0 of each group searches its own; group 0 also writes the ends)
    if (lg == 0) {
        const int64_t dr = (int64_t)A.rp[m] + (int64_t)g * m, dc = (int64_t)A.cp[n] + (int64_t)g * n;
        const int64_t tr = grp * dr / ngrp, tc = grp * dc / ngrp;
        int64_t lo = 0, hi = m;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)A.rp[mid] + (int64_t)g * mid >= tr) hi = mid; else lo = mid + 1;
        }
        A.bnd[grp] = (int)lo;
        lo = 0;
        hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)A.cp[mid] + (int64_t)g * mid >= tc) hi = mid; else lo = mid + 1;
        }
        A.bnd[A.bnd_cap + grp] = (int)lo;
        if (grp == 0) {
            A.bnd[ngrp] = m;
            A.bnd[A.bnd_cap + ngrp] = n;
        }
    }
    double bb = 0, rz = 0;
    for (int64_t j = tid; j < n; j += stride) {
        const T bj = A.b[j];
        A.x[j] = (T)0;
        A.r[j] = bj;
        const T zj = A.Dinv[j] * bj;
        A.z[j] = zj;
        A.pa[j] = (T)0;
        bb += (double)bj * (double)bj;
        rz += (double)bj * (double)zj;
    }
    {
        double s0 = block_sum(bb, sh), s1 = block_sum(rz, sh);
        if (threadIdx.x == 0) { P0[blockIdx.x] = s0; P1[blockIdx.x] = s1; }
    }
    if (!grid_barrier(A.bar, G, A.err)) return;
    sum_partials(A.part, G, 2, s_val);
    bb = s_val[0];
    rz = s_val[1];
    const double tol2 = A.tol * A.tol * bb;
    // this group's rows [r0, r0 + nr) and columns [c0, c0 + nc); trip counts uniform over the warp
    const int r0 = A.bnd[grp], nr = A.bnd[grp + 1] - r0;
    const int c0 = A.bnd[A.bnd_cap + grp], nc = A.bnd[A.bnd_cap + grp + 1] - c0;
    const int rtrips = __reduce_max_sync(0xffffffffu, nr), ctrips = __reduce_max_sync(0xffffffffu, nc);
    int it = 0;
    double rr = bb;
    T beta = (T)0;
    T *pprev = A.pa, *pcur = A.pb;
    if (bb > 0.0 && rz > 0.0) {
        for (it = 0; it < A.maxit;) {
            // row pass with p = z + beta pprev (the trip count is uniform across a warp: groups
            // past their range contribute zero but still take part in the shuffles)
            // two rows per group and trip (rows i and i + 1), their loads interleaved: the
            // passes are bound by the latency of the index -> gather chains, not by bandwidth
            for (int t = 0; t < rtrips; t += 2) {
                const int ia = r0 + t, ib = ia + 1;
                const bool va = t < nr, vb = t + 1 < nr;
                T acca = (T)0, accb = (T)0;
                int ea = 0, ha = 0, eb = 0, hb = 0;
                if (va) { ea = A.rp[ia] + lg; ha = A.rp[ia + 1]; }
                if (vb) { eb = A.rp[ib] + lg; hb = A.rp[ib + 1]; }
                while (ea < ha || eb < hb) {
                    if (ea < ha) {
                        const int j = A.sj[ea];
                        acca += A.th[ea] * (A.z[j] + beta * pprev[j]);
                        ea += g;
                    }
                    if (eb < hb) {
                        const int j = A.sj[eb];
                        accb += A.th[eb] * (A.z[j] + beta * pprev[j]);
                        eb += g;
                    }
                }
                acca = group_sum(acca, g);
                accb = group_sum(accb, g);
                if (lg == 0 && va) A.w[ia] = A.Minv[ia] * acca;
                if (lg == 0 && vb) A.w[ib] = A.Minv[ib] * accb;
            }
            if (!grid_barrier(A.bar, G, A.err)) return;
            // column pass (two columns per group and trip)
            double pq = 0;
            for (int t = 0; t < ctrips; t += 2) {
                const int ja = c0 + t, jb = ja + 1;
                const bool va = t < nc, vb = t + 1 < nc;
                T pa = (T)0, pb2 = (T)0, acca = (T)0, accb = (T)0;
                int ka = 0, ha = 0, kb = 0, hb = 0;
                if (va) { pa = A.z[ja] + beta * pprev[ja]; ka = A.cp[ja] + lg; ha = A.cp[ja + 1]; }
                if (vb) { pb2 = A.z[jb] + beta * pprev[jb]; kb = A.cp[jb] + lg; hb = A.cp[jb + 1]; }
                while (ka < ha || kb < hb) {
                    if (ka < ha) {
                        acca += A.thc[ka] * (pa - A.w[A.crow[ka]]);
                        ka += g;
                    }
                    if (kb < hb) {
                        accb += A.thc[kb] * (pb2 - A.w[A.crow[kb]]);
                        kb += g;
                    }
                }
                acca = group_sum(acca, g);
                accb = group_sum(accb, g);
                if (lg == 0 && va) {
                    A.q[ja] = acca;
                    pcur[ja] = pa;
                    pq += (double)pa * (double)acca;
                }
                if (lg == 0 && vb) {
                    A.q[jb] = accb;
                    pcur[jb] = pb2;
                    pq += (double)pb2 * (double)accb;
                }
            }
            {
                double s0 = block_sum(pq, sh);
                if (threadIdx.x == 0) P0[blockIdx.x] = s0;
            }
            if (!grid_barrier(A.bar, G, A.err)) return;
            sum_partials(A.part, G, 1, s_val);
            pq = s_val[0];
            if (!(pq > 0.0)) break;  // breakdown (exact zero direction or loss of definiteness)
            const double alpha = rz / pq;
            double rzn = 0, rrn = 0;
            for (int64_t j = tid; j < n; j += stride) {
                const T pj = pcur[j];
                const T rj = A.r[j] - (T)alpha * A.q[j];
                const T zj = A.Dinv[j] * rj;
                A.x[j] += (T)alpha * pj;
                A.r[j] = rj;
                A.z[j] = zj;
                rzn += (double)rj * (double)zj;
                rrn += (double)rj * (double)rj;
            }
            {
                double s1 = block_sum(rzn, sh), s2 = block_sum(rrn, sh);
                if (threadIdx.x == 0) { P1[blockIdx.x] = s1; P2[blockIdx.x] = s2; }
            }
            if (!grid_barrier(A.bar, G, A.err)) return;
            sum_partials(A.part + G, G, 2, s_val + 1);
            rzn = s_val[1];
            rr = s_val[2];
            ++it;
            if (rr <= tol2 || !(rzn > 0.0)) break;
            beta = (T)(rzn / rz);
            rz = rzn;
            T *t = pprev; pprev = pcur; pcur = t;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.scal[SC_PCG_ITERS] = (double)it;
        A.scal[SC_PCG_RELRES] = bb > 0 ? sqrt(rr / bb) : 0.0;
    }
}

// ---- cluster variant (FP32).  One thread-block cluster of R CTAs (16 where the GPC allows it)
// runs the whole CG.  CTA r owns a contiguous slice of the rows and one of the columns of S_M
// (balanced on pairs + rows / columns, never more than 2*ceil(m/R)+1 rows or 2*ceil(n/R)+1
// columns), keeps its slices of theta and of the indices in shared memory (a tail that does not
// fit is read from global memory), and every CTA keeps full copies of the direction p, the
// preconditioned residual z and w = M^{-1} V p in shared memory.  A CTA pushes the w / z entries
// it computes into every CTA's copy with distributed-shared-memory stores, and the hardware
// cluster barrier (release / acquire at cluster scope) publishes them together with the partial
// dot products.  Three barriers per iteration, no spin loop: the CTAs of a cluster are
// co-scheduled, and every CTA takes the same branch decisions because it sums the same partials
// in the same order.
constexpr int kClT = 1024;
constexpr int kClMaxR = 16;

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_addr(const void *local, unsigned rank) {
    uint32_t ra;
    const uint32_t la = (uint32_t)__cvta_generic_to_shared(local);
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(rank));
    return ra;
}

__device__ __forceinline__ void st_cluster(uint32_t addr, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

__device__ __forceinline__ float ld_cluster(uint32_t addr) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
}

// Sums shared slots [0, ns) over the R CTAs (R <= 32): lane q of warp 0 reads CTA q's slots, a
// fixed xor-shuffle tree adds them (the same order in every CTA, so every CTA gets the same bits),
// and the sums land in out[0, ns) for the whole block.
__device__ __forceinline__ void cluster_reduce(const float *slots, int ns, unsigned R, float *out) {
    if (threadIdx.x < 32) {
        const unsigned lane = threadIdx.x;
        float v[3];
#pragma unroll
        for (int s = 0; s < 3; ++s)
            v[s] = (s < ns && lane < R) ? ld_cluster(cluster_addr(&slots[s], lane)) : 0.f;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            float x = v[s];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0 && s < ns) out[s] = x;
        }
    }
    __syncthreads();
}

// Slice boundary r of R over [0, cnt]: the first index whose weight ptr[i] + i reaches
// r*(ptr[cnt] + cnt)/R, clamped to within ceil(cnt/(2R)) of r*cnt/R.  Monotone in r, so the
// slices tile [0, cnt) and none is longer than 2*ceil(cnt/R) + 1.  Block-wide (every thread gets
// the result); `sh` holds kClT/32 ints.
__device__ __forceinline__ int slice_bound(const int32_t *ptr, int cnt, int r, int R, int *sh) {
    if (r <= 0) return 0;
    if (r >= R) return cnt;
    const int64_t total = (int64_t)ptr[cnt] + cnt;
    const int64_t target = total * r / R;
    int c = 0;  // number of i in [0, cnt] with weight below target (weights strictly increase)
    for (int i = threadIdx.x; i <= cnt; i += blockDim.x) c += ((int64_t)ptr[i] + i < target) ? 1 : 0;
    c = block_sum(c, sh);
    if (threadIdx.x == 0) sh[0] = c;
    __syncthreads();
    c = sh[0];
    __syncthreads();
    const int mid = (int)((int64_t)cnt * r / R), h = (cnt + 2 * R - 1) / (2 * R);
    return max(0, min(cnt, min(mid + h, max(mid - h, c))));
}

struct ClLayout {
    int64_t bytes;              // fixed part (vectors, slice pointers)
    int ncap, mcap;             // own columns / rows at most
};

__host__ __device__ inline ClLayout cl_layout(int m, int n, int R) {
    ClLayout L;
    L.ncap = 2 * ((n + R - 1) / R) + 2;
    L.mcap = 2 * ((m + R - 1) / R) + 2;
    // p, z (n each), w (m), own x, r, q, Dinv (ncap each), own Minv (mcap), slice pointers
    L.bytes = 4 * ((int64_t)2 * n + m + 4 * (int64_t)L.ncap + L.mcap) + 4 * ((int64_t)L.ncap + L.mcap + 2);
    L.bytes = (L.bytes + 15) & ~(int64_t)15;
    return L;
}

__global__ void __launch_bounds__(kClT, 1) pcg_cluster_kernel(PcgArgs<float> A, int g, int smem_bytes) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ float sh[kClT / 32];
    __shared__ int shi[kClT / 32];
    __shared__ float s_part[6];  // 0: p.q  1: r.z  2: r.r  3, 4: b.b, b.z at the start
    __shared__ float s_sum[3];
    const int R = (int)gridDim.x;  // the grid is exactly one cluster
    const int m = A.m, n = A.n;
    const ClLayout L = cl_layout(m, n, R);
    float *p_full = (float *)dsm, *z_full = p_full + n, *w_full = z_full + n;
    float *x_o = w_full + m, *r_o = x_o + L.ncap, *q_o = r_o + L.ncap, *d_o = q_o + L.ncap;
    float *minv_o = d_o + L.ncap;
    int32_t *rp_o = (int32_t *)(minv_o + L.mcap), *cp_o = rp_o + L.mcap + 1;
    unsigned char *ent = dsm + L.bytes;

    const int rank = (int)blockIdx.x;
    const int r0 = slice_bound(A.rp, m, rank, R, shi), r1 = slice_bound(A.rp, m, rank + 1, R, shi);
    const int c0 = slice_bound(A.cp, n, rank, R, shi), c1 = slice_bound(A.cp, n, rank + 1, R, shi);
    const int nr = r1 - r0, nc = c1 - c0;
    const int e0 = A.rp[r0], ne_r = A.rp[r1] - e0;
    const int k0 = A.cp[c0], ne_c = A.cp[c1] - k0;
    // entries kept in shared memory: all when they fit, else the same share of each slice
    const int64_t room = ((int64_t)smem_bytes - L.bytes) / 8;  // theta (4 B) + index (4 B)
    int cap_r = ne_r, cap_c = ne_c;
    if ((int64_t)ne_r + ne_c > room) {
        cap_r = (int)(room * ne_r / max(1, ne_r + ne_c));
        cap_c = (int)(room - cap_r);
        cap_c = min(cap_c, ne_c);
    }
    float *th_s = (float *)ent, *thc_s = th_s + cap_r;
    int32_t *sj_s = (int32_t *)(thc_s + cap_c), *crow_s = sj_s + cap_r;
    const float *__restrict__ th_g = A.th + e0;
    const float *__restrict__ thc_g = A.thc + k0;
    const int32_t *__restrict__ sj_g = A.sj + e0;
    const int32_t *__restrict__ crow_g = A.crow + k0;

    // every CTA of the cluster must be running before any distributed-shared-memory access
    cluster_sync();
    for (int t = threadIdx.x; t <= nr; t += blockDim.x) rp_o[t] = A.rp[r0 + t] - e0;
    for (int t = threadIdx.x; t <= nc; t += blockDim.x) cp_o[t] = A.cp[c0 + t] - k0;
    for (int t = threadIdx.x; t < nr; t += blockDim.x) minv_o[t] = A.Minv[r0 + t];
    for (int t = threadIdx.x; t < cap_r; t += blockDim.x) {
        th_s[t] = th_g[t];
        sj_s[t] = sj_g[t];
    }
    for (int t = threadIdx.x; t < cap_c; t += blockDim.x) {
        thc_s[t] = thc_g[t];
        crow_s[t] = crow_g[t];
    }
    float bb = 0.f, bz = 0.f;
    for (int t = threadIdx.x; t < nc; t += blockDim.x) {
        const int j = c0 + t;
        const float bj = A.b[j], dj = A.Dinv[j], zj = dj * bj;
        x_o[t] = 0.f;
        r_o[t] = bj;
        d_o[t] = dj;
        for (int q = 0; q < R; ++q) st_cluster(cluster_addr(&z_full[j], q), zj);
        bb += bj * bj;
        bz += bj * zj;
    }
    {
        const float s3 = block_sum(bb, sh), s4 = block_sum(bz, sh);
        if (threadIdx.x == 0) { s_part[3] = s3; s_part[4] = s4; }
    }
    cluster_sync();
    cluster_reduce(&s_part[3], 2, R, s_sum);
    bb = s_sum[0];
    float rz = s_sum[1];
    for (int j = threadIdx.x; j < n; j += blockDim.x) p_full[j] = z_full[j];
    __syncthreads();

    const double tol2 = A.tol * A.tol * (double)bb;
    const int lg = threadIdx.x & (g - 1);
    const int grp = threadIdx.x / g, ngrp = blockDim.x / g;
    const int wgrp0 = (threadIdx.x & ~31) / g;
    int it = 0;
    double rr = (double)bb;
    if (bb > 0.f && rz > 0.f) {
        for (it = 0; it < A.maxit;) {
            // w_i = M_i^{-1} sum_j theta_ij p_j over the own rows; pushed to every CTA
            for (int i0 = wgrp0; i0 < nr; i0 += ngrp) {
                const int il = i0 + (grp - wgrp0);
                float acc = 0.f;
                if (il < nr) {
                    const int lo = rp_o[il], hi = rp_o[il + 1];
                    for (int e = lo + lg; e < hi; e += g) {
                        const bool in = e < cap_r;
                        const int j = in ? sj_s[e] : sj_g[e];
                        const float t = in ? th_s[e] : th_g[e];
                        acc += t * p_full[j];
                    }
                }
                acc = group_sum(acc, g);
                if (il < nr) {
                    const float wi = minv_o[il] * acc;
                    for (int q = lg; q < R; q += g) st_cluster(cluster_addr(&w_full[r0 + il], q), wi);
                }
            }
            cluster_sync();
            // q_j = sum_i theta_ij (p_j - w_i) over the own columns
            float pq = 0.f;
            for (int j0 = wgrp0; j0 < nc; j0 += ngrp) {
                const int jl = j0 + (grp - wgrp0);
                float acc = 0.f, pj = 0.f;
                if (jl < nc) {
                    pj = p_full[c0 + jl];
                    const int lo = cp_o[jl], hi = cp_o[jl + 1];
                    for (int k = lo + lg; k < hi; k += g) {
                        const bool in = k < cap_c;
                        const int i = in ? crow_s[k] : crow_g[k];
                        const float t = in ? thc_s[k] : thc_g[k];
                        acc += t * (pj - w_full[i]);
                    }
                }
                acc = group_sum(acc, g);
                if (lg == 0 && jl < nc) {
                    q_o[jl] = acc;
                    pq += pj * acc;
                }
            }
            {
                const float s0 = block_sum(pq, sh);
                if (threadIdx.x == 0) s_part[0] = s0;
            }
            cluster_sync();
            cluster_reduce(&s_part[0], 1, R, s_sum);
            pq = s_sum[0];
            if (!(pq > 0.f)) break;
            const float alpha = rz / pq;
            float rzn = 0.f, rrn = 0.f;
            for (int t = threadIdx.x; t < nc; t += blockDim.x) {
                const int j = c0 + t;
                const float rj = r_o[t] - alpha * q_o[t];
                const float zj = d_o[t] * rj;
                x_o[t] += alpha * p_full[j];
                r_o[t] = rj;
                for (int q = 0; q < R; ++q) st_cluster(cluster_addr(&z_full[j], q), zj);
                rzn += rj * zj;
                rrn += rj * rj;
            }
            {
                const float s1 = block_sum(rzn, sh), s2 = block_sum(rrn, sh);
                if (threadIdx.x == 0) { s_part[1] = s1; s_part[2] = s2; }
            }
            cluster_sync();
            cluster_reduce(&s_part[1], 2, R, s_sum);
            rzn = s_sum[0];
            rr = (double)s_sum[1];
            ++it;
            if (rr <= tol2 || !(rzn > 0.f)) break;
            const float beta = rzn / rz;
            rz = rzn;
            for (int j = threadIdx.x; j < n; j += blockDim.x) p_full[j] = z_full[j] + beta * p_full[j];
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < nc; t += blockDim.x) A.x[c0 + t] = x_o[t];
    // no CTA may exit while another can still read its shared memory
    cluster_sync();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.scal[SC_PCG_ITERS] = (double)it;
        A.scal[SC_PCG_RELRES] = bb > 0.f ? sqrt(rr / (double)bb) : 0.0;
    }
}

template <typename T>
Error launch_pcg(Newton &W, const Support &S, const T *th, const T *thc, const T *Minv, const T *Dinv,
                 const T *b, T *x, T *r, T *z, T *p, T *q, T *w, double tol, int maxit, cudaStream_t st) {
    int per_sm = 0;
    OT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_kernel<T>, kPcgT, 0));
    // lane-group size ~ half the average row length (power of two)
    const double avg = (double)std::max<int64_t>(S.psi, 1) / (double)std::max(W.m, 1);
    // (at most 16: measured at 256^2 with 33 pairs per row, 16 lanes beat 32 by 8 %)
    int g = 1;
    while (g < 16 && 2 * g <= avg) g <<= 1;
    const int64_t threads = (int64_t)std::max(W.m, W.n) * g;
    const int maxg = std::max(1, per_sm) * W.num_sms;
    int G = W.pcg_grid > 0 ? W.pcg_grid : (int)std::max<int64_t>(1, ceil_div(threads, kPcgT));
    G = std::min(G, std::min(maxg, kMaxPartBlocks / 3));
    // the boundary arrays hold ngrp + 1 = G kPcgT / g + 1 entries per half
    G = (int)std::min<int64_t>(G, std::max<int64_t>(1, (W.pcg_bnd_cap - 1) * g / kPcgT));
    OT_CUDA(cudaMemsetAsync(W.bar, 0, 2 * sizeof(unsigned), st));
    OT_CUDA(cudaMemsetAsync(W.err, 0, sizeof(int), st));
    T *pb = (T *)W.pcg_pb;
    if (sizeof(T) == 4) pb = (T *)W.pcg_pb32;
    PcgArgs<T> A{W.m, W.n, S.row_ptr, S.j, S.col_ptr, S.col_row, th, thc, Minv, Dinv, b, x, r, z, p, pb, q, w,
                 W.part, W.bar, W.err, tol, maxit, W.scal, W.pcg_bnd, W.pcg_bnd_cap};
    const int kid = sizeof(T) == 8 ? KT_PCG64 : KT_PCG32;
    const int R = W.pcg_cluster;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (W.verbose >= 3) {
        OT_CUDA(cudaEventCreate(&ev[0]));
        OT_CUDA(cudaEventCreate(&ev[1]));
        OT_CUDA(cudaEventRecord(ev[0], st));
    }
    const ClLayout L = cl_layout(W.m, W.n, std::max(R, 1));
    bool clustered = false;
    if constexpr (sizeof(T) == 4) {
      if (R > 1 && 2 * L.bytes <= W.pcg_cluster_smem) {
        clustered = true;
        // one thread-block cluster with the operator slices in shared memory
        int gc = 1;
        while (gc < 32 && 2 * gc <= avg) gc <<= 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(R);
        cfg.blockDim = dim3(kClT);
        cfg.dynamicSmemBytes = (size_t)W.pcg_cluster_smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = R;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const int sb = W.pcg_cluster_smem;
        ktimer_begin(kid, st);
        OT_CUDA(cudaLaunchKernelEx(&cfg, pcg_cluster_kernel, A, gc, sb));
        OT_LAUNCHED();
        ktimer_end(kid, st);
      }
    }
    if (!clustered) {
        void *args[] = {&A, &g};
        ktimer_begin(kid, st);
        OT_CUDA(cudaLaunchCooperativeKernel((void *)pcg_kernel<T>, dim3(G), dim3(kPcgT), args, 0, st));
        OT_LAUNCHED();
        ktimer_end(kid, st);
    }
    if (W.verbose >= 3) {
        float ms = 0.f;
        OT_CUDA(cudaEventRecord(ev[1], st));
        OT_CUDA(cudaEventSynchronize(ev[1]));
        OT_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
        W.last_pcg_ms = ms;
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
    }
    // algorithmic bytes of one CG iteration: both passes read theta, an index and a gathered
    // vector entry per support pair, plus the per-row / per-column vectors
    W.pcg_bytes_per_iter = (double)S.psi * 2.0 * (2.0 * sizeof(T) + 4.0) + (double)W.m * (3.0 * 4.0 + 2.0 * sizeof(T)) +
                           (double)W.n * (2.0 * 4.0 + 12.0 * sizeof(T));
    return ok();
}

// ------------------------------------------------------------------------ FP64 matvec / refinement
__global__ void mv_rows_kernel(int m, const int32_t *__restrict__ rp, const int32_t *__restrict__ sj,
                               const double *__restrict__ th, const double *__restrict__ Minv,
                               const double *__restrict__ x, double *__restrict__ w) {
    GRID_STRIDE(i, m) {
        double acc = 0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) acc += th[e] * x[sj[e]];
        w[i] = Minv[i] * acc;
    }
}

// res = rhs - S_M x ; partial ||res||^2
__global__ void mv_cols_res_kernel(int n, const int32_t *__restrict__ cp, const int32_t *__restrict__ crow,
                                   const double *__restrict__ thc, const double *__restrict__ w,
                                   const double *__restrict__ x, const double *__restrict__ rhs,
                                   double *__restrict__ res, double *part) {
    __shared__ double sh[kT / 32];
    double sq = 0;
    GRID_STRIDE(j, n) {
        const double xj = x[j];
        double acc = 0;
        for (int k = cp[j]; k < cp[j + 1]; ++k) acc += thc[k] * (xj - w[crow[k]]);
        const double r = rhs[j] - acc;
        res[j] = r;
        sq += r * r;
    }
    put_sum(sq, part, SC_NORM_A, sh);
}

__global__ void norm_kernel(int n, const double *__restrict__ x, double *part, int slot) {
    __shared__ double sh[kT / 32];
    double sq = 0;
    GRID_STRIDE(j, n) sq += x[j] * x[j];
    put_sum(sq, part, slot, sh);
}

__global__ void to_f32_kernel(int n, const double *__restrict__ x, float *__restrict__ y) {
    GRID_STRIDE(j, n) y[j] = (float)x[j];
}

__global__ void axpy_f32_kernel(int n, const float *__restrict__ d, double *__restrict__ x) {
    GRID_STRIDE(j, n) x[j] += (double)d[j];
}

__global__ void copy_kernel(int n, const double *__restrict__ a, double *__restrict__ b) {
    GRID_STRIDE(j, n) b[j] = a[j];
}

// ------------------------------------------------------------------------ back-substitution

__global__ void dsdp_kernel(int64_t psi, const int32_t *__restrict__ si, const int32_t *__restrict__ sj,
                            const double *__restrict__ p, const double *__restrict__ s,
                            const double *__restrict__ r2, const double *__restrict__ r3,
                            const double *__restrict__ du, const double *__restrict__ dv,
                            double *__restrict__ ds, double *__restrict__ dp) {
    GRID_STRIDE(e, psi) {
        const double d = (r2 ? r2[e] : 0.0) - du[si[e]] - dv[sj[e]];
        ds[e] = d;
        dp[e] = ((r3 ? r3[e] : 0.0) - p[e] * d) / s[e];
    }
}

// ------------------------------------------------------------------------ steps etc.
__global__ void ratio_kernel(int64_t psi, const double *__restrict__ p, const double *__restrict__ dp,
                             const double *__restrict__ s, const double *__restrict__ ds, double *part) {
    __shared__ double sh[kT / 32];
    double rp = INFINITY, rs = INFINITY;
    GRID_STRIDE(e, psi) {
        if (dp[e] < 0) rp = fmin(rp, -p[e] / dp[e]);
        if (ds[e] < 0) rs = fmin(rs, -s[e] / ds[e]);
    }
    put_min(rp, part, SC_AP, sh);
    put_min(rs, part, SC_AS, sh);
}

__global__ void trial_kernel(int64_t psi, const double *__restrict__ p, const double *__restrict__ dp,
                             const double *__restrict__ s, const double *__restrict__ ds, double ap, double as,
                             double *part) {
    __shared__ double sh[kT / 32];
    double acc = 0;
    GRID_STRIDE(e, psi) acc += (p[e] + ap * dp[e]) * (s[e] + as * ds[e]);
    put_sum(acc, part, SC_MUAFF, sh);
}

__global__ void corr_r3_kernel(int64_t psi, const double *__restrict__ p, const double *__restrict__ s,
                               const double *__restrict__ dpa, const double *__restrict__ dsa, double smu,
                               double *__restrict__ r3) {
    GRID_STRIDE(e, psi) r3[e] = smu - p[e] * s[e] - (dpa ? dpa[e] * dsa[e] : 0.0);
}

__global__ void centr_r3_kernel(int64_t psi, const double *__restrict__ p, const double *__restrict__ s,
                                const double *__restrict__ dp, const double *__restrict__ ds, double tp,
                                double ts, double lo, double hi, double *__restrict__ r3) {
    GRID_STRIDE(e, psi) {
        const double vv = (p[e] + tp * dp[e]) * (s[e] + ts * ds[e]);
        double t = fmin(fmax(vv, lo), hi) - vv;
        r3[e] = fmax(t, -hi);
    }
}

__global__ void add_kernel(int64_t count, double *__restrict__ x, const double *__restrict__ y) {
    GRID_STRIDE(k, count) x[k] += y[k];
}

__global__ void step_entries_kernel(int64_t psi, double *__restrict__ p, double *__restrict__ s,
                                    const double *__restrict__ dp, const double *__restrict__ ds, double ap,
                                    double as, double *part) {
    __shared__ double sh[kT / 32];
    double acc = 0;
    GRID_STRIDE(e, psi) {
        const double pn = p[e] + ap * dp[e], sn = s[e] + as * ds[e];
        p[e] = pn;
        s[e] = sn;
        acc += pn * sn;
    }
    put_sum(acc, part, SC_PSNEW, sh);
}

__global__ void axpy_kernel(int64_t count, double a, const double *__restrict__ y, double *__restrict__ x) {
    GRID_STRIDE(k, count) x[k] += a * y[k];
}


__global__ void dot_kernel(int n, const double *__restrict__ a, const double *__restrict__ b, double *part,
                           int slot) {
    __shared__ double sh[kT / 32];
    double t = 0;
    GRID_STRIDE(j, n) t += a[j] * b[j];
    put_sum(t, part, slot, sh);
}

// p = z + b p   (b = 0 starts the recurrence)
__global__ void pcg_dir_kernel(int n, double b, const double *__restrict__ z, double *__restrict__ p) {
    GRID_STRIDE(j, n) p[j] = z[j] + b * p[j];
}

// sum of the nb stage-1 partials of `slot`, in the same order in every block; all threads get it
__device__ __forceinline__ double sum_slot(const double *part, int slot, int nb, double *sh, double *bc) {
    double a = 0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) a += part[(int64_t)slot * kMaxPartBlocks + k];
    a = block_sum(a, sh);
    if (threadIdx.x == 0) *bc = a;
    __syncthreads();
    const double r = *bc;
    __syncthreads();
    return r;
}

// S_M x in FP64 with G lanes per row / column (coalesced entry reads); warps take row groups with
// a uniform trip count so the shuffles always see full warps
template <int G>
__global__ void mvg_rows_kernel(int m, const int32_t *__restrict__ rp, const int32_t *__restrict__ sj,
                                const double *__restrict__ th, const double *__restrict__ Minv,
                                const double *__restrict__ x, double *__restrict__ w) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lg = threadIdx.x & (G - 1);
    const int64_t grp = t / G, ngrp = (int64_t)gridDim.x * blockDim.x / G, g0 = (t & ~(int64_t)31) / G;
    for (int64_t i0 = g0; i0 < m; i0 += ngrp) {
        const int64_t i = i0 + (grp - g0);
        double acc = 0;
        if (i < m)
            for (int e = rp[i] + lg; e < rp[i + 1]; e += G) acc += th[e] * x[sj[e]];
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lg == 0 && i < m) w[i] = Minv[i] * acc;
    }
}

template <int G>
__global__ void mvg_cols_kernel(int n, const int32_t *__restrict__ cp, const int32_t *__restrict__ crow,
                                const double *__restrict__ thc, const double *__restrict__ w,
                                const double *__restrict__ x, double *__restrict__ y, double *part) {
    __shared__ double sh[kT / 32];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lg = threadIdx.x & (G - 1);
    const int64_t grp = t / G, ngrp = (int64_t)gridDim.x * blockDim.x / G, g0 = (t & ~(int64_t)31) / G;
    double xy = 0;
    for (int64_t j0 = g0; j0 < n; j0 += ngrp) {
        const int64_t j = j0 + (grp - g0);
        double acc = 0, xj = 0;
        if (j < n) {
            xj = x[j];
            for (int k = cp[j] + lg; k < cp[j + 1]; k += G) acc += thc[k] * (xj - w[crow[k]]);
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lg == 0 && j < n) {
            y[j] = acc;
            xy += xj * acc;
        }
    }
    put_sum(xy, part, SC_SUM_A, sh);
}

// x += a p, r -= a q with a = r.z / p.q: p.q reduced here from its partials (nbq of them), r.z
// read from its scalar slot; block 0 records p.q; partial r.r
__global__ void dcg_step2_kernel(int n, int nbq, double *__restrict__ scal, int rz_slot, const double *__restrict__ p,
                                 const double *__restrict__ q, double *__restrict__ x, double *__restrict__ r,
                                 double *part) {
    __shared__ double sh[kT / 32];
    __shared__ double bc;
    const double pq = sum_slot(part, SC_SUM_A, nbq, sh, &bc);
    const double rz = scal[rz_slot];
    if (blockIdx.x == 0 && threadIdx.x == 0) scal[SC_SUM_A] = pq;
    const double a = (pq > 0 && rz > 0) ? rz / pq : 0.0;
    double rr = 0;
    GRID_STRIDE(j, n) {
        x[j] += a * p[j];
        const double rj = r[j] - a * q[j];
        r[j] = rj;
        rr += rj * rj;
    }
    put_sum(rr, part, SC_NORM_A, sh);
}

// p = z + b p with b = r.z(new) / r.z(old): r.z(new) reduced here (nbz partials of new_slot) and
// recorded by block 0, which also records r.r (nbr partials)
__global__ void dcg_dir2_kernel(int n, int nbz, int nbr, double *__restrict__ scal, int old_slot, int new_slot,
                                const double *__restrict__ z, double *__restrict__ p, const double *__restrict__ part) {
    __shared__ double sh[kT / 32];
    __shared__ double bc;
    const double rzn = sum_slot(part, new_slot, nbz, sh, &bc);
    const double rzo = scal[old_slot];
    const double b = (rzo > 0 && rzn > 0) ? rzn / rzo : 0.0;
    GRID_STRIDE(j, n) p[j] = z[j] + b * p[j];
    if (blockIdx.x == 0) {
        const double rr = sum_slot(part, SC_NORM_A, nbr, sh, &bc);
        if (threadIdx.x == 0) {
            scal[new_slot] = rzn;
            scal[SC_NORM_A] = rr;
        }
    }
}

template <typename T>
Error dev_alloc(T **p, int64_t count) {
    OT_CUDA(cudaMalloc((void **)p, sizeof(T) * (size_t)std::max<int64_t>(count, 1)));
    return ok();
}

}  // namespace

// ------------------------------------------------------------------------ S_M x = rhs
static Error residual_norm(Newton &W, const Support &S, const double *x, double *res, double *nrm, cudaStream_t st) {
    const unsigned gm = grid_of(W.m, W.num_sms), gn = grid_of(W.n, W.num_sms);
    mv_rows_kernel<<<gm, kT, 0, st>>>(W.m, S.row_ptr, S.j, W.theta, W.Minv, x, W.w64);
    OT_LAUNCHED();
    mv_cols_res_kernel<<<gn, kT, 0, st>>>(W.n, S.col_ptr, S.col_row, W.theta_col, W.w64, x, W.rhs, res, W.part);
    OT_LAUNCHED();
    Finish f{1, {SC_NORM_A}, {(int)gn}, {0}};
    OT_TRY(finish(f, W, st));
    double hs[SC_COUNT];
    OT_TRY(read_scalars(W, hs, st));
    *nrm = std::sqrt(hs[SC_NORM_A]);
    return ok();
}

static Error rhs_norm(Newton &W, double *nrm, cudaStream_t st) {
    const unsigned gn = grid_of(W.n, W.num_sms);
    norm_kernel<<<gn, kT, 0, st>>>(W.n, W.rhs, W.part, SC_NORM_B);
    OT_LAUNCHED();
    Finish f{1, {SC_NORM_B}, {(int)gn}, {0}};
    OT_TRY(finish(f, W, st));
    double hs[SC_COUNT];
    OT_TRY(read_scalars(W, hs, st));
    *nrm = std::sqrt(hs[SC_NORM_B]);
    return ok();
}

static Error solve_pcg64(Newton &W, const Support &S, double tol, int max_cg, double *dv, SolveStats *ss,
                         cudaStream_t st) {
    const unsigned gn = grid_of(W.n, W.num_sms);
    OT_TRY(launch_pcg<double>(W, S, W.theta, W.theta_col, W.Minv, W.Dinv, W.rhs, W.x64, W.r64, W.z64, W.p64,
                              W.q64, W.w64, tol, max_cg, st));
    double hs[SC_COUNT];
    OT_TRY(read_scalars(W, hs, st));
    int errv = 0;
    OT_CUDA(cudaMemcpy(&errv, W.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (errv) return fail(OT_ERR_TIMEOUT, "pcg: grid barrier wait limit reached");
    ss->cg_iters = (int)hs[SC_PCG_ITERS];
    ss->relres = hs[SC_PCG_RELRES];
    ktimer_add_work(KT_PCG64, ss->cg_iters * W.pcg_bytes_per_iter);
    if (W.verbose >= 3)
        fprintf(stderr, "      pcg64 psi %lld its %d relres %.2e ms %.3f\n", (long long)S.psi, ss->cg_iters,
                ss->relres, W.last_pcg_ms);
    copy_kernel<<<gn, kT, 0, st>>>(W.n, W.x64, dv);
    OT_LAUNCHED();
    return ok();
}

// FP32 PCG inside FP64 iterative refinement: dv = 0, res = rhs; repeat
//   solve S32 d = float(res) ; dv += d ; res = rhs - S64 dv      until |res| <= tol |rhs|
static Error solve_mixed(Newton &W, const Support &S, double tol, int max_cg, double *dv, SolveStats *ss,
                         cudaStream_t st) {
    const unsigned gn = grid_of(W.n, W.num_sms);
    const double inner = std::max(tol, 1e-4);
    OT_CUDA(cudaMemsetAsync(dv, 0, sizeof(double) * W.n, st));
    copy_kernel<<<gn, kT, 0, st>>>(W.n, W.rhs, W.res64);
    OT_LAUNCHED();
    double nrm0 = 0.0;
    OT_TRY(rhs_norm(W, &nrm0, st));
    double nrm = nrm0;
    int budget = max_cg;
    for (int ref = 0; ref < 12 && nrm > tol * nrm0 && budget > 0; ++ref) {
        to_f32_kernel<<<gn, kT, 0, st>>>(W.n, W.res64, W.b32);
        OT_LAUNCHED();
        OT_TRY(launch_pcg<float>(W, S, W.theta32, W.theta32_col, W.Minv32, W.Dinv32, W.b32, W.x32, W.r32, W.z32,
                                 W.p32, W.q32, W.w32, inner, budget, st));
        axpy_f32_kernel<<<gn, kT, 0, st>>>(W.n, W.x32, dv);
        OT_LAUNCHED();
        const double prev = nrm;
        OT_TRY(residual_norm(W, S, dv, W.res64, &nrm, st));
        double hs[SC_COUNT];
        OT_TRY(read_scalars(W, hs, st));
        int errv = 0;
        OT_CUDA(cudaMemcpy(&errv, W.err, sizeof(int), cudaMemcpyDeviceToHost));
        if (errv) return fail(OT_ERR_TIMEOUT, "pcg: grid barrier wait limit reached");
        const int its = (int)hs[SC_PCG_ITERS];
        ktimer_add_work(KT_PCG32, its * W.pcg_bytes_per_iter);
        if (W.verbose >= 3)
            fprintf(stderr, "      pcg32 psi %lld its %d relres %.2e ms %.3f\n", (long long)S.psi, its,
                    hs[SC_PCG_RELRES], W.last_pcg_ms);
        ss->cg_iters += its;
        budget -= std::max(its, 1);
        ss->refinements = ref + 1;
        if (!(nrm < 0.9 * prev)) break;  // refinement stagnates
    }
    ss->relres = nrm0 > 0 ? nrm / nrm0 : 0.0;
    return ok();
}

// PCG (FP64) on S_M preconditioned by the LDL^T factorisation of the sparsified Schur complement
// (chol.cuh), or by the FP32 dense factorisation (dense32.cuh).  With no pair dropped the FP64
// factorisation is exact and one iteration suffices; the dropped pairs (negligible theta in their
// row) only perturb the spectrum slightly, and the FP32 factors are accurate entry by entry, so a
// few iterations recover FP64 accuracy (iterative refinement in conjugate-gradient form).
constexpr int kD32MaxCg = 60;

// ------------------------------------------------------------------------ persistent refinement CG
// The FP64 CG preconditioned by the FP32 dense factor (z = L^-T D^+ L^-1 r through X = L^-1), all
// iterations in one cooperative launch: per iteration the row pass, the column pass with p.q, the
// step with r.r, the convergence test, the three stages of the preconditioner (partial products of
// X r by 512 x 64 tiles, their row sums scaled by D^+, the column products of X^T), r.z and the new
// direction, seven grid barriers.  Every block sums the partials of a dot product in the same fixed
// order, so all take the same decisions.  Same arithmetic as the launch-per-stage loop.
constexpr int kCgT = 512;
constexpr int kCgRows = 512, kCgCols = 64;   // preconditioner tile: 128 row quads x 4 column groups

struct D32CgArgs {
    int m, n, ld, ncb;
    const int32_t *rp, *sj, *cp, *crow;
    const double *th, *thc, *Minv, *rhs;
    const float *X, *D;
    float *part, *w32;
    double *x, *r, *z, *p, *q, *w64;
    double *red;          // 3 slots x gridDim partial sums
    unsigned *bar;
    int *err;
    double target2;       // stop when r.r <= target2 * b.b
    int maxit;
    double *scal;         // SC_PCG_ITERS, SC_PCG_RELRES
};

// part[cb ld + i] = sum over the tile's columns j <= i of X_ij r_j, for the lower-triangle tiles
__device__ __forceinline__ void cg_fwd(const D32CgArgs &A, const double *__restrict__ r, float *rs, float4 *red4) {
    const int n = A.n, ld = A.ld, ncb = A.ncb;
    const int per = kCgRows / kCgCols;
    const int nrb = (n + kCgRows - 1) / kCgRows;
    int tiles = 0;
    for (int rb = 0; rb < nrb; ++rb) tiles += min(ncb, (rb + 1) * per);
    const int rq = threadIdx.x & (kCgRows / 4 - 1), cgp = threadIdx.x / (kCgRows / 4);
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
        int idx = t, rb = 0;
        while (idx >= min(ncb, (rb + 1) * per)) { idx -= min(ncb, (rb + 1) * per); ++rb; }
        const int cb = idx, c0 = cb * kCgCols, i = rb * kCgRows + rq * 4;
        if (threadIdx.x < kCgCols) rs[threadIdx.x] = c0 + (int)threadIdx.x < n ? (float)r[c0 + threadIdx.x] : 0.f;
        __syncthreads();
        const bool live = i < n && i + 3 >= c0;
        const int jn = min(kCgCols, n - c0);
        const int jlo = cgp * (kCgCols / 4), jhi = min(jlo + kCgCols / 4, jn);
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (live) {
            const float *col = A.X + (size_t)c0 * ld + i;
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
        if (cgp > 0) red4[(cgp - 1) * (kCgRows / 4) + rq] = acc;
        __syncthreads();
        if (cgp == 0 && live) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float4 o = red4[q * (kCgRows / 4) + rq];
                acc.x += o.x; acc.y += o.y; acc.z += o.z; acc.w += o.w;
            }
            *(float4 *)(A.part + (size_t)cb * ld + i) = acc;
        }
        __syncthreads();
    }
}

// w32_i = D_i^+ sum_cb part[cb ld + i]
__device__ __forceinline__ void cg_mid(const D32CgArgs &A) {
    GRID_STRIDE(i, A.n) {
        const int last = (int)i / kCgCols;
        float y = 0.f;
        for (int cb = 0; cb <= last; ++cb) y += A.part[(size_t)cb * A.ld + i];
        const float d = A.D[i];
        A.w32[i] = isinf(d) ? 0.f : y / d;
    }
}

// z_j = sum_{i >= j} X_ij w32_i (one warp per column); returns this thread's part of r.z
__device__ __forceinline__ double cg_bwd(const D32CgArgs &A, const double *__restrict__ r) {
    const int n = A.n, lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    double rz = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n; j += warps) {
        const float *col = A.X + (size_t)j * A.ld;
        float acc = 0.f;
        const int i0 = (int)j & ~3;
        for (int i = i0 + lane * 4; i < n; i += 128) {
            const float4 v = *(const float4 *)(col + i);
            if (i >= j && i + 3 < n) {
                acc += v.x * A.w32[i] + v.y * A.w32[i + 1] + v.z * A.w32[i + 2] + v.w * A.w32[i + 3];
            } else {
                if (i >= j && i < n) acc += v.x * A.w32[i];
                if (i + 1 >= j && i + 1 < n) acc += v.y * A.w32[i + 1];
                if (i + 2 >= j && i + 2 < n) acc += v.z * A.w32[i + 2];
                if (i + 3 >= j && i + 3 < n) acc += v.w * A.w32[i + 3];
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const double zj = (double)acc;
            A.z[j] = zj;
            rz += r[j] * zj;
        }
    }
    return rz;
}

template <int LG>
__global__ void __launch_bounds__(kCgT) d32_cg_kernel(D32CgArgs A) {
    __shared__ double sh[kCgT / 32];
    __shared__ double s_val[3];
    __shared__ float rs[kCgCols];
    __shared__ float4 red4[3 * (kCgRows / 4)];
    const unsigned G = gridDim.x;
    const int n = A.n, m = A.m;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)G * blockDim.x;
    const int lg = threadIdx.x & (LG - 1);
    const int64_t grp = tid / LG, ngrp = stride / LG, wgrp0 = (tid & ~(int64_t)31) / LG;
    double *P0 = A.red, *P1 = A.red + G, *P2 = A.red + 2 * G;
    // x = 0, r = rhs, z = M^-1 r, p = z
    double rr = 0.0;
    for (int64_t j = tid; j < n; j += stride) {
        const double bj = A.rhs[j];
        A.x[j] = 0.0;
        A.r[j] = bj;
        rr += bj * bj;
    }
    if (!grid_barrier(A.bar, G, A.err)) return;
    cg_fwd(A, A.r, rs, red4);
    if (!grid_barrier(A.bar, G, A.err)) return;
    cg_mid(A);
    if (!grid_barrier(A.bar, G, A.err)) return;
    double rz = cg_bwd(A, A.r);
    {
        const double s1 = block_sum(rz, sh), s2 = block_sum(rr, sh);
        if (threadIdx.x == 0) { P1[blockIdx.x] = s1; P2[blockIdx.x] = s2; }
    }
    if (!grid_barrier(A.bar, G, A.err)) return;
    for (int64_t j = tid; j < n; j += stride) A.p[j] = A.z[j];
    sum_partials(A.red + G, G, 2, s_val + 1);
    rz = s_val[1];
    const double bb = s_val[2];
    rr = bb;
    // once converged, one more iteration refines x (as the launch-per-stage loop, which runs one
    // iteration ahead of its test, does); the count and the residual reported are those of the test
    int it = 0;
    bool extra = false;
    double rr_test = rr;
    if (bb > 0.0 && rz > 0.0 && A.maxit > 0) {
        for (;;) {
            // the new direction p must be complete before the row pass gathers it
            if (!grid_barrier(A.bar, G, A.err)) return;
            for (int64_t i0 = wgrp0; i0 < m; i0 += ngrp) {
                const int64_t i = i0 + (grp - wgrp0);
                double acc = 0.0;
                if (i < m)
                    for (int e = A.rp[i] + lg; e < A.rp[i + 1]; e += LG) acc += A.th[e] * A.p[A.sj[e]];
                acc = group_sum(acc, LG);
                if (lg == 0 && i < m) A.w64[i] = A.Minv[i] * acc;
            }
            if (!grid_barrier(A.bar, G, A.err)) return;
            double pq = 0.0;
            for (int64_t j0 = wgrp0; j0 < n; j0 += ngrp) {
                const int64_t j = j0 + (grp - wgrp0);
                double acc = 0.0, pj = 0.0;
                if (j < n) {
                    pj = A.p[j];
                    for (int k = A.cp[j] + lg; k < A.cp[j + 1]; k += LG) acc += A.thc[k] * (pj - A.w64[A.crow[k]]);
                }
                acc = group_sum(acc, LG);
                if (lg == 0 && j < n) {
                    A.q[j] = acc;
                    pq += pj * acc;
                }
            }
            {
                const double s0 = block_sum(pq, sh);
                if (threadIdx.x == 0) P0[blockIdx.x] = s0;
            }
            if (!grid_barrier(A.bar, G, A.err)) return;
            sum_partials(A.red, G, 1, s_val);
            pq = s_val[0];
            if (!(pq > 0.0)) break;   // breakdown: the step would be a no-op
            const double alpha = rz > 0.0 ? rz / pq : 0.0;
            double rrn = 0.0;
            for (int64_t j = tid; j < n; j += stride) {
                A.x[j] += alpha * A.p[j];
                const double rj = A.r[j] - alpha * A.q[j];
                A.r[j] = rj;
                rrn += rj * rj;
            }
            {
                const double s2 = block_sum(rrn, sh);
                if (threadIdx.x == 0) P2[blockIdx.x] = s2;
            }
            if (!grid_barrier(A.bar, G, A.err)) return;
            sum_partials(A.red + 2 * G, G, 1, s_val + 2);
            rr = s_val[2];
            if (extra) break;
            ++it;
            rr_test = rr;
            if (it >= A.maxit) break;
            if (rr <= A.target2 * bb) extra = true;
            cg_fwd(A, A.r, rs, red4);
            if (!grid_barrier(A.bar, G, A.err)) return;
            cg_mid(A);
            if (!grid_barrier(A.bar, G, A.err)) return;
            double rzn = cg_bwd(A, A.r);
            {
                const double s1 = block_sum(rzn, sh);
                if (threadIdx.x == 0) P1[blockIdx.x] = s1;
            }
            if (!grid_barrier(A.bar, G, A.err)) return;
            sum_partials(A.red + G, G, 1, s_val + 1);
            rzn = s_val[1];
            const double beta = (rz > 0.0 && rzn > 0.0) ? rzn / rz : 0.0;
            for (int64_t j = tid; j < n; j += stride) A.p[j] = A.z[j] + beta * A.p[j];
            rz = rzn;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.scal[SC_PCG_ITERS] = (double)it;
        A.scal[SC_PCG_RELRES] = bb > 0.0 ? sqrt(rr_test / bb) : 0.0;
    }
}


// the persistent form of solve_direct's loop for the FP32 dense preconditioner
static Error solve_d32_persistent(Newton &W, const Support &S, double target, int cap, double *dv, SolveStats *ss,
                                  cudaStream_t st) {
    Dense32 &F = *W.d32;
    const double avg = (double)S.psi / (double)std::max(1, std::min(W.m, W.n));
    const int LG = avg >= 12 ? 16 : (avg >= 6 ? 8 : 4);
    const void *fn = LG == 16 ? (const void *)d32_cg_kernel<16>
                   : (LG == 8 ? (const void *)d32_cg_kernel<8> : (const void *)d32_cg_kernel<4>);
    int per_sm = 0;
    OT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kCgT, 0));
    const int maxg = std::max(1, per_sm) * W.num_sms;
    const int64_t want = std::max<int64_t>(ceil_div((int64_t)std::max(W.m, W.n) * LG, kCgT),
                                           ceil_div((int64_t)W.n, kCgT / 32));
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>(want, std::min(maxg, kMaxPartBlocks / 3)));
    OT_CUDA(cudaMemsetAsync(W.bar, 0, 2 * sizeof(unsigned), st));
    OT_CUDA(cudaMemsetAsync(W.err, 0, sizeof(int), st));
    D32CgArgs A{W.m, W.n, F.ld, (int)ceil_div(W.n, kCgCols), S.row_ptr, S.j, S.col_ptr, S.col_row, W.theta,
                W.theta_col, W.Minv, W.rhs, F.X, F.D, F.part, F.w, dv, W.r64, W.z64, W.p64, W.q64, W.w64, W.part,
                W.bar, W.err, target * target, cap, W.scal};
    void *args[] = {&A};
    ktimer_begin(KT_DCG, st);
    const cudaError_t le = cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kCgT), args, 0, st);
    if (le == cudaErrorCooperativeLaunchTooLarge) {   // the device cannot hold the grid now
        cudaGetLastError();
        ktimer_end(KT_DCG, st);
        return fail(OT_ERR_UNSUPPORTED, "refinement CG: cooperative grid not resident");
    }
    OT_CUDA(le);
    OT_LAUNCHED();
    ktimer_end(KT_DCG, st);
    double hs[SC_COUNT];
    OT_TRY(read_scalars(W, hs, st));
    int errv = 0;
    OT_CUDA(cudaMemcpy(&errv, W.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (errv) return fail(OT_ERR_TIMEOUT, "refinement CG: grid barrier wait limit reached");
    ss->cg_iters = (int)hs[SC_PCG_ITERS];
    ss->direct = 0;
    ss->relres = hs[SC_PCG_RELRES];
    // per iteration: the operator's bytes (as the stage-per-launch form) plus the triangle of L^-1 twice
    ktimer_add_work(KT_DCG, ss->cg_iters * (40.0 * (double)S.psi + 20.0 * (double)W.m + 68.0 * (double)W.n +
                                            4.0 * (double)W.n * (double)W.n));
    return ok();
}

static Error solve_direct(Newton &W, const Support &S, double tol, int max_cg, double *dv, SolveStats *ss,
                          cudaStream_t st) {
    const unsigned gm = grid_of(W.m, W.num_sms), gn = grid_of(W.n, W.num_sms);
    Chol *C = W.direct;
    const bool ic_only = !C && !W.d32 && !W.tree && W.ic;
    // near optimality the primal-infeasibility part of the right-hand side is tiny next to the
    // complementarity part, so the direct branch solves far below the PCG tolerance; the incomplete
    // factor is the iterative phase's preconditioner and stops at the PCG tolerance
    const double target = ic_only ? tol : (W.direct_cg_tol > 0 ? std::max(W.direct_cg_tol, std::min(tol, 1e-10))
                                                               : std::min(tol, 1e-10));
    if (W.d32 && !C && !W.tree) {
        const Error e = solve_d32_persistent(W, S, target, std::min(max_cg, kD32MaxCg), dv, ss, st);
        if (e.code != OT_ERR_UNSUPPORTED) return e;   // else the launch-per-stage loop below
    }
    double *x = W.x64, *r = W.r64, *z = W.z64, *p = W.p64, *q = W.q64;
    double hs[SC_COUNT];
    OT_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * W.n, st));
    copy_kernel<<<gn, kT, 0, st>>>(W.n, W.rhs, r);
    OT_LAUNCHED();
    auto precond = [&](const double *in, double *out) -> Error {
        if (W.tree) return tree_solve(*W.tree, S, W.theta, in, out, st);
        if (C) return W.dense ? dense_solve(*W.dense, in, out, st) : chol_solve(*C, in, out, st);
        if (W.d32) return d32_apply(*W.d32, in, out, st);
        return ic_apply(*W.ic, in, out, st);
    };
    OT_TRY(precond(r, z));
    pcg_dir_kernel<<<gn, kT, 0, st>>>(W.n, 0.0, z, p);
    OT_LAUNCHED();
    dot_kernel<<<gn, kT, 0, st>>>(W.n, r, z, W.part, SC_RZ0);
    OT_LAUNCHED();
    dot_kernel<<<gn, kT, 0, st>>>(W.n, r, r, W.part, SC_NORM_B);
    OT_LAUNCHED();
    {
        Finish f{2, {SC_RZ0, SC_NORM_B}, {(int)gn, (int)gn}, {0, 0}};
        OT_TRY(finish(f, W, st));
    }
    // |rhs|^2 and r.z reach the host with the first iteration's scalars (no separate round trip);
    // with r.z <= 0 that iteration's step is a no-op
    double bb = -1.0;
    double rr = 0.0;
    int it = 0;
    // an accurate FP32 factor gains several digits per iteration; one that needs many more has
    // met a matrix beyond FP32 and hands the system to the FP64 factorisation
    const int cap = (C || ic_only || W.tree) ? max_cg : std::min(max_cg, kD32MaxCg);
    // alpha and beta stay on the device; the host reads p.q and r.r of each iteration while the
    // GPU already applies the preconditioner for the next one (wasted only at the last iteration)
    {
        // lanes per row / column for the FP64 products: about the average row length, <= 16
        const double avg = (double)S.psi / (double)std::max(1, std::min(W.m, W.n));
        const int G = avg >= 12 ? 16 : (avg >= 6 ? 8 : 4);
        const unsigned gmr = (unsigned)std::min<int64_t>(ceil_div((int64_t)W.m * G, kT), 8LL * W.num_sms);
        const unsigned gnc = (unsigned)std::min<int64_t>(ceil_div((int64_t)W.n * G, kT), kMaxPartBlocks);
        // algorithmic bytes of one operator application and step: per support pair theta (8), an
        // index (4) and a gathered vector entry (8) in each pass; per row the offset, M^-1 and w;
        // per column the offset, q, p twice and the step's reads of x, r and writes of x, r
        const double dcg_bytes = 40.0 * (double)S.psi + 20.0 * (double)W.m + 68.0 * (double)W.n;
        auto issue = [&](int k) -> Error {
            const int cur = (k & 1) ? SC_RZ1 : SC_RZ0, nxt = (k & 1) ? SC_RZ0 : SC_RZ1;
            ktimer_begin(KT_DCG, st);
            if (G == 16) {
                mvg_rows_kernel<16><<<gmr, kT, 0, st>>>(W.m, S.row_ptr, S.j, W.theta, W.Minv, p, W.w64);
                OT_LAUNCHED();
                mvg_cols_kernel<16><<<gnc, kT, 0, st>>>(W.n, S.col_ptr, S.col_row, W.theta_col, W.w64, p, q, W.part);
            } else if (G == 8) {
                mvg_rows_kernel<8><<<gmr, kT, 0, st>>>(W.m, S.row_ptr, S.j, W.theta, W.Minv, p, W.w64);
                OT_LAUNCHED();
                mvg_cols_kernel<8><<<gnc, kT, 0, st>>>(W.n, S.col_ptr, S.col_row, W.theta_col, W.w64, p, q, W.part);
            } else {
                mvg_rows_kernel<4><<<gmr, kT, 0, st>>>(W.m, S.row_ptr, S.j, W.theta, W.Minv, p, W.w64);
                OT_LAUNCHED();
                mvg_cols_kernel<4><<<gnc, kT, 0, st>>>(W.n, S.col_ptr, S.col_row, W.theta_col, W.w64, p, q, W.part);
            }
            OT_LAUNCHED();
            dcg_step2_kernel<<<gn, kT, 0, st>>>(W.n, (int)gnc, W.scal, cur, p, q, x, r, W.part);
            OT_LAUNCHED();
            ktimer_end(KT_DCG, st);
            ktimer_add_work(KT_DCG, dcg_bytes);
            OT_TRY(precond(r, z));
            dot_kernel<<<gn, kT, 0, st>>>(W.n, r, z, W.part, nxt);
            OT_LAUNCHED();
            dcg_dir2_kernel<<<gn, kT, 0, st>>>(W.n, (int)gn, (int)gn, W.scal, cur, nxt, z, p, W.part);
            OT_LAUNCHED();
            OT_CUDA(cudaMemcpyAsync(W.hscal + (k & 1) * SC_COUNT, W.scal, sizeof(double) * SC_COUNT,
                                    cudaMemcpyDeviceToHost, st));
            OT_CUDA(cudaEventRecord(W.ev_scal2[k & 1], st));
            return ok();
        };
        // with the FP32 factor, one iteration is queued ahead of the one being checked: alpha and
        // beta live on the device, so an iteration issued past convergence only refines x further
        int issued = 0;
        if (cap > 0) {
            OT_TRY(issue(0));
            issued = 1;
        }
        const bool ahead = C == nullptr;  // only where the preconditioner is cheap
        while (it < issued) {
            if (issued < cap && (ahead || issued == it)) {
                OT_TRY(issue(issued));
                ++issued;
            }
            OT_CUDA(cudaEventSynchronize(W.ev_scal2[it & 1]));
            const double *h = W.hscal + (it & 1) * SC_COUNT;
            if (bb < 0) {
                bb = h[SC_NORM_B];
                rr = bb;
                if (!(bb > 0) || !(h[SC_RZ0] > 0)) break;
            }
            const double pq = h[SC_SUM_A];
            if (!(pq > 0)) break;  // breakdown: this step was a no-op
            rr = h[SC_NORM_A];
            ++it;
            if (rr <= target * target * bb) break;
        }
        // an iteration still queued ahead completes before the copy below (stream order)
    }
    if (bb < 0) {  // no iteration ran (max_cg 0): the residual is the right-hand side
        OT_TRY(read_scalars(W, hs, st));
        bb = hs[SC_NORM_B];
        rr = bb;
    }
    copy_kernel<<<gn, kT, 0, st>>>(W.n, x, dv);
    OT_LAUNCHED();
    if (C) {
        int errv = 0;
        OT_CUDA(cudaMemcpyAsync(&errv, W.dense ? W.dense->err : C->err, sizeof(int), cudaMemcpyDeviceToHost, st));
        OT_CUDA(cudaStreamSynchronize(st));
        if (errv) return fail(OT_ERR_TIMEOUT, "ldl solve: grid barrier wait limit reached");
    }
    ss->cg_iters = it;
    ss->direct = C ? 1 : 0;
    ss->relres = bb > 0 ? std::sqrt(rr / bb) : 0.0;
    return ok();
}

Error newton_alloc(Newton &W, int32_t m, int32_t n, int64_t cap, int num_sms) {
    W.m = m;
    W.n = n;
    W.num_sms = num_sms;
    // largest cluster (16, else 8, else none) of full-shared-memory CTAs the device schedules
    W.pcg_cluster = 0;
    W.pcg_cluster_smem = 0;
    {
        int dev = 0, optin = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess) {
            const int sb = optin - 1024;  // room for the kernel's static shared memory
            if (sb > 0 &&
                cudaFuncSetAttribute(pcg_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sb) == cudaSuccess &&
                cudaFuncSetAttribute(pcg_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                    cudaSuccess) {
                for (int c : {kClMaxR, 8}) {
                    cudaLaunchConfig_t cfg = {};
                    cfg.gridDim = dim3(c);
                    cfg.blockDim = dim3(kClT);
                    cfg.dynamicSmemBytes = (size_t)sb;
                    cudaLaunchAttribute attr[1];
                    attr[0].id = cudaLaunchAttributeClusterDimension;
                    attr[0].val.clusterDim.x = c;
                    attr[0].val.clusterDim.y = 1;
                    attr[0].val.clusterDim.z = 1;
                    cfg.attrs = attr;
                    cfg.numAttrs = 1;
                    int nclusters = 0;
                    if (cudaOccupancyMaxActiveClusters(&nclusters, pcg_cluster_kernel, &cfg) == cudaSuccess &&
                        nclusters >= 1) {
                        W.pcg_cluster = c;
                        W.pcg_cluster_smem = sb;
                        break;
                    }
                }
            }
        }
        cudaGetLastError();  // a refused attribute or query only disables the cluster variant
    }
    OT_TRY(newton_grow(W, cap));
    for (double **p : {&W.r1a, &W.beta1, &W.M, &W.Minv, &W.du, &W.du2, &W.du3, &W.w64}) OT_TRY(dev_alloc(p, m));
    for (float **p : {&W.Minv32, &W.w32}) OT_TRY(dev_alloc(p, m));
    for (double **p : {&W.r1b, &W.beta2, &W.N, &W.Dinv, &W.Sdiag, &W.rhs, &W.dv, &W.dv2, &W.dv3, &W.res64, &W.y64, &W.x64,
                       &W.r64, &W.z64, &W.p64, &W.q64})
        OT_TRY(dev_alloc(p, n));
    for (float **p : {&W.Dinv32, &W.b32, &W.x32, &W.r32, &W.z32, &W.p32, &W.q32, &W.pcg_pb32}) OT_TRY(dev_alloc(p, n));
    OT_TRY(dev_alloc(&W.pcg_pb, n));
    // grid PCG lane groups: G kPcgT / g <= (blocks per SM <= 2048 / kPcgT) x SMs x kPcgT
    W.pcg_bnd_cap = (int64_t)(2048 / kPcgT) * std::max(num_sms, 1) * kPcgT + 1;
    OT_TRY(dev_alloc(&W.pcg_bnd, 2 * W.pcg_bnd_cap));
    OT_TRY(dev_alloc(&W.parent, (int64_t)m + n));
    OT_TRY(dev_alloc(&W.comp_sum, (int64_t)m + n));
    OT_TRY(dev_alloc(&W.comp_cnt, (int64_t)m + n));
    OT_TRY(dev_alloc(&W.part, (int64_t)SC_COUNT * kMaxPartBlocks));
    OT_CUDA(cudaHostAlloc((void **)&W.hscal, 2 * sizeof(double) * SC_COUNT, cudaHostAllocDefault));
    OT_CUDA(cudaEventCreateWithFlags(&W.ev_scal, cudaEventDisableTiming));
    OT_CUDA(cudaEventCreateWithFlags(&W.ev_scal2[0], cudaEventDisableTiming));
    OT_CUDA(cudaEventCreateWithFlags(&W.ev_scal2[1], cudaEventDisableTiming));
    OT_TRY(dev_alloc(&W.scal, SC_COUNT));
    OT_TRY(dev_alloc(&W.bar, 2));
    OT_TRY(dev_alloc(&W.err, 1));
    return ok();
}

Error newton_grow(Newton &W, int64_t cap) {
    if (cap <= W.cap) return ok();
    double **d[] = {&W.c, &W.theta, &W.excl, &W.r2, &W.r3, &W.g, &W.dp, &W.ds, &W.dp2, &W.ds2, &W.dp3, &W.ds3,
                    &W.theta_col};
    for (double **p : d) { if (*p) cudaFree(*p); *p = nullptr; OT_TRY(dev_alloc(p, cap)); }
    for (float **p : {&W.theta32, &W.theta32_col}) { if (*p) cudaFree(*p); *p = nullptr; OT_TRY(dev_alloc(p, cap)); }
    if (W.flag) cudaFree(W.flag);
    W.flag = nullptr;
    OT_TRY(dev_alloc(&W.flag, cap));
    W.cap = cap;
    return ok();
}

void newton_free(Newton &W) {
    void *ptrs[] = {W.c, W.theta, W.excl, W.r2, W.r3, W.g, W.dp, W.ds, W.dp2, W.ds2, W.dp3, W.ds3, W.theta32,
                    W.theta_col, W.theta32_col, W.flag, W.r1a, W.beta1, W.M, W.Minv, W.du, W.du2, W.du3, W.w64,
                    W.Minv32, W.w32, W.r1b, W.beta2, W.N, W.Dinv, W.Sdiag, W.rhs, W.dv, W.dv2, W.dv3, W.res64, W.y64,
                    W.x64, W.r64, W.z64, W.p64, W.q64, W.Dinv32, W.b32, W.x32, W.r32, W.z32, W.p32, W.q32, W.pcg_pb, W.pcg_pb32,
                    W.pcg_bnd, W.parent, W.comp_sum, W.comp_cnt, W.part, W.scal, W.bar, W.err};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (W.hscal) cudaFreeHost(W.hscal);
    if (W.ev_scal) cudaEventDestroy(W.ev_scal);
    for (cudaEvent_t e : W.ev_scal2)
        if (e) cudaEventDestroy(e);
    W = Newton();
}

Error support_costs(Newton &W, const CostDev &cd, const Support &S, cudaStream_t st) {
    if (S.psi == 0) return ok();
    support_cost_kernel<<<grid_of(S.psi, W.num_sms), kT, 0, st>>>(cd, S.psi, S.i, S.j, W.c);
    OT_LAUNCHED();
    return ok();
}

Error residuals(Newton &W, const Support &S, const double *a_s, const double *b_s, const double *u,
                const double *v, cudaStream_t st) {
    const unsigned gm = grid_of(W.m, W.num_sms), ge = grid_of(S.psi, W.num_sms);
    // 8 lanes per column; at most kMaxPartBlocks blocks (one partial slot each)
    const unsigned gn = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)W.n * 8, kT),
                                                                          std::min(8 * W.num_sms, kMaxPartBlocks)));
    res_rows_kernel<<<gm, kT, 0, st>>>(W.m, S.row_ptr, S.p, a_s, W.r1a, W.part);
    OT_LAUNCHED();
    res_cols_group_kernel<8><<<gn, kT, 0, st>>>(W.n, S.col_ptr, S.col_perm, S.p, b_s, W.r1b, W.part);
    OT_LAUNCHED();
    res_entries_kernel<<<ge, kT, 0, st>>>(S.psi, S.i, S.j, W.c, S.p, S.s, u, v, W.r2, W.part);
    OT_LAUNCHED();
    Finish f{8,
             {SC_R1A_SQ, SC_R1A_L1, SC_R1B_SQ, SC_R1B_L1, SC_R2SQ, SC_PS, SC_CP, SC_CSQ},
             {(int)gm, (int)gm, (int)gn, (int)gn, (int)ge, (int)ge, (int)ge, (int)ge},
             {0, 0, 0, 0, 0, 0, 0, 0}};
    OT_TRY(finish(f, W, st));
    Finish f2{1, {SC_CMAX}, {(int)ge}, {2}};
    OT_TRY(finish(f2, W, st));
    return ok();
}

Error schur_setup(Newton &W, const Support &S, cudaStream_t st) {
    const unsigned gm = grid_of(W.m, W.num_sms), gn = grid_of(W.n, W.num_sms), ge = grid_of(S.psi, W.num_sms);
    theta_kernel<<<ge, kT, 0, st>>>(S.psi, S.p, S.s, W.theta, W.theta32);
    OT_LAUNCHED();
    {
        const unsigned g8m = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)W.m * 8, kT),
                                                                              8LL * W.num_sms));
        const unsigned g8n = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)W.n * 8, kT),
                                                                              8LL * W.num_sms));
        theta_rows_group_kernel<8><<<g8m, kT, 0, st>>>(W.m, S.row_ptr, W.theta, W.excl, W.M, W.Minv, W.Minv32);
        OT_LAUNCHED();
        theta_cols_group_kernel<8><<<g8n, kT, 0, st>>>(W.n, S.col_ptr, S.col_perm, S.col_row, W.theta, W.excl,
                                                        W.Minv, W.theta_col, W.theta32_col, W.N, W.Dinv, W.Dinv32,
                                                        W.Sdiag);
        OT_LAUNCHED();
    }
    const int nn = W.m + W.n;
    const unsigned gnn = grid_of(nn, W.num_sms);
    uf_init_kernel<<<gnn, kT, 0, st>>>(nn, W.parent);
    OT_LAUNCHED();
    uf_hook_kernel<<<ge, kT, 0, st>>>(S.psi, W.m, S.i, S.j, W.parent);
    OT_LAUNCHED();
    uf_final_kernel<<<gnn, kT, 0, st>>>(nn, W.parent);
    OT_LAUNCHED();
    onecomp_kernel<<<gn, kT, 0, st>>>(W.m, W.n, W.parent, W.part);
    OT_LAUNCHED();
    Finish f{1, {SC_ONECOMP}, {(int)gn}, {0}};
    OT_TRY(finish(f, W, st));
    // the support graph is fixed for the iteration: every solve's projection reads this once
    double hs[SC_COUNT];
    OT_TRY(read_scalars(W, hs, st));
    W.onecomp = hs[SC_ONECOMP] == 0.0;
    return ok();
}

__global__ void count_roots_kernel(int nn, const int32_t *__restrict__ parent, double *part) {
    __shared__ double sh[kT / 32];
    double c = 0;
    GRID_STRIDE(v, nn) c += parent[v] == (int32_t)v ? 1.0 : 0.0;
    put_sum(c, part, SC_ONECOMP, sh);
}

Error support_components(Newton &W, int64_t *ncomp, cudaStream_t st) {
    const int nn = W.m + W.n;
    const unsigned gnn = grid_of(nn, W.num_sms);
    count_roots_kernel<<<gnn, kT, 0, st>>>(nn, W.parent, W.part);
    OT_LAUNCHED();
    Finish f{1, {SC_ONECOMP}, {(int)gnn}, {0}};
    OT_TRY(finish(f, W, st));
    double hs[SC_COUNT];
    OT_TRY(read_scalars(W, hs, st));
    *ncomp = (int64_t)hs[SC_ONECOMP];
    return ok();
}

Error support_connected(Newton &W, const Support &S, bool *one, cudaStream_t st) {
    const int nn = W.m + W.n;
    const unsigned gnn = grid_of(nn, W.num_sms), ge = grid_of(S.psi, W.num_sms), gn = grid_of(W.n, W.num_sms);
    uf_init_kernel<<<gnn, kT, 0, st>>>(nn, W.parent);
    OT_LAUNCHED();
    uf_hook_kernel<<<ge, kT, 0, st>>>(S.psi, W.m, S.i, S.j, W.parent);
    OT_LAUNCHED();
    uf_final_kernel<<<gnn, kT, 0, st>>>(nn, W.parent);
    OT_LAUNCHED();
    onecomp_kernel<<<gn, kT, 0, st>>>(W.m, W.n, W.parent, W.part);
    OT_LAUNCHED();
    Finish f{1, {SC_ONECOMP}, {(int)gn}, {0}};
    OT_TRY(finish(f, W, st));
    double hs[SC_COUNT];
    OT_TRY(read_scalars(W, hs, st));
    *one = hs[SC_ONECOMP] == 0.0;
    return ok();
}

// project x to mean zero on every connected component (reads scal[SC_ONECOMP] on the host)
static Error project(Newton &W, double *x, bool one_comp, cudaStream_t st) {
    const unsigned gn = grid_of(W.n, W.num_sms);
    if (one_comp) {
        sum_kernel<<<gn, kT, 0, st>>>(W.n, x, W.part, SC_SUM_B);
        OT_LAUNCHED();
        Finish f{1, {SC_SUM_B}, {(int)gn}, {0}};
        OT_TRY(finish(f, W, st));
        center_kernel<<<gn, kT, 0, st>>>(W.n, x, W.scal, SC_SUM_B);
        OT_LAUNCHED();
    } else {
        const int nn = W.m + W.n;
        OT_CUDA(cudaMemsetAsync(W.comp_sum, 0, sizeof(double) * nn, st));
        OT_CUDA(cudaMemsetAsync(W.comp_cnt, 0, sizeof(double) * nn, st));
        comp_accum_kernel<<<gn, kT, 0, st>>>(W.m, W.n, W.parent, x, W.comp_sum, W.comp_cnt);
        OT_LAUNCHED();
        comp_center_kernel<<<gn, kT, 0, st>>>(W.m, W.n, W.parent, x, W.comp_sum, W.comp_cnt);
        OT_LAUNCHED();
    }
    return ok();
}

Error newton_solve(Newton &W, const Support &S, const Rhs &R, double cg_tol, int max_cg, int precision,
                   double *du, double *dv, double *ds, double *dp, SolveStats *stats, cudaStream_t st) {
    const unsigned gm = grid_of(W.m, W.num_sms), gn = grid_of(W.n, W.num_sms), ge = grid_of(S.psi, W.num_sms);
    g_kernel<<<ge, kT, 0, st>>>(S.psi, W.theta, S.p, R.r2, R.r3, W.g);
    OT_LAUNCHED();
    {
        const unsigned g8m = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)W.m * 8, kT),
                                                                              8LL * W.num_sms));
        beta1_group_kernel<8><<<g8m, kT, 0, st>>>(W.m, S.row_ptr, W.g, R.r1a, W.beta1);
        OT_LAUNCHED();
    }
    {
        const unsigned gg = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)W.n * 8, kT),
                                                                             8LL * W.num_sms));
        rhs_group_kernel<8><<<gg, kT, 0, st>>>(W.n, S.col_ptr, S.col_perm, S.col_row, W.g, W.theta_col, W.Minv,
                                               W.beta1, R.r1b, W.beta2, W.rhs);
        OT_LAUNCHED();
    }
    const bool one = W.onecomp;
    OT_TRY(project(W, W.rhs, one, st));

    SolveStats ss;
    if (W.direct || W.d32 || W.ic || W.tree) {
        OT_TRY(solve_direct(W, S, cg_tol, max_cg, dv, &ss, st));
    } else if (precision == 0) {
        OT_TRY(solve_pcg64(W, S, cg_tol, max_cg, dv, &ss, st));
    } else {
        OT_TRY(solve_mixed(W, S, cg_tol, max_cg, dv, &ss, st));
        if (W.fp64_fallback && !(ss.relres <= cg_tol)) {
            // FP32 cannot resolve this system (condition beyond ~1/eps32): redo it in FP64
            SolveStats s64;
            OT_TRY(solve_pcg64(W, S, cg_tol, max_cg, dv, &s64, st));
            s64.cg_iters += ss.cg_iters;
            ss = s64;
            W.fallbacks++;
        }
    }
    OT_TRY(project(W, dv, one, st));
    {
        const unsigned gg = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)W.m * 8, kT),
                                                                             8LL * W.num_sms));
        du_group_kernel<8><<<gg, kT, 0, st>>>(W.m, S.row_ptr, S.j, W.theta, W.Minv, W.beta1, dv, du);
        OT_LAUNCHED();
    }
    dsdp_kernel<<<ge, kT, 0, st>>>(S.psi, S.i, S.j, S.p, S.s, R.r2, R.r3, du, dv, ds, dp);
    OT_LAUNCHED();
    if (stats) *stats = ss;
    return ok();
}

Error step_lengths(Newton &W, const Support &S, const double *dp, const double *ds, double, cudaStream_t st) {
    const unsigned ge = grid_of(S.psi, W.num_sms);
    ratio_kernel<<<ge, kT, 0, st>>>(S.psi, S.p, dp, S.s, ds, W.part);
    OT_LAUNCHED();
    Finish f{2, {SC_AP, SC_AS}, {(int)ge, (int)ge}, {1, 1}};
    return finish(f, W, st);
}

Error trial_complementarity(Newton &W, const Support &S, const double *dp, const double *ds, double ap, double as,
                            cudaStream_t st) {
    const unsigned ge = grid_of(S.psi, W.num_sms);
    trial_kernel<<<ge, kT, 0, st>>>(S.psi, S.p, dp, S.s, ds, ap, as, W.part);
    OT_LAUNCHED();
    Finish f{1, {SC_MUAFF}, {(int)ge}, {0}};
    return finish(f, W, st);
}

Error corrector_r3(Newton &W, const Support &S, double smu, const double *dpa, const double *dsa, cudaStream_t st) {
    corr_r3_kernel<<<grid_of(S.psi, W.num_sms), kT, 0, st>>>(S.psi, S.p, S.s, dpa, dsa, smu, W.r3);
    OT_LAUNCHED();
    return ok();
}

Error centrality_r3(Newton &W, const Support &S, const double *dp, const double *ds, double tp, double ts,
                    double lo, double hi, cudaStream_t st) {
    centr_r3_kernel<<<grid_of(S.psi, W.num_sms), kT, 0, st>>>(S.psi, S.p, S.s, dp, ds, tp, ts, lo, hi, W.r3);
    OT_LAUNCHED();
    return ok();
}

Error add_direction(Newton &W, const Support &S, double *dp, double *ds, double *du, double *dv,
                    const double *dp2, const double *ds2, const double *du2, const double *dv2, cudaStream_t st) {
    add_kernel<<<grid_of(S.psi, W.num_sms), kT, 0, st>>>(S.psi, dp, dp2);
    OT_LAUNCHED();
    add_kernel<<<grid_of(S.psi, W.num_sms), kT, 0, st>>>(S.psi, ds, ds2);
    OT_LAUNCHED();
    add_kernel<<<grid_of(W.m, W.num_sms), kT, 0, st>>>(W.m, du, du2);
    OT_LAUNCHED();
    add_kernel<<<grid_of(W.n, W.num_sms), kT, 0, st>>>(W.n, dv, dv2);
    OT_LAUNCHED();
    return ok();
}

Error take_step(Newton &W, Support &S, double *u, double *v, const double *dp, const double *ds, const double *du,
                const double *dv, double ap, double as, cudaStream_t st) {
    const unsigned ge = grid_of(S.psi, W.num_sms);
    step_entries_kernel<<<ge, kT, 0, st>>>(S.psi, S.p, S.s, dp, ds, ap, as, W.part);
    OT_LAUNCHED();
    axpy_kernel<<<grid_of(W.m, W.num_sms), kT, 0, st>>>(W.m, as, du, u);
    OT_LAUNCHED();
    axpy_kernel<<<grid_of(W.n, W.num_sms), kT, 0, st>>>(W.n, as, dv, v);
    OT_LAUNCHED();
    Finish f{1, {SC_PSNEW}, {(int)ge}, {0}};
    return finish(f, W, st);
}

Error read_scalars(Newton &W, double *host, cudaStream_t st) {
    OT_CUDA(cudaMemcpyAsync(W.hscal, W.scal, sizeof(double) * SC_COUNT, cudaMemcpyDeviceToHost, st));
    OT_CUDA(cudaStreamSynchronize(st));
    std::memcpy(host, W.hscal, sizeof(double) * SC_COUNT);
    return ok();
}

// ------------------------------------------------------------------------ Mehrotra start
namespace {
__global__ void fill_kernel(int64_t count, double val, double *__restrict__ x) {
    GRID_STRIDE(k, count) x[k] = val;
}
__global__ void start_min_kernel(int64_t psi, const double *__restrict__ pt, const double *__restrict__ st_,
                                 double *part) {
    __shared__ double sh[kT / 32];
    double a = INFINITY, b = INFINITY;
    GRID_STRIDE(e, psi) { a = fmin(a, pt[e]); b = fmin(b, st_[e]); }
    put_min(a, part, SC_SUM_A, sh);
    put_min(b, part, SC_SUM_B, sh);
}
__global__ void start_shift_kernel(int64_t psi, double *__restrict__ pt, double *__restrict__ st_, double dp,
                                   double ds, double *part) {
    __shared__ double sh[kT / 32];
    double ps = 0, sp = 0, ss = 0;
    GRID_STRIDE(e, psi) {
        const double a = pt[e] + dp, b = st_[e] + ds;
        pt[e] = a;
        st_[e] = b;
        ps += a * b;
        sp += a;
        ss += b;
    }
    put_sum(ps, part, SC_NORM_A, sh);
    put_sum(sp, part, SC_SUM_A, sh);
    put_sum(ss, part, SC_SUM_B, sh);
}
__global__ void add_const2_kernel(int64_t psi, double *__restrict__ p, double *__restrict__ s, double dp, double ds) {
    GRID_STRIDE(e, psi) { p[e] += dp; s[e] += ds; }
}
}  // namespace

// s~ = max(c - u_i - v_j, 0) for given duals (warm start)
__global__ void warm_slack_kernel(int64_t psi, const int32_t *__restrict__ si, const int32_t *__restrict__ sj,
                                  const double *__restrict__ c, const double *__restrict__ u,
                                  const double *__restrict__ v, double *__restrict__ s) {
    GRID_STRIDE(e, psi) s[e] = fmax((c[e] - u[si[e]]) - v[sj[e]], 0.0);
}

Error mehrotra_start(Newton &W, Support &S, const double *a_s, const double *b_s, double *u, double *v,
                     int precision, double cg_tol, int max_cg, int *cg_iters, cudaStream_t st, bool warm_duals) {
    const unsigned ge = grid_of(S.psi, W.num_sms);
    fill_kernel<<<ge, kT, 0, st>>>(S.psi, 1.0, S.p);
    OT_LAUNCHED();
    fill_kernel<<<ge, kT, 0, st>>>(S.psi, 1.0, S.s);
    OT_LAUNCHED();
    OT_TRY(schur_setup(W, S, st));
    SolveStats s1, s2;
    // p~ = A^T (A A^T)^+ f : with theta = 1, r1 = f, r2 = r3 = 0 the direction has dp = A^T dy
    Rhs Rf{a_s, b_s, nullptr, nullptr};
    OT_TRY(newton_solve(W, S, Rf, cg_tol, max_cg, precision, W.du, W.dv, W.ds, W.dp, &s1, st));
    if (warm_duals) {
        // the caller's duals (already in u, v) replace the least-squares ones; their negative
        // reduced costs are clipped rather than shifting every slack (Mehrotra's shift would
        // spread one bad prediction over the whole support)
        warm_slack_kernel<<<ge, kT, 0, st>>>(S.psi, S.i, S.j, W.c, u, v, W.ds2);
        OT_LAUNCHED();
    } else {
        // y~ = (A A^T)^+ A c : r2 = c gives dy = y~ and ds = c - A^T y~ = s~
        Rhs Rc{nullptr, nullptr, W.c, nullptr};
        OT_TRY(newton_solve(W, S, Rc, cg_tol, max_cg, precision, u, v, W.ds2, W.dp2, &s2, st));
    }
    if (cg_iters) *cg_iters = s1.cg_iters + s2.cg_iters;
    // dp holds p~, ds2 holds s~
    start_min_kernel<<<ge, kT, 0, st>>>(S.psi, W.dp, W.ds2, W.part);
    OT_LAUNCHED();
    Finish f{2, {SC_SUM_A, SC_SUM_B}, {(int)ge, (int)ge}, {1, 1}};
    OT_TRY(finish(f, W, st));
    double hs[SC_COUNT];
    OT_TRY(read_scalars(W, hs, st));
    const double dpv = std::max(-1.5 * hs[SC_SUM_A], 0.0), dsv = std::max(-1.5 * hs[SC_SUM_B], 0.0);
    start_shift_kernel<<<ge, kT, 0, st>>>(S.psi, W.dp, W.ds2, dpv, dsv, W.part);
    OT_LAUNCHED();
    Finish f2{3, {SC_NORM_A, SC_SUM_A, SC_SUM_B}, {(int)ge, (int)ge, (int)ge}, {0, 0, 0}};
    OT_TRY(finish(f2, W, st));
    OT_TRY(read_scalars(W, hs, st));
    const double ps = hs[SC_NORM_A];
    const double dp2 = 0.5 * ps / hs[SC_SUM_B], ds2 = 0.5 * ps / hs[SC_SUM_A];
    add_const2_kernel<<<ge, kT, 0, st>>>(S.psi, W.dp, W.ds2, dp2, ds2);
    OT_LAUNCHED();
    OT_CUDA(cudaMemcpyAsync(S.p, W.dp, sizeof(double) * S.psi, cudaMemcpyDeviceToDevice, st));
    OT_CUDA(cudaMemcpyAsync(S.s, W.ds2, sizeof(double) * S.psi, cudaMemcpyDeviceToDevice, st));
    if (!(ps > 0) || !std::isfinite(dp2) || !std::isfinite(ds2))
        return fail(OT_ERR_NUMERIC, "initial point: degenerate starting point");
    return ok();
}

}  // namespace ot
