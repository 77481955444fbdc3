// Direct branch near optimality (Sections 4.2-4.3).
//
// S_M = N - V^T M^-1 V is assembled by rows of V: every pair (j, j') of targets sharing a source
// i contributes -theta_ij theta_ij' / M_i; duplicates are combined after a stable sort, so the
// sums are deterministic.  The diagonal is the cancellation-free S_jj = sum_i theta_ij excl_ij/M_i.
//
// Ordering: minimum degree by explicit elimination on the host (ties: smallest index).  Near
// optimality the support approaches a forest, whose S_M is chordal (Theorem 2 and its
// corollary), so a minimum-degree order produces little or no fill.
//
// Numeric LDL^T and the triangular solves are level scheduled: the host groups the columns by
// their level in the dependency DAG of L, and one cooperative launch walks the levels with a
// bounded grid barrier between them, one warp per column.  A pivot d <= eps * S_jj becomes
// +infinity (the modified factorisation mentioned in Section 4.2), which grounds one node per
// connected component of the singular S_M.
#include "chol.cuh"
#include "ordering.h"
#include "primitives.cuh"

#include <algorithm>
#include <cmath>
#include <set>

namespace ot {
namespace {

constexpr int kT = 256;

#define GS(var, count) \
    for (int64_t var = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; var < (count); var += (int64_t)gridDim.x * blockDim.x)

inline unsigned gridn(int64_t work) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(2048, ceil_div(work, kT)));
}

// ----------------------------------------------------------------------------- assembly
// per source row: kept pairs (theta >= drop * row max), kept-only sums, pair counts
__global__ void sp_rows_kernel(int m, const int32_t *__restrict__ rp, const double *__restrict__ th, double drop,
                               uint8_t *__restrict__ keep, double *__restrict__ exd, double *__restrict__ Mt,
                               uint32_t *__restrict__ cnt) {
    GS(i, m) {
        const int lo = rp[i], hi = rp[i + 1];
        double tmax = 0;
        for (int e = lo; e < hi; ++e) tmax = fmax(tmax, th[e]);
        const double cut = drop * tmax;
        int dk = 0;
        double pre = 0;
        for (int e = lo; e < hi; ++e) {
            const bool k = th[e] >= cut && th[e] > 0;
            keep[e] = k ? 1 : 0;
            exd[e] = pre;
            if (k) { pre += th[e]; ++dk; }
        }
        double suf = 0;
        for (int e = hi - 1; e >= lo; --e) {
            exd[e] += suf;
            if (keep[e]) suf += th[e];
        }
        Mt[i] = pre;
        cnt[i] = (uint32_t)(dk * (dk - 1));
    }
}

__global__ void asm_emit_kernel(int m, int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ sj,
                                const double *__restrict__ th, const uint8_t *__restrict__ keep,
                                const double *__restrict__ Mt, const uint32_t *__restrict__ off,
                                uint64_t *__restrict__ key, uint32_t *__restrict__ val, double *__restrict__ raw) {
    GS(i, m) {
        const int lo = rp[i], hi = rp[i + 1];
        uint32_t o = off[i];
        const double mi = Mt[i] > 0 ? 1.0 / Mt[i] : 0.0;
        for (int a = lo; a < hi; ++a) {
            if (!keep[a]) continue;
            for (int b = lo; b < hi; ++b) {
                if (a == b || !keep[b]) continue;
                key[o] = (uint64_t)sj[a] * (uint64_t)n + (uint64_t)sj[b];
                val[o] = o;
                raw[o] = -(th[a] * th[b]) * mi;
                ++o;
            }
        }
    }
}

// diagonal of the kept graph's Schur complement: sum over kept pairs theta * (kept others) / Mt
__global__ void sp_diag_kernel(int n, const int32_t *__restrict__ cp, const int32_t *__restrict__ perm,
                               const int32_t *__restrict__ crow, const double *__restrict__ th,
                               const uint8_t *__restrict__ keep, const double *__restrict__ exd,
                               const double *__restrict__ Mt, double *__restrict__ diag) {
    GS(j, n) {
        double d = 0;
        for (int k = cp[j]; k < cp[j + 1]; ++k) {
            const int e = perm[k];
            if (!keep[e]) continue;
            const double mt = Mt[crow[k]];
            if (mt > 0) d += th[e] * exd[e] / mt;
        }
        diag[j] = d;
    }
}

__global__ void run_flag_kernel(int64_t cnt, const uint64_t *__restrict__ key, uint32_t *__restrict__ f) {
    GS(t, cnt) f[t] = (t == 0 || key[t] != key[t - 1]) ? 1u : 0u;
}

__global__ void run_start_kernel(int64_t cnt, const uint32_t *__restrict__ f, const uint32_t *__restrict__ pos,
                                 uint32_t *__restrict__ start) {
    GS(t, cnt) if (f[t]) start[pos[t]] = (uint32_t)t;
}

// one thread per distinct (row, col): sum its run in sorted (= generation) order
__global__ void run_reduce_kernel(int64_t nu, int64_t cnt, int n, const uint32_t *__restrict__ start,
                                  const uint64_t *__restrict__ key, const uint32_t *__restrict__ val,
                                  const double *__restrict__ raw, int32_t *__restrict__ Aj,
                                  int32_t *__restrict__ Arow, double *__restrict__ Ax) {
    GS(u, nu) {
        const uint32_t s = start[u], e = (u + 1 < nu) ? start[u + 1] : (uint32_t)cnt;
        double acc = 0;
        for (uint32_t t = s; t < e; ++t) acc += raw[val[t]];
        Ax[u] = acc;
        Arow[u] = (int32_t)(key[s] / (uint64_t)n);
        Aj[u] = (int32_t)(key[s] % (uint64_t)n);
    }
}

__global__ void ptr_from_sorted_kernel(int64_t nnz, int n, const int32_t *__restrict__ row, int32_t *__restrict__ p) {
    GS(q, (int64_t)n + 1) {
        int64_t lo = 0, hi = nnz;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (row[mid] < q) lo = mid + 1; else hi = mid;
        }
        p[q] = (int32_t)lo;
    }
}

// A entry (r, c) -> position of (iperm r, iperm c) in the CSC of L when it is below the diagonal
__global__ void a2l_kernel(int n, const int32_t *__restrict__ Ap, const int32_t *__restrict__ Aj,
                           const int32_t *__restrict__ iperm, const int32_t *__restrict__ Lp,
                           const int32_t *__restrict__ Li, int64_t *__restrict__ a2l, int *err) {
    GS(r, n) {
        const int pr = iperm[r];
        for (int e = Ap[r]; e < Ap[r + 1]; ++e) {
            const int pc = iperm[Aj[e]];
            if (pr <= pc) { a2l[e] = -1; continue; }
            int lo = Lp[pc], hi = Lp[pc + 1];
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (Li[mid] < pr) lo = mid + 1; else hi = mid;
            }
            if (lo < Lp[pc + 1] && Li[lo] == pr) a2l[e] = lo;
            else { a2l[e] = -1; atomicExch(err, 1); }
        }
    }
}

// ----------------------------------------------------------------------------- numeric
__global__ void ldl_init_kernel(int n, int64_t nnzL, const int32_t *__restrict__ perm,
                                const double *__restrict__ Adiag, double *__restrict__ Lx,
                                double *__restrict__ dperm, int *__restrict__ done) {
    GS(t, nnzL) Lx[t] = 0.0;
    GS(q, n) {
        dperm[q] = Adiag[perm[q]];
        done[q] = 0;
    }
}

__global__ void ldl_scatter_kernel(int64_t nnzA, const int64_t *__restrict__ a2l, const double *__restrict__ Ax,
                                   double *__restrict__ Lx) {
    GS(e, nnzA) if (a2l[e] >= 0) Lx[a2l[e]] = Ax[e];
}

// Level-scheduled kernels.  Columns are grouped by their level in the dependency DAG of L
// (level(q) = 1 + max level of the columns q depends on); columns of one level are independent.
// One cooperative launch walks the levels with a grid barrier between them (bounded waits, see
// grid_barrier), one warp per column.

// left-looking column: L(:,q) and D_q from the already final columns of lower levels
__device__ __forceinline__ void ldl_column(int q, int lane, const int32_t *__restrict__ Lp,
                                           const int32_t *__restrict__ Li, const int32_t *__restrict__ Rp,
                                           const int32_t *__restrict__ Rj, const int64_t *__restrict__ Rpos,
                                           double *Lx, const double *__restrict__ dperm, double *D, int *err,
                                           double eps) {
    const int lo = Lp[q], hi = Lp[q + 1];
    const double d0 = dperm[q];
    double d = d0;
    for (int t = Rp[q]; t < Rp[q + 1]; ++t) {
        const int k = Rj[t];
        const double dk = D[k];
        if (isinf(dk)) continue;
        const int64_t pq = Rpos[t];
        const double ljk = Lx[pq];
        d -= ljk * ljk * dk;
        const double f = dk * ljk;
        const int kend = Lp[k + 1];
        for (int64_t idx = pq + 1 + lane; idx < kend; idx += 32) {
            const int r = Li[idx];
            const double lrk = Lx[idx];
            int a = lo, b = hi;
            while (a < b) {
                int mid = (a + b) >> 1;
                if (Li[mid] < r) a = mid + 1; else b = mid;
            }
            if (a < hi && Li[a] == r) Lx[a] -= lrk * f;
            else atomicExch(err, 2);
        }
        __syncwarp();
    }
    const bool inf_pivot = !(d > eps * d0);
    for (int idx = lo + lane; idx < hi; idx += 32) Lx[idx] = inf_pivot ? 0.0 : Lx[idx] / d;
    if (lane == 0) D[q] = inf_pivot ? INFINITY : d;
}

__global__ void __launch_bounds__(kT)
ldl_numeric_kernel(int nlev, const int32_t *__restrict__ lvl_ptr, const int32_t *__restrict__ lvl_cols,
                   const int32_t *__restrict__ Lp, const int32_t *__restrict__ Li, const int32_t *__restrict__ Rp,
                   const int32_t *__restrict__ Rj, const int64_t *__restrict__ Rpos, double *Lx,
                   const double *__restrict__ dperm, double *D, unsigned *bar, int *err, double eps) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int lv = 0; lv < nlev; ++lv) {
        for (int c = lvl_ptr[lv] + gw; c < lvl_ptr[lv + 1]; c += nw)
            ldl_column(lvl_cols[c], lane, Lp, Li, Rp, Rj, Rpos, Lx, dperm, D, err, eps);
        if (!grid_barrier(bar, gridDim.x, err)) return;
    }
}

// forward (z = L^-1 P b, y = D^-1 z, levels ascending) then backward (x = L^-T y, levels
// descending), out = P^T x; one launch per solve
__global__ void __launch_bounds__(kT)
ldl_solve_kernel(int nlev, const int32_t *__restrict__ lvl_ptr, const int32_t *__restrict__ lvl_cols,
                 const int32_t *__restrict__ perm, const int32_t *__restrict__ Lp, const int32_t *__restrict__ Li,
                 const int32_t *__restrict__ Rp, const int32_t *__restrict__ Rj,
                 const int64_t *__restrict__ Rpos, const double *__restrict__ Lx, const double *__restrict__ D,
                 const double *__restrict__ b, double *z, double *y, double *x, double *out, unsigned *bar,
                 int *err) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int lv = 0; lv < nlev; ++lv) {
        for (int c = lvl_ptr[lv] + gw; c < lvl_ptr[lv + 1]; c += nw) {
            const int q = lvl_cols[c];
            double acc = 0;
            for (int t = Rp[q] + lane; t < Rp[q + 1]; t += 32) acc += Lx[Rpos[t]] * z[Rj[t]];
            acc = warp_sum(acc);
            if (lane == 0) {
                const double zq = b[perm[q]] - acc;
                z[q] = zq;
                const double dq = D[q];
                y[q] = isinf(dq) ? 0.0 : zq / dq;
            }
        }
        if (!grid_barrier(bar, gridDim.x, err)) return;
    }
    for (int lv = nlev - 1; lv >= 0; --lv) {
        for (int c = lvl_ptr[lv] + gw; c < lvl_ptr[lv + 1]; c += nw) {
            const int q = lvl_cols[c];
            double acc = 0;
            for (int t = Lp[q] + lane; t < Lp[q + 1]; t += 32) acc += Lx[t] * x[Li[t]];
            acc = warp_sum(acc);
            if (lane == 0) {
                const double xq = y[q] - acc;
                x[q] = xq;
                out[perm[q]] = xq;
            }
        }
        if (lv > 0 && !grid_barrier(bar, gridDim.x, err)) return;
    }
}

template <typename T>
Error dalloc(T **p, int64_t count) {
    OT_CUDA(cudaMalloc((void **)p, sizeof(T) * (size_t)std::max<int64_t>(count, 1)));
    return ok();
}

template <typename T>
void dfree(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

// cooperative grid for the level-scheduled kernels: enough warps for the widest level, capped by
// what can be co-resident
template <typename K>
Error coop_grid(K kernel, int width, int *grid) {
    int dev = 0, sms = 0, per_sm = 0;
    OT_CUDA(cudaGetDevice(&dev));
    OT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    OT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kT, 0));
    const int want = (int)std::max<int64_t>(1, ceil_div(width, kT / 32));
    *grid = std::max(1, std::min(want, std::max(per_sm, 1) * sms));
    return ok();
}

}  // namespace

Error chol_alloc(Chol &C, int32_t n) {
    C.n = n;
    OT_TRY(dalloc(&C.Ap, (int64_t)n + 1));
    OT_TRY(dalloc(&C.Adiag, n));
    OT_TRY(dalloc(&C.perm, n));
    OT_TRY(dalloc(&C.iperm, n));
    OT_TRY(dalloc(&C.Lp, (int64_t)n + 1));
    OT_TRY(dalloc(&C.Rp, (int64_t)n + 1));
    OT_TRY(dalloc(&C.D, n));
    OT_TRY(dalloc(&C.dperm, n));
    OT_TRY(dalloc(&C.z, n));
    OT_TRY(dalloc(&C.x, n));
    OT_TRY(dalloc(&C.y, n));
    OT_TRY(dalloc(&C.done, n));
    OT_TRY(dalloc(&C.counter, 1));
    OT_TRY(dalloc(&C.bar, 2));
    OT_TRY(dalloc(&C.lvl_cols, n));
    OT_TRY(dalloc(&C.err, 1));
    if (C.max_nnzL <= 0) C.max_nnzL = std::max<int64_t>(48LL * n, 1LL << 20);
    return ok();
}

void chol_free(Chol &C) {
    dfree(C.Ap); dfree(C.Aj); dfree(C.Ax); dfree(C.Adiag); dfree(C.a2l); dfree(C.keep); dfree(C.exd); dfree(C.Mt);
    dfree(C.perm); dfree(C.iperm); dfree(C.Lp); dfree(C.Li); dfree(C.Rp); dfree(C.Rj); dfree(C.Rpos);
    dfree(C.Lx); dfree(C.D); dfree(C.dperm); dfree(C.z); dfree(C.x); dfree(C.y); dfree(C.done); dfree(C.counter); dfree(C.bar); dfree(C.lvl_ptr); dfree(C.lvl_cols);
    dfree(C.err);
    C = Chol();
}

Error chol_assemble(Chol &C, Newton &W, const Support &S, double drop, bool *pattern_changed, cudaStream_t st) {
    const int m = W.m, n = W.n;
    if (S.psi > C.capE) {
        dfree(C.keep); dfree(C.exd);
        C.capE = std::max<int64_t>(S.psi, (int64_t)(1.5 * C.capE));
        OT_TRY(dalloc(&C.keep, C.capE));
        OT_TRY(dalloc(&C.exd, C.capE));
    }
    if (!C.Mt) OT_TRY(dalloc(&C.Mt, m));
    C.drop = drop;
    DevTemp<uint32_t> cnt, off, tot;
    OT_TRY(cnt.alloc(m, st));
    OT_TRY(off.alloc(m, st));
    OT_TRY(tot.alloc(1, st));
    sp_rows_kernel<<<gridn(m), kT, 0, st>>>(m, S.row_ptr, W.theta, drop, C.keep, C.exd, C.Mt, cnt.p);
    OT_LAUNCHED();
    OT_TRY(scan_exclusive_u32(cnt.p, off.p, m, tot.p, st));
    uint32_t total = 0;
    OT_CUDA(cudaMemcpyAsync(&total, tot.p, sizeof(total), cudaMemcpyDeviceToHost, st));
    OT_CUDA(cudaStreamSynchronize(st));
    DevTemp<uint64_t> key;
    DevTemp<uint32_t> val, flag, pos, start;
    DevTemp<double> raw;
    OT_TRY(key.alloc(total, st)); OT_TRY(val.alloc(total, st)); OT_TRY(raw.alloc(total, st));
    OT_TRY(flag.alloc(total, st)); OT_TRY(pos.alloc(total, st)); OT_TRY(start.alloc(total, st));
    uint32_t nu = 0;
    if (total > 0) {
        asm_emit_kernel<<<gridn(m), kT, 0, st>>>(m, n, S.row_ptr, S.j, W.theta, C.keep, C.Mt, off.p, key.p, val.p,
                                                 raw.p);
        OT_LAUNCHED();
        int bits = 1;
        while (bits < 64 && (((uint64_t)n * n - 1) >> bits)) ++bits;
        OT_TRY(radix_sort_pairs(key.p, val.p, total, bits, st));
        run_flag_kernel<<<gridn(total), kT, 0, st>>>(total, key.p, flag.p);
        OT_LAUNCHED();
        OT_TRY(scan_exclusive_u32(flag.p, pos.p, total, tot.p, st));
        OT_CUDA(cudaMemcpyAsync(&nu, tot.p, sizeof(nu), cudaMemcpyDeviceToHost, st));
        OT_CUDA(cudaStreamSynchronize(st));
    }
    if ((int64_t)nu > C.capA) {
        dfree(C.Aj); dfree(C.Ax); dfree(C.a2l);
        C.capA = std::max<int64_t>(nu, (int64_t)(1.5 * C.capA));
        OT_TRY(dalloc(&C.Aj, C.capA));
        OT_TRY(dalloc(&C.Ax, C.capA));
        OT_TRY(dalloc(&C.a2l, C.capA));
    }
    DevTemp<int32_t> arow;
    OT_TRY(arow.alloc(nu, st));
    if (nu > 0) {
        run_start_kernel<<<gridn(total), kT, 0, st>>>(total, flag.p, pos.p, start.p);
        OT_LAUNCHED();
        run_reduce_kernel<<<gridn(nu), kT, 0, st>>>(nu, total, n, start.p, key.p, val.p, raw.p, C.Aj, arow.p, C.Ax);
        OT_LAUNCHED();
    }
    ptr_from_sorted_kernel<<<gridn((int64_t)n + 1), kT, 0, st>>>(nu, n, arow.p, C.Ap);
    OT_LAUNCHED();
    sp_diag_kernel<<<gridn(n), kT, 0, st>>>(n, S.col_ptr, S.col_perm, S.col_row, W.theta, C.keep, C.exd, C.Mt,
                                            C.Adiag);
    OT_LAUNCHED();
    C.nnzA = nu;
    // pattern on the host (for the symbolic analysis and change detection)
    std::vector<int32_t> hp(n + 1), hj(nu);
    OT_CUDA(cudaMemcpyAsync(hp.data(), C.Ap, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, st));
    if (nu) OT_CUDA(cudaMemcpyAsync(hj.data(), C.Aj, sizeof(int32_t) * nu, cudaMemcpyDeviceToHost, st));
    OT_CUDA(cudaStreamSynchronize(st));
    const bool changed = !C.have_symbolic || hp != C.hAp || hj != C.hAj;
    if (changed) {
        C.hAp.swap(hp);
        C.hAj.swap(hj);
        C.have_symbolic = false;
    }
    *pattern_changed = changed;
    return ok();
}

Error chol_symbolic(Chol &C, cudaStream_t st) {
    const int n = C.n;
    ordering::Graph g;
    g.n = n;
    g.ptr = C.hAp;
    g.adj = C.hAj;
    // minimum degree while its fill stays small (near optimality: a near-forest, Theorem 2),
    // otherwise nested dissection by level structures
    // 1) a chordal S_M (a forest support, Theorem 2) factors with zero fill in reverse
    //    maximum-cardinality-search order; 2) otherwise minimum degree while its fill stays
    //    small; 3) otherwise nested dissection by level structures.
    const int64_t nnzA = (int64_t)g.adj.size();
    const int64_t lower = nnzA / 2;
    std::vector<int32_t> perm, Lp, Li;
    bool ok_sym = false;
    // reuse the last ordering while the pattern has not grown much and its fill stays moderate
    if ((int)C.hperm.size() == n && nnzA <= (C.perm_nnzA * 5) / 4) {
        perm = C.hperm;
        ok_sym = ordering::symbolic_factor(g, perm, std::min<int64_t>(C.max_nnzL, 2 * C.perm_nnzL + lower + n), Lp, Li);
    }
    if (!ok_sym) {
        ordering::mcs_order(g, perm);
        ok_sym = ordering::symbolic_factor(g, perm, lower, Lp, Li);
        if (!ok_sym) {
            const bool sparse = nnzA <= 16LL * n;
            if (!sparse || !ordering::minimum_degree(g, std::min<int64_t>(64LL * n + 4096, 1LL << 22), perm))
                ordering::nested_dissection(g, perm);
            ok_sym = ordering::symbolic_factor(g, perm, C.max_nnzL, Lp, Li);
        }
        if (ok_sym) {
            C.hperm = perm;
            C.perm_nnzA = nnzA;
            C.perm_nnzL = (int64_t)Li.size();
        }
    }
    if (!ok_sym) return fail(OT_ERR_UNSUPPORTED, "symbolic: fill above the direct-solver limit");
    const int64_t nnzL = (int64_t)Li.size();
    std::vector<int32_t> iperm(n);
    for (int q = 0; q < n; ++q) iperm[perm[q]] = q;
    std::vector<int32_t> Rp(n + 1, 0), Rj(nnzL);
    std::vector<int64_t> Rpos(nnzL);
    for (int64_t t = 0; t < nnzL; ++t) Rp[Li[t] + 1]++;
    for (int r = 0; r < n; ++r) Rp[r + 1] += Rp[r];
    std::vector<int32_t> fill(Rp.begin(), Rp.end() - 1);
    for (int q = 0; q < n; ++q)
        for (int t = Lp[q]; t < Lp[q + 1]; ++t) {
            const int r = Li[t];
            Rj[fill[r]] = q;
            Rpos[fill[r]] = t;
            fill[r]++;
        }
    if (nnzL > C.capL) {
        dfree(C.Li); dfree(C.Rj); dfree(C.Rpos); dfree(C.Lx);
        C.capL = std::max<int64_t>(nnzL, (int64_t)(1.5 * C.capL));
        OT_TRY(dalloc(&C.Li, C.capL));
        OT_TRY(dalloc(&C.Rj, C.capL));
        OT_TRY(dalloc(&C.Rpos, C.capL));
        OT_TRY(dalloc(&C.Lx, C.capL));
    }
    OT_CUDA(cudaMemcpyAsync(C.perm, perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
    OT_CUDA(cudaMemcpyAsync(C.iperm, iperm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
    OT_CUDA(cudaMemcpyAsync(C.Lp, Lp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st));
    OT_CUDA(cudaMemcpyAsync(C.Rp, Rp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st));
    if (nnzL) {
        OT_CUDA(cudaMemcpyAsync(C.Li, Li.data(), sizeof(int32_t) * nnzL, cudaMemcpyHostToDevice, st));
        OT_CUDA(cudaMemcpyAsync(C.Rj, Rj.data(), sizeof(int32_t) * nnzL, cudaMemcpyHostToDevice, st));
        OT_CUDA(cudaMemcpyAsync(C.Rpos, Rpos.data(), sizeof(int64_t) * nnzL, cudaMemcpyHostToDevice, st));
    }
    C.nnzL = nnzL;
    C.fill_pct = 100.0 * (double)nnzL / ((double)n * n);
    // levels of the dependency DAG of L: level(r) >= level(q) + 1 for every L(r, q) != 0
    {
        std::vector<int32_t> level(n, 0);
        int nlev = 0;
        for (int q = 0; q < n; ++q) {
            nlev = std::max(nlev, level[q] + 1);
            for (int t = Lp[q]; t < Lp[q + 1]; ++t) level[Li[t]] = std::max(level[Li[t]], level[q] + 1);
        }
        std::vector<int32_t> lptr(nlev + 1, 0), lcols(n);
        for (int q = 0; q < n; ++q) lptr[level[q] + 1]++;
        int width = 0;
        for (int l = 0; l < nlev; ++l) { width = std::max(width, lptr[l + 1]); lptr[l + 1] += lptr[l]; }
        std::vector<int32_t> fillp(lptr.begin(), lptr.end() - 1);
        for (int q = 0; q < n; ++q) lcols[fillp[level[q]]++] = q;
        if (nlev + 1 > C.cap_lev) {
            dfree(C.lvl_ptr);
            C.cap_lev = std::max(nlev + 1, 2 * C.cap_lev);
            OT_TRY(dalloc(&C.lvl_ptr, C.cap_lev));
        }
        OT_CUDA(cudaMemcpyAsync(C.lvl_ptr, lptr.data(), sizeof(int32_t) * (nlev + 1), cudaMemcpyHostToDevice, st));
        OT_CUDA(cudaMemcpyAsync(C.lvl_cols, lcols.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
        OT_CUDA(cudaStreamSynchronize(st));
        C.nlev = nlev;
        C.max_width = width;
    }
    OT_CUDA(cudaMemsetAsync(C.err, 0, sizeof(int), st));
    if (C.nnzA > 0) {
        a2l_kernel<<<gridn(n), kT, 0, st>>>(n, C.Ap, C.Aj, C.iperm, C.Lp, C.Li, C.a2l, C.err);
        OT_LAUNCHED();
    }
    int errv = 0;
    OT_CUDA(cudaMemcpyAsync(&errv, C.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    OT_CUDA(cudaStreamSynchronize(st));
    if (errv) return fail(OT_ERR_NUMERIC, "symbolic: assembled entry outside the pattern of L");
    C.have_symbolic = true;
    return ok();
}

Error chol_numeric(Chol &C, double eps, cudaStream_t st) {
    const int n = C.n;
    ldl_init_kernel<<<gridn(std::max<int64_t>(C.nnzL, n)), kT, 0, st>>>(n, C.nnzL, C.perm, C.Adiag, C.Lx, C.dperm,
                                                                        C.done);
    OT_LAUNCHED();
    if (C.nnzA > 0) {
        ldl_scatter_kernel<<<gridn(C.nnzA), kT, 0, st>>>(C.nnzA, C.a2l, C.Ax, C.Lx);
        OT_LAUNCHED();
    }
    OT_CUDA(cudaMemsetAsync(C.bar, 0, 2 * sizeof(unsigned), st));
    OT_CUDA(cudaMemsetAsync(C.err, 0, sizeof(int), st));
    int grid = 1;
    OT_TRY(coop_grid(ldl_numeric_kernel, C.max_width, &grid));
    int nlev = C.nlev;
    const int32_t *lp = C.lvl_ptr, *lc = C.lvl_cols, *Lp = C.Lp, *Li = C.Li, *Rp = C.Rp, *Rj = C.Rj;
    const int64_t *Rpos = C.Rpos;
    double *Lx = C.Lx, *D = C.D;
    const double *dp = C.dperm;
    unsigned *bar = C.bar;
    int *err = C.err;
    void *args[] = {&nlev, &lp, &lc, &Lp, &Li, &Rp, &Rj, &Rpos, &Lx, &dp, &D, &bar, &err, &eps};
    ktimer_begin(KT_LDL_NUMERIC, st);
    OT_CUDA(cudaLaunchCooperativeKernel((void *)ldl_numeric_kernel, dim3(grid), dim3(kT), args, 0, st));
    OT_LAUNCHED();
    ktimer_end(KT_LDL_NUMERIC, st);
    int errv = 0;
    OT_CUDA(cudaMemcpyAsync(&errv, C.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    OT_CUDA(cudaStreamSynchronize(st));
    if (errv == OT_ERR_TIMEOUT) return fail(OT_ERR_TIMEOUT, "ldl: grid barrier wait limit reached");
    if (errv) return fail(OT_ERR_NUMERIC, "ldl: update outside the pattern of L");
    return ok();
}

Error chol_solve(Chol &C, const double *b, double *x, cudaStream_t st) {
    OT_CUDA(cudaMemsetAsync(C.bar, 0, 2 * sizeof(unsigned), st));
    int grid = 1;
    OT_TRY(coop_grid(ldl_solve_kernel, C.max_width, &grid));
    int nlev = C.nlev;
    const int32_t *lp = C.lvl_ptr, *lc = C.lvl_cols, *pm = C.perm, *Lp = C.Lp, *Li = C.Li, *Rp = C.Rp, *Rj = C.Rj;
    const int64_t *Rpos = C.Rpos;
    const double *Lx = C.Lx, *D = C.D;
    double *z = C.z, *y = C.y, *xx = C.x;
    unsigned *bar = C.bar;
    int *err = C.err;
    void *args[] = {&nlev, &lp, &lc, &pm, &Lp, &Li, &Rp, &Rj, &Rpos, &Lx, &D, &b, &z, &y, &xx, &x, &bar, &err};
    ktimer_begin(KT_LDL_SOLVE, st);
    OT_CUDA(cudaLaunchCooperativeKernel((void *)ldl_solve_kernel, dim3(grid), dim3(kT), args, 0, st));
    OT_LAUNCHED();
    ktimer_end(KT_LDL_SOLVE, st);
    return ok();
}

}  // namespace ot
