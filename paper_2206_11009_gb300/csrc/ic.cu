// Incomplete Cholesky with a drop tolerance in a multicolour order (see ic.cuh).
#include "ic.cuh"

#include <algorithm>
#include <cmath>

namespace ot {
namespace {

constexpr int kT = 256;

template <typename T>
Error ic_dalloc(T **p, int64_t count) {
    OT_CUDA(cudaMalloc((void **)p, sizeof(T) * (size_t)std::max<int64_t>(count, 1)));
    return ok();
}
template <typename T>
void ic_dfree(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

inline unsigned blocks_for(int64_t count) { return (unsigned)std::max<int64_t>(1, ceil_div(count, kT)); }

// Rows [r0, r1) of one colour, one thread per row (their entries all lie in earlier colours):
//   l_rs = (S_rs - sum_{t < s} l_rt l_st d_t) / d_s   over the pattern, in increasing s,
//   d_r  = S_rr - sum_s l_rs^2 d_s,
// with the drop rule and the +infinity pivot rule of ic.cuh.  Terms of grounded columns (d = inf)
// are zero.
__global__ void ic_rows_kernel(int r0, int r1, const int32_t *__restrict__ Lp, const int32_t *__restrict__ Lj,
                               const int64_t *__restrict__ Lsrc, const double *__restrict__ Ax,
                               const double *__restrict__ Ad, double tau, double eps, double *__restrict__ Lx,
                               double *__restrict__ D, int32_t *__restrict__ dropped) {
    const int r = r0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= r1) return;
    const int lo = Lp[r], hi = Lp[r + 1];
    const double arr = Ad[r];
    double dsum = 0.0;
    int ndrop = 0;
    for (int e = lo; e < hi; ++e) {
        const int s = Lj[e];
        double acc = Ax[Lsrc[e]];
        int a = lo, b = Lp[s];
        const int bend = Lp[s + 1];
        while (a < e && b < bend) {
            const int ta = Lj[a], tb = Lj[b];
            if (ta == tb) {
                const double dt = D[ta];
                if (dt < INFINITY) acc -= Lx[a] * Lx[b] * dt;
                ++a;
                ++b;
            } else if (ta < tb) {
                ++a;
            } else {
                ++b;
            }
        }
        const double ds = D[s];
        double l = ds < INFINITY ? acc / ds : 0.0;
        if (l != 0.0 && fabs(l * ds) < tau * sqrt(arr * Ad[s])) {
            l = 0.0;
            ++ndrop;
        }
        Lx[e] = l;
        if (ds < INFINITY) dsum += l * l * ds;
    }
    const double d = arr - dsum;
    D[r] = d > eps * arr ? d : INFINITY;
    if (ndrop) atomicAdd(dropped, ndrop);
}

// forward substitution for one colour: y_r = b_{perm r} - sum_s l_rs y_s
__global__ void ic_fwd_kernel(int r0, int r1, const int32_t *__restrict__ perm, const int32_t *__restrict__ Lp,
                              const int32_t *__restrict__ Lj, const double *__restrict__ Lx,
                              const double *__restrict__ b, double *__restrict__ y) {
    const int r = r0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= r1) return;
    double acc = b[perm[r]];
    for (int e = Lp[r]; e < Lp[r + 1]; ++e) acc -= Lx[e] * y[Lj[e]];
    y[r] = acc;
}

// backward substitution for one colour: x_s = y_s / d_s - sum_{r > s} l_rs x_r (through U = L^T);
// the result goes both to the new-order work vector and to the caller's vector in target order
__global__ void ic_bwd_kernel(int r0, int r1, const int32_t *__restrict__ perm, const int32_t *__restrict__ Up,
                              const int32_t *__restrict__ Uj, const int64_t *__restrict__ Upos,
                              const double *__restrict__ Lx, const double *__restrict__ D,
                              double *__restrict__ y, double *__restrict__ x) {
    const int s = r0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= r1) return;
    const double d = D[s];
    double acc = d < INFINITY ? y[s] / d : 0.0;
    for (int e = Up[s]; e < Up[s + 1]; ++e) acc -= Lx[Upos[e]] * y[Uj[e]];
    y[s] = acc;   // y now holds x in the new order (rows of later colours were finished before)
    x[perm[s]] = acc;
}

__global__ void ic_gather_kernel(int n, const int32_t *__restrict__ perm, const double *__restrict__ src,
                                 double *__restrict__ dst) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) dst[r] = src[perm[r]];
}

}  // namespace

Error ic_alloc(IncChol &F, int32_t n) {
    F.n = n;
    OT_TRY(ic_dalloc(&F.perm, n));
    OT_TRY(ic_dalloc(&F.Lp, (int64_t)n + 1));
    OT_TRY(ic_dalloc(&F.Up, (int64_t)n + 1));
    OT_TRY(ic_dalloc(&F.D, n));
    OT_TRY(ic_dalloc(&F.Ad, n));
    OT_TRY(ic_dalloc(&F.y, n));
    OT_TRY(ic_dalloc(&F.dropped, 1));
    return ok();
}

void ic_free(IncChol &F) {
    ic_dfree(F.perm); ic_dfree(F.Lp); ic_dfree(F.Lj); ic_dfree(F.Lsrc); ic_dfree(F.Lx); ic_dfree(F.Up);
    ic_dfree(F.Uj); ic_dfree(F.Upos); ic_dfree(F.D); ic_dfree(F.Ad); ic_dfree(F.y); ic_dfree(F.dropped);
    F = IncChol();
}

Error ic_factor(IncChol &F, const Chol &C, double tau, double eps, cudaStream_t st) {
    const int n = C.n;
    if (F.n != n || !F.perm) return fail(OT_ERR_ARG, "ic_factor: not allocated for this size");
    if ((int)C.hAp.size() != n + 1) return fail(OT_ERR_ARG, "ic_factor: S_M not assembled");
    const std::vector<int32_t> &Ap0 = C.hAp, &Aj0 = C.hAj;
    // the pattern: the entries of S_M that survive the drop test on their own value,
    // |S_rs| >= tau sqrt(S_rr S_ss) (the rest would be dropped at once); values from the device
    const int64_t nnzA = (int64_t)Aj0.size();
    std::vector<double> ax(nnzA), ad(n);
    if (nnzA) OT_CUDA(cudaMemcpyAsync(ax.data(), C.Ax, sizeof(double) * nnzA, cudaMemcpyDeviceToHost, st));
    OT_CUDA(cudaMemcpyAsync(ad.data(), C.Adiag, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    OT_CUDA(cudaStreamSynchronize(st));
    std::vector<int32_t> Ap(n + 1, 0), Aj;
    std::vector<int64_t> Asrc;
    Aj.reserve(nnzA);
    Asrc.reserve(nnzA);
    for (int v = 0; v < n; ++v) {
        for (int e = Ap0[v]; e < Ap0[v + 1]; ++e) {
            const int u = Aj0[e];
            if (u == v || !(std::fabs(ax[e]) >= tau * std::sqrt(ad[v] * ad[u]))) continue;
            Aj.push_back(u);
            Asrc.push_back(e);
        }
        Ap[v + 1] = (int32_t)Aj.size();
    }
    // greedy colouring in target order: the smallest colour no earlier neighbour holds
    std::vector<int32_t> color(n, -1), seen;
    int nc = 0;
    for (int v = 0; v < n; ++v) {
        for (int e = Ap[v]; e < Ap[v + 1]; ++e) {
            const int c = color[Aj[e]];
            if (c >= 0) seen[c] = v;
        }
        int c = 0;
        while (c < nc && seen[c] == v) ++c;
        color[v] = c;
        if (c == nc) { ++nc; seen.push_back(-1); }
    }
    std::vector<int32_t> cptr(nc + 1, 0), perm(n), iperm(n);
    for (int v = 0; v < n; ++v) cptr[color[v] + 1]++;
    for (int c = 0; c < nc; ++c) cptr[c + 1] += cptr[c];
    {
        std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
        for (int v = 0; v < n; ++v) {
            const int r = fill[color[v]]++;
            perm[r] = v;
            iperm[v] = r;
        }
    }
    // L: for new row r, the neighbours with a smaller new index (all in earlier colours), sorted
    std::vector<int32_t> Lp(n + 1, 0), Lj;
    std::vector<int64_t> Lsrc;
    Lj.reserve(Aj.size() / 2 + 1);
    Lsrc.reserve(Aj.size() / 2 + 1);
    std::vector<std::pair<int32_t, int64_t>> row;
    for (int r = 0; r < n; ++r) {
        const int v = perm[r];
        row.clear();
        for (int e = Ap[v]; e < Ap[v + 1]; ++e) {
            const int s = iperm[Aj[e]];
            if (s < r) row.push_back({s, Asrc[e]});
        }
        std::sort(row.begin(), row.end());
        for (auto &pr : row) { Lj.push_back(pr.first); Lsrc.push_back(pr.second); }
        Lp[r + 1] = (int32_t)Lj.size();
    }
    const int64_t nnzL = (int64_t)Lj.size();
    // U = L^T by rows: row s lists (r, position of l_rs), r increasing
    std::vector<int32_t> Up(n + 1, 0), Uj(nnzL);
    std::vector<int64_t> Upos(nnzL);
    for (int64_t t = 0; t < nnzL; ++t) Up[Lj[t] + 1]++;
    for (int s = 0; s < n; ++s) Up[s + 1] += Up[s];
    {
        std::vector<int32_t> fill(Up.begin(), Up.end() - 1);
        for (int r = 0; r < n; ++r)
            for (int t = Lp[r]; t < Lp[r + 1]; ++t) {
                const int q = fill[Lj[t]]++;
                Uj[q] = r;
                Upos[q] = t;
            }
    }
    if (nnzL > F.capL) {
        ic_dfree(F.Lj); ic_dfree(F.Lsrc); ic_dfree(F.Lx); ic_dfree(F.Uj); ic_dfree(F.Upos);
        F.capL = std::max<int64_t>(nnzL, (int64_t)(1.5 * F.capL));
        OT_TRY(ic_dalloc(&F.Lj, F.capL));
        OT_TRY(ic_dalloc(&F.Lsrc, F.capL));
        OT_TRY(ic_dalloc(&F.Lx, F.capL));
        OT_TRY(ic_dalloc(&F.Uj, F.capL));
        OT_TRY(ic_dalloc(&F.Upos, F.capL));
    }
    OT_CUDA(cudaMemcpyAsync(F.perm, perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
    OT_CUDA(cudaMemcpyAsync(F.Lp, Lp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st));
    OT_CUDA(cudaMemcpyAsync(F.Up, Up.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st));
    if (nnzL) {
        OT_CUDA(cudaMemcpyAsync(F.Lj, Lj.data(), sizeof(int32_t) * nnzL, cudaMemcpyHostToDevice, st));
        OT_CUDA(cudaMemcpyAsync(F.Lsrc, Lsrc.data(), sizeof(int64_t) * nnzL, cudaMemcpyHostToDevice, st));
        OT_CUDA(cudaMemcpyAsync(F.Uj, Uj.data(), sizeof(int32_t) * nnzL, cudaMemcpyHostToDevice, st));
        OT_CUDA(cudaMemcpyAsync(F.Upos, Upos.data(), sizeof(int64_t) * nnzL, cudaMemcpyHostToDevice, st));
    }
    ic_gather_kernel<<<blocks_for(n), kT, 0, st>>>(n, F.perm, C.Adiag, F.Ad);
    OT_LAUNCHED();
    OT_CUDA(cudaMemsetAsync(F.dropped, 0, sizeof(int32_t), st));
    for (int c = 0; c < nc; ++c) {
        const int r0 = cptr[c], r1 = cptr[c + 1];
        ic_rows_kernel<<<blocks_for(r1 - r0), kT, 0, st>>>(r0, r1, F.Lp, F.Lj, F.Lsrc, C.Ax, F.Ad, tau, eps, F.Lx,
                                                           F.D, F.dropped);
        OT_LAUNCHED();
    }
    // the host vectors above must outlive the asynchronous copies
    OT_CUDA(cudaStreamSynchronize(st));
    F.hcolor_ptr = cptr;
    F.ncolors = nc;
    F.nnzL = nnzL;
    F.tau = tau;
    return ok();
}

Error ic_apply(const IncChol &F, const double *b, double *x, cudaStream_t st) {
    const int nc = F.ncolors;
    for (int c = 0; c < nc; ++c) {
        const int r0 = F.hcolor_ptr[c], r1 = F.hcolor_ptr[c + 1];
        ic_fwd_kernel<<<blocks_for(r1 - r0), kT, 0, st>>>(r0, r1, F.perm, F.Lp, F.Lj, F.Lx, b, F.y);
        OT_LAUNCHED();
    }
    for (int c = nc - 1; c >= 0; --c) {
        const int r0 = F.hcolor_ptr[c], r1 = F.hcolor_ptr[c + 1];
        ic_bwd_kernel<<<blocks_for(r1 - r0), kT, 0, st>>>(r0, r1, F.perm, F.Up, F.Uj, F.Upos, F.Lx, F.D, F.y, x);
        OT_LAUNCHED();
    }
    return ok();
}

}  // namespace ot
