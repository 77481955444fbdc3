// Solver driver and C ABI: the outer iteration of the hybrid IPM / column-generation method
// (Section 3.4's commented listing: residuals, mu, sigma and r3, Newton direction, step lengths,
// update, pricing, support update), with the readings stated in ot_ipm.h.
#include "chol.cuh"
#include "dense32.cuh"
#include "ic.cuh"
#include "tree.cuh"
#include "newton.cuh"
#include "pricing.cuh"
#include "primitives.cuh"
#include "support.cuh"

#include <algorithm>
#include <atomic>
#include <mutex>
#include <thread>
#include <cmath>
#include <chrono>
#include <cstdarg>
#include <cstring>
#include <vector>

namespace ot {

std::atomic<int64_t> g_launches{0};

static thread_local std::string t_last_error;

// ---- kernel timing registry (pairs of events per kernel id, resolved when read)
namespace {
struct KTimer {
    std::atomic<bool> on{false};
    std::mutex mu;  // solves of a batch run on several host threads
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[KT_COUNT];
    std::vector<cudaEvent_t> open[KT_COUNT];
    double ms[KT_COUNT] = {0};
    int64_t count[KT_COUNT] = {0};
    double work[KT_COUNT] = {0};
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get() {
        cudaEvent_t e;
        if (!pool.empty()) { e = pool.back(); pool.pop_back(); return e; }
        cudaEventCreate(&e);
        return e;
    }
};
KTimer g_kt;
}  // namespace

void ktimer_begin(int id, cudaStream_t st) {
    if (!g_kt.on) return;
    std::lock_guard<std::mutex> lk(g_kt.mu);
    cudaEvent_t e = g_kt.get();
    cudaEventRecord(e, st);
    g_kt.open[id].push_back(e);
}

void ktimer_add_work(int id, double w) {
    if (!g_kt.on) return;
    std::lock_guard<std::mutex> lk(g_kt.mu);
    g_kt.work[id] += w;
}

void ktimer_end(int id, cudaStream_t st) {
    if (!g_kt.on) return;
    std::lock_guard<std::mutex> lk(g_kt.mu);
    if (g_kt.open[id].empty()) return;
    cudaEvent_t e = g_kt.get();
    cudaEventRecord(e, st);
    g_kt.pending[id].push_back({g_kt.open[id].back(), e});
    g_kt.open[id].pop_back();
}
void set_thread_error(const char *msg) { t_last_error = msg ? msg : ""; }

namespace {

constexpr double kBetaMin = 0.1, kBetaMax = 10.0, kAlphaBoost = 0.1, kAcceptGain = 1.01;
// Section 4.3: switch to LDL^T once psi fell by kSwitchDrop over the last 5 iterations; switch back
// (the remark after Section 4.3) when psi grows kSwitchBack above its minimum since the switch.
constexpr double kSwitchDrop = 0.1, kSwitchBack = 1.05;
// Section 4.2: a pivot that kept less than kPivotEps of its diagonal becomes +infinity.
constexpr double kPivotEps = 1e-12;
// a PCG result with relative residual above kPcgFail x tolerance counts as a failed solve
constexpr double kPcgFail = 10.0;
// preconditioned-CG iterations above which the next factorisation drops less
constexpr int kDirectCgMany = 25;
// incomplete Cholesky drop tolerance: divided by 10 after more than kIcManyCg CG iterations in one
// solve, never below kIcTauFloor
constexpr int kIcManyCg = 200;
constexpr double kIcTauFloor = 1e-6;
// up to this many targets the direct branch factors S_M densely
constexpr int kDenseMaxN = 8192;
constexpr int kDense32MaxN = 8192;
constexpr int kDense32LateMaxN = 16384;  // late iterations above kDenseMaxN: FP32 dense factor
constexpr int kDense32AbsMaxN = 65536;   // the FP32 dense factor's largest n (2 x 4 n^2 bytes: 34 GB)
constexpr int kBatchWorkers = 2;            // host threads of a batch (ot_ipm_solve_batch)
constexpr int kWarmCheck = 5;       // a warm start is judged from this iteration on ...
constexpr int kWarmSettle = 15;     // ... up to this one
constexpr double kWarmGrowth = 2.0; // abandoned when mu exceeds this multiple of its first value  // mixed precision: FP32 dense factor preconditions every solve

// c-transform lower bound (weak duality): ubar_i = min_j (c_ij - v_j); LB = a^T ubar + b^T v.
__global__ void ctrans_kernel(CostDev cd, const double *__restrict__ v, unsigned long long *__restrict__ rowmin) {
    const int m = cd.m, n = cd.n;
    constexpr int CH = 256;
    const int nch = (n + CH - 1) / CH;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; t < (int64_t)m * nch;
         t += (int64_t)gridDim.x * blockDim.y) {
        const int i = (int)(t / nch), c0 = (int)(t % nch) * CH;
        double best = INFINITY;
        for (int j = c0 + threadIdx.x; j < min(n, c0 + CH); j += blockDim.x)
            best = fmin(best, __dsub_rn(cost_at(cd, i, j), v[j]));
        best = warp_min(best);
        if (threadIdx.x == 0) atomicMin(&rowmin[i], f64_key(best));
    }
}

__global__ void lb_kernel(int m, int n, const unsigned long long *__restrict__ rowmin, const double *__restrict__ a,
                          const double *__restrict__ b, const double *__restrict__ v, double *out) {
    __shared__ double sh[32];
    double acc = 0;
    for (int64_t k = threadIdx.x; k < (int64_t)m + n; k += blockDim.x)
        acc += k < m ? a[k] * f64_from_key(rowmin[k]) : b[k - m] * v[k - m];
    double r = block_sum(acc, sh);
    if (threadIdx.x == 0) *out = r;
}

__global__ void count_below_kernel(const int32_t *__restrict__ cnt, const double *__restrict__ d, double thr,
                                   int *__restrict__ out) {
    int c = 0;
    for (int k = threadIdx.x; k < *cnt; k += blockDim.x) c += d[k] < thr ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    __shared__ int sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        *out = t;
    }
}

__global__ void check_dense_kernel(int64_t count, const double *__restrict__ C, int *__restrict__ bad) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x)
        if (!(C[k] >= 0.0) || !isfinite(C[k])) atomicExch(bad, 1);
}

__global__ void gather_dense_kernel(int m, int n, int n0, const int32_t *__restrict__ rmap,
                                    const int32_t *__restrict__ cmap, const double *__restrict__ C0,
                                    double *__restrict__ C) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < (int64_t)m * n; k += (int64_t)gridDim.x * blockDim.x)
        C[k] = C0[(int64_t)rmap[k / n] * n0 + cmap[k % n]];
}

__global__ void scatter_kernel(int count, const int32_t *__restrict__ map, const double *__restrict__ x,
                               double *__restrict__ y) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) y[map[k]] = x[k];
}

// Duals of the points the presolve removed (c-transforms, one block per removed point):
// u_i = min over kept targets j of c_ij - v_j; then v_j = min over all sources i of c_ij - u_i.
__global__ void complete_u_kernel(CostDev cf, const int32_t *__restrict__ rows, int n_kept,
                                  const int32_t *__restrict__ kept_cols, const double *__restrict__ v_kept,
                                  double *__restrict__ u_full) {
    __shared__ double sh[32];
    const int i = rows[blockIdx.x];
    double best = INFINITY;
    for (int r = threadIdx.x; r < n_kept; r += blockDim.x)
        best = fmin(best, __dsub_rn(cost_at(cf, i, kept_cols[r]), v_kept[r]));
    best = block_min(best, sh);
    if (threadIdx.x == 0) u_full[i] = best;
}

__global__ void complete_v_kernel(CostDev cf, const int32_t *__restrict__ cols, const double *__restrict__ u_full,
                                  double *__restrict__ v_full) {
    __shared__ double sh[32];
    const int j = cols[blockIdx.x];
    double best = INFINITY;
    for (int i = threadIdx.x; i < cf.m; i += blockDim.x) best = fmin(best, __dsub_rn(cost_at(cf, i, j), u_full[i]));
    best = block_min(best, sh);
    if (threadIdx.x == 0) v_full[j] = best;
}

// Multiscale warm start: the duals of the 2x2-binned problem at the fine points.  Cell (bx, by)
// holds the fine coordinates (o + 2b, o + 2b + 1), so a fine point sits at the continuous coarse
// coordinate (x - o - 0.5) / 2; the four surrounding cells are blended bilinearly over those that
// are occupied (the point's own cell is always among them and always occupied).
__global__ void upsample_kernel(int count, const int32_t *__restrict__ x, const int32_t *__restrict__ y, int ox,
                                int oy, int W, int H, const int32_t *__restrict__ lattice,
                                const double *__restrict__ uc, double scale, double *__restrict__ out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        const double xi = (x[k] - ox - 0.5) * 0.5, eta = (y[k] - oy - 0.5) * 0.5;
        const int bx = (int)floor(xi), by = (int)floor(eta);
        const double fx = xi - bx, fy = eta - by;
        double acc = 0.0, wsum = 0.0;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const int cx = bx + dx, cy = by + dy;
                if (cx < 0 || cy < 0 || cx >= W || cy >= H) continue;
                const int idx = lattice[(int64_t)cy * W + cx];
                if (idx < 0) continue;
                const double w = (dx ? fx : 1.0 - fx) * (dy ? fy : 1.0 - fy);
                acc += w * uc[idx];
                wsum += w;
            }
        out[k] = wsum > 0.0 ? scale * acc / wsum : 0.0;
    }
}

__global__ void scale_copy_kernel(int64_t count, const double *__restrict__ x, double f, double *__restrict__ y) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x)
        y[k] = x[k] * f;
}

}  // namespace
}  // namespace ot

using namespace ot;

struct ot_ipm {
    int32_t m = 0, n = 0;
    ot_options opt{};
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    double sigma_f = 1.0, fnorm = 0.0;
    // device problem
    double *a_s = nullptr, *b_s = nullptr, *C = nullptr;
    int32_t *sx = nullptr, *sy = nullptr, *tx = nullptr, *ty = nullptr;
    int32_t ox = 0, oy = 0;
    CostDev cd;
    double *u = nullptr, *v = nullptr;
    Support S[2];
    int cur = 0;
    Newton W;
    Chol chol;
    DenseLDL dense;
    Dense32 d32;
    std::vector<int64_t> psi_hist;
    bool direct_mode = false;
    bool d32_escalated = false;  // the FP32-preconditioned CG failed once: FP64 LDL^T from then on
    int64_t warm_added = 0;      // pairs the warm start added to the cold support
    bool warm_active = false;    // warm-started and still inside the check window
    int device = 0;              // CUDA device the handle lives on
    int32_t warm_restarts = 0;   // warm starts abandoned for the cold one
    int64_t psi_min = 0;
    double max_fill = 0.0;
    double drop = 1e-8;            // drop tolerance of the LDL^T preconditioner (adapted)
    int direct_cg_last = 0;
    int32_t *pi = nullptr, *pj = nullptr, *pcount = nullptr;
    double *pd = nullptr;
    int *pstrong = nullptr;
    unsigned long long *rowmin = nullptr;
    double *lbv = nullptr;
    // iteration state
    int iter = 0;
    double mu0 = -1.0;
    int strong = 1;
    bool done = false;
    int64_t cg_total = 0;
    int direct_total = 0;
    double last_lb = -INFINITY, last_gap = INFINITY, last_mu = 0.0;
    std::string err;
    // zero-mass presolve: the solve runs on the points with positive mass (m x n above)
    int32_t m0 = 0, n0 = 0;                   // the caller's sizes
    bool presolved = false;
    std::vector<int32_t> src_map, dst_map;    // solve index -> caller index
    std::vector<int32_t> src_inv, dst_inv;    // caller index -> solve index, -1 if removed
    int32_t *d_src_map = nullptr, *d_dst_map = nullptr;
    int32_t *fsx = nullptr, *fsy = nullptr, *ftx = nullptr, *fty = nullptr;  // caller's points
    double *fC = nullptr;                     // caller's dense costs (presolved dense problems)
    std::vector<double> warm_ur, warm_vr;     // warm-start inputs on the kept points
    std::vector<int32_t> warm_ir, warm_jr;
    JSet jset;                                // heuristic pricing set (Section 3.4), built on first use
    IncChol ic;                               // incomplete Cholesky preconditioner (precond 1)
    TreeSolver tree;                          // exact solver for forest supports
    int64_t tree_iters = 0;                   // iterations solved on a forest support
    double ic_tau = 1e-2;                     // its current drop tolerance
    int ic_cg_max = 0;                        // most CG iterations of one solve this iteration
    std::vector<double> as_host, bs_host;     // scaled masses (for the initial support's completion)
    std::vector<double> ms_u, ms_v;           // multiscale warm-start duals (host)
    int32_t ms_levels = 0;                    // coarse levels solved for the warm start
    double create_seconds = 0.0;
};

namespace {

Error support_alloc(Support &S, int64_t cap, int32_t m, int32_t n) {
    OT_CUDA(cudaMalloc((void **)&S.i, sizeof(int32_t) * cap));
    OT_CUDA(cudaMalloc((void **)&S.j, sizeof(int32_t) * cap));
    OT_CUDA(cudaMalloc((void **)&S.p, sizeof(double) * cap));
    OT_CUDA(cudaMalloc((void **)&S.s, sizeof(double) * cap));
    OT_CUDA(cudaMalloc((void **)&S.col_perm, sizeof(int32_t) * cap));
    OT_CUDA(cudaMalloc((void **)&S.col_row, sizeof(int32_t) * cap));
    if (!S.row_ptr) OT_CUDA(cudaMalloc((void **)&S.row_ptr, sizeof(int32_t) * ((int64_t)m + 1)));
    if (!S.col_ptr) OT_CUDA(cudaMalloc((void **)&S.col_ptr, sizeof(int32_t) * ((int64_t)n + 1)));
    S.cap = cap;
    return ok();
}

void support_free_arrays(Support &S) {
    for (void *p : {(void *)S.i, (void *)S.j, (void *)S.p, (void *)S.s, (void *)S.col_perm, (void *)S.col_row})
        if (p) cudaFree(p);
    S.i = S.j = S.col_perm = S.col_row = nullptr;
    S.p = S.s = nullptr;
}

void support_free(Support &S) {
    support_free_arrays(S);
    if (S.row_ptr) cudaFree(S.row_ptr);
    if (S.col_ptr) cudaFree(S.col_ptr);
    S = Support();
}

// grow both support buffers (and the work arrays) to hold `need` entries
Error ensure_capacity(ot_ipm *h, int64_t need) {
    if (need <= h->S[0].cap && need <= h->S[1].cap) return ok();
    const int64_t cap = std::max<int64_t>(need, (int64_t)(1.5 * std::max(h->S[0].cap, h->S[1].cap)));
    Support &A = h->S[h->cur];
    Support &B = h->S[1 - h->cur];
    // B is scratch: reallocate; A holds data: copy into a fresh allocation
    support_free_arrays(B);
    OT_TRY(support_alloc(B, cap, h->m, h->n));
    Support nA;
    nA.row_ptr = A.row_ptr;
    nA.col_ptr = A.col_ptr;
    OT_TRY(support_alloc(nA, cap, h->m, h->n));
    const int64_t psi = A.psi;
    OT_CUDA(cudaMemcpyAsync(nA.i, A.i, sizeof(int32_t) * psi, cudaMemcpyDeviceToDevice, h->st));
    OT_CUDA(cudaMemcpyAsync(nA.j, A.j, sizeof(int32_t) * psi, cudaMemcpyDeviceToDevice, h->st));
    OT_CUDA(cudaMemcpyAsync(nA.p, A.p, sizeof(double) * psi, cudaMemcpyDeviceToDevice, h->st));
    OT_CUDA(cudaMemcpyAsync(nA.s, A.s, sizeof(double) * psi, cudaMemcpyDeviceToDevice, h->st));
    OT_CUDA(cudaMemcpyAsync(nA.col_perm, A.col_perm, sizeof(int32_t) * psi, cudaMemcpyDeviceToDevice, h->st));
    OT_CUDA(cudaMemcpyAsync(nA.col_row, A.col_row, sizeof(int32_t) * psi, cudaMemcpyDeviceToDevice, h->st));
    OT_CUDA(cudaStreamSynchronize(h->st));
    support_free_arrays(A);
    nA.psi = psi;
    A = nA;
    OT_TRY(newton_grow(h->W, cap));
    return ok();
}

Error lower_bound(ot_ipm *h, double *lb) {
    OT_CUDA(cudaMemsetAsync(h->rowmin, 0xff, sizeof(unsigned long long) * h->m, h->st));
    dim3 blk(32, 8);
    const int64_t work = (int64_t)h->m * ceil_div(h->n, 256);
    ctrans_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, 8), 16LL * h->num_sms)), blk, 0,
                    h->st>>>(h->cd, h->v, h->rowmin);
    OT_LAUNCHED();
    lb_kernel<<<1, 1024, 0, h->st>>>(h->m, h->n, h->rowmin, h->a_s, h->b_s, h->v, h->lbv);
    OT_LAUNCHED();
    OT_CUDA(cudaMemcpyAsync(lb, h->lbv, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    OT_CUDA(cudaStreamSynchronize(h->st));
    return ok();
}

// A forest support (psi == m + n - #components: Theorem 2's structure near optimality) is solved
// exactly on the tree; *is_forest tells whether this iteration's support is one.
Error forest_setup(ot_ipm *h, const Support &S, bool *is_forest, cudaStream_t st) {
    *is_forest = false;
    if (S.psi > (int64_t)h->m + h->n - 1) return ok();
    int64_t ncomp = 0;
    OT_TRY(support_components(h->W, &ncomp, st));
    if (S.psi != (int64_t)h->m + h->n - ncomp) return ok();
    if (!h->tree.order) OT_TRY(tree_alloc(h->tree, h->m, h->n, std::max<int64_t>(S.psi, (int64_t)h->m + h->n)));
    OT_TRY(tree_build(h->tree, S, h->W.parent, st));
    *is_forest = true;
    return ok();
}

Error price_support(ot_ipm *h, const Support &S, int32_t kmax, int32_t *count, PriceStats *ps, bool use_j) {
    PriceInput in;
    in.kind = h->cd.kind;
    in.C = h->C;
    if (use_j) {
        if (!h->jset.i)
            OT_TRY(jset_build(h->cd.kind, h->m, h->n, h->sx, h->sy, h->tx, h->ty, h->C, h->opt.jset_cmax, &h->jset,
                              h->st));
        in.ji = h->jset.i;
        in.jj = h->jset.j;
        in.jn = h->jset.n;
        in.jlim = h->jset.lim;
        in.jcmax = h->jset.cmax;
    }
    in.m = h->m; in.n = h->n;
    in.sx = h->sx; in.sy = h->sy; in.tx = h->tx; in.ty = h->ty;
    in.u = h->u; in.v = h->v;
    in.sup_i = S.i; in.sup_j = S.j; in.row_ptr = S.row_ptr; in.psi = S.psi;
    in.kmax = kmax;
    in.precision = h->opt.precision;
    in.origin_x = h->ox; in.origin_y = h->oy;
    in.num_sms = h->num_sms;
    in.rows = h->opt.scan_rows;
    OT_TRY(price_topk(in, h->pi, h->pj, h->pd, h->pcount, ps, h->st));
    OT_CUDA(cudaMemcpyAsync(count, h->pcount, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st));
    OT_CUDA(cudaStreamSynchronize(h->st));
    return ok();
}

double step_of(double ratio, double scale) { return std::min(1.0, scale * ratio); }

// wall-clock phase breakdown of one iteration (verbose >= 2): synchronises at each mark
struct PhaseClock {
    bool on;
    cudaStream_t st;
    std::chrono::steady_clock::time_point t;
    std::string line;
    PhaseClock(bool on_, cudaStream_t s) : on(on_), st(s) {
        if (on) { cudaStreamSynchronize(st); t = std::chrono::steady_clock::now(); }
    }
    void mark(const char *name) {
        if (!on) return;
        cudaStreamSynchronize(st);
        auto now = std::chrono::steady_clock::now();
        char buf[64];
        snprintf(buf, sizeof(buf), " %s %.2f", name, std::chrono::duration<double, std::milli>(now - t).count());
        line += buf;
        t = now;
    }
};

// Stopping measure of the current point (the quantity the first iteration's test reads).
Error start_crit(ot_ipm *h, double *crit) {
    Newton &W = h->W;
    Support &S = h->S[h->cur];
    double hs[SC_COUNT];
    OT_TRY(residuals(W, S, h->a_s, h->b_s, h->u, h->v, h->st));
    OT_TRY(read_scalars(W, hs, h->st));
    const double psi = (double)S.psi, mu = hs[SC_PS] / psi;
    const double r1n = std::sqrt(hs[SC_R1A_SQ] + hs[SC_R1B_SQ]);
    *crit = std::max({r1n / (1.0 + h->fnorm), std::sqrt(hs[SC_R2SQ]) / (1.0 + std::sqrt(hs[SC_CSQ])),
                      psi * mu / (1.0 + std::fabs(hs[SC_CP]))});
    if (!std::isfinite(*crit)) *crit = INFINITY;
    return ok();
}

Error cold_support(ot_ipm *h, cudaStream_t st);

// Abandon a warm start: the cold initial support and Mehrotra's point, as ot_ipm_create builds
// them; the iteration count carries on.
Error cold_restart(ot_ipm *h) {
    const ot_options &o = h->opt;
    cudaStream_t st = h->st;
    OT_TRY(cold_support(h, st));
    Support &S = h->S[h->cur];
    OT_TRY(support_costs(h->W, h->cd, S, st));
    int cgs = 0;
    OT_TRY(mehrotra_start(h->W, S, h->a_s, h->b_s, h->u, h->v, o.precision, o.cg_tol_pred, 20 * o.max_cg, &cgs, st));
    h->cg_total += cgs;
    h->mu0 = -1.0;
    h->psi_hist.clear();
    h->direct_mode = false;
    h->strong = 0;
    h->warm_active = false;
    h->warm_restarts++;
    h->warm_added = 0;
    return ok();
}

Error do_step(ot_ipm *h, ot_iter_info *info) {
    const ot_options &o = h->opt;
    cudaStream_t st = h->st;
    Newton &W = h->W;
    Support &S = h->S[h->cur];
    const int32_t m = h->m, n = h->n;
    ot_iter_info inf{};
    inf.iter = h->iter;
    inf.psi = S.psi;
    double hs[SC_COUNT];

    PhaseClock pc(o.verbose >= 2, st);
    OT_TRY(residuals(W, S, h->a_s, h->b_s, h->u, h->v, st));
    OT_TRY(read_scalars(W, hs, st));
    pc.mark("res");
    const double psi = (double)S.psi;
    const double mu = hs[SC_PS] / psi;
    const double ctp = hs[SC_CP];
    const double r1n = std::sqrt(hs[SC_R1A_SQ] + hs[SC_R1B_SQ]);
    const double crit = std::max({r1n / (1.0 + h->fnorm), std::sqrt(hs[SC_R2SQ]) / (1.0 + std::sqrt(hs[SC_CSQ])),
                                  psi * mu / (1.0 + std::fabs(ctp))});
    const double r1_l1 = (hs[SC_R1A_L1] + hs[SC_R1B_L1]) / h->sigma_f;
    const double cmax_red = hs[SC_CMAX];
    if (!std::isfinite(mu) || !std::isfinite(crit)) return fail(OT_ERR_NUMERIC, "non-finite mu or residual");
    if (h->mu0 < 0) h->mu0 = mu;
    if (h->warm_active && h->iter >= kWarmCheck) {
        if (mu > kWarmGrowth * h->mu0) {
            OT_TRY(cold_restart(h));
            return do_step(h, info);
        }
        if (h->iter >= kWarmSettle) h->warm_active = false;
    }
    h->last_mu = mu;
    inf.mu = mu;
    inf.crit = crit;
    if (crit < o.tol && r1_l1 <= o.feas_l1 && h->strong == 0) {
        double lb;
        OT_TRY(lower_bound(h, &lb));
        const double gap = (ctp - lb) / (1.0 + std::fabs(ctp));
        h->last_lb = lb;
        h->last_gap = gap;
        if (gap <= o.tol) {
            h->done = true;
            inf.done = 1;
            if (info) *info = inf;
            return ok();
        }
    }
    if (h->iter >= o.max_iter) {
        if (info) *info = inf;
        return fail(OT_ERR_MAXITER, "iteration limit reached");
    }

    // ---- Newton direction: Mehrotra predictor-corrector + centrality correctors
    OT_TRY(schur_setup(W, S, st));
    pc.mark("schur");
    // iterative (PCG) or direct (LDL^T) solves of S_M, Section 4.3
    h->psi_hist.push_back(S.psi);
    bool use_direct = o.linear_solver == 2;
    if (o.linear_solver == 0) {
        const size_t L = h->psi_hist.size();
        if (!h->direct_mode && L >= 6) {
            const double p5 = (double)h->psi_hist[L - 6], p0 = (double)h->psi_hist[L - 1];
            if ((p5 - p0) / p5 >= kSwitchDrop) { h->direct_mode = true; h->psi_min = S.psi; }
        }
        if (h->direct_mode) {
            h->psi_min = std::min(h->psi_min, S.psi);
            if ((double)S.psi > kSwitchBack * (double)h->psi_min) h->direct_mode = false;
        }
        use_direct = h->direct_mode;
    }
    W.direct = nullptr;
    W.dense = nullptr;
    W.d32 = nullptr;
    W.ic = nullptr;
    W.tree = nullptr;
    // Section 4.3 / Theorem 2: a forest support needs no factorisation at all
    bool forest = false;
    if (o.linear_solver != 1) OT_TRY(forest_setup(h, S, &forest, st));
    if (forest) {
        W.tree = &h->tree;
        h->tree_iters++;
        inf.direct = 1;
    }
    // mixed precision on moderate n: the FP32 dense factorisation of this iteration's S_M
    // preconditions an FP64 CG in every solve; the FP64 LDL^T branch only takes over when that CG
    // misses its target (the switch on the support's shrinkage is for the Jacobi PCG)
    // every iteration up to kDense32MaxN by default; a caller may raise the limit to kDense32AbsMaxN
    const int64_t d32_max = o.dense32_max_n > 0 ? std::min<int64_t>(o.dense32_max_n, kDense32AbsMaxN)
                                                : (o.dense32_max_n < 0 ? 0 : kDense32MaxN);
    const bool use_d32 = o.precision == 1 && o.linear_solver == 0 && o.precond != 1 && n <= d32_max;
    if (forest) {
        use_direct = false;
    } else if (use_d32 && !h->d32_escalated) {
        use_direct = false;
        if (!h->d32.A) { OT_TRY(d32_alloc(h->d32, n)); h->d32.tc_mode = h->opt.tc_update; }
        OT_TRY(d32_assemble(h->d32, W, S, st));
        OT_TRY(d32_factor(h->d32, (float)kPivotEps, st));
        W.d32 = &h->d32;
    } else if (use_d32) {
        use_direct = true;
    }
    const int direct_cg_prev = h->direct_cg_last;
    h->direct_cg_last = 0;
    // factor S_M once for every solve of this iteration; false when the fill is over budget
    const int64_t dense_max = o.dense_max_n > 0 ? std::min<int64_t>(o.dense_max_n, kDenseMaxN)
                                                : (o.dense_max_n < 0 ? 0 : kDenseMaxN);
    auto enable_direct = [&]() -> Error {
        if (n > kDenseMaxN && n <= kDense32LateMaxN && o.dense_max_n >= 0) {
            // beyond the FP64 dense size, the late iterations precondition the FP64 CG with the
            // FP32 dense factorisation (pivots from off-diagonal sums, exact grounding)
            if (!h->d32.A) { OT_TRY(d32_alloc(h->d32, n)); h->d32.tc_mode = h->opt.tc_update; }
            OT_TRY(d32_assemble(h->d32, W, S, st));
            OT_TRY(d32_factor(h->d32, (float)kPivotEps, st));
            W.d32 = &h->d32;
            h->max_fill = 100.0;
            h->direct_total++;
            inf.direct = 1;
            return ok();
        }
        if (n <= dense_max) {
            // moderate n: exact assembly and a dense blocked LDL^T (the exact factor is dense-ish)
            if (!h->dense.A) OT_TRY(dense_alloc(h->dense, n));
            bool changed = false;
            OT_TRY(chol_assemble(h->chol, W, S, 0.0, &changed, st));
            OT_CUDA(cudaMemsetAsync(h->dense.err, 0, sizeof(int), st));
            OT_TRY(dense_factor(h->dense, h->chol, kPivotEps, st));
            W.direct = &h->chol;
            W.dense = &h->dense;
            h->max_fill = 100.0;
            h->direct_total++;
            inf.direct = 1;
            return ok();
        }
        // Section 4.2: the drop tolerance is lowered when the preconditioned CG needed too many
        // iterations, and raised here while the factor's fill is over budget
        if (direct_cg_prev > kDirectCgMany) h->drop = std::max(h->drop * 1e-2, 0.0);
        if (h->drop < 1e-14) h->drop = 0.0;
        Error e = ok();
        for (int attempt = 0; attempt < 4; ++attempt) {
            bool changed = false;
            OT_TRY(chol_assemble(h->chol, W, S, h->drop, &changed, st));
            e = ok();
            if (changed || !h->chol.have_symbolic) e = chol_symbolic(h->chol, st);
            if (e.code != OT_ERR_UNSUPPORTED) break;
            h->drop = h->drop > 0 ? std::min(h->drop * 1e2, 1e-2) : 1e-10;
        }
        if (e.code == OT_OK) {
            OT_TRY(chol_numeric(h->chol, kPivotEps, st));
            W.direct = &h->chol;
            h->max_fill = std::max(h->max_fill, h->chol.fill_pct);
            h->direct_total++;
            inf.direct = 1;
            return ok();
        }
        return e.code == OT_ERR_UNSUPPORTED ? ok() : e;
    };
    if (use_direct) OT_TRY(enable_direct());
    // Section 4.2: the iterative phase preconditioned by the incomplete Cholesky factor
    h->ic_cg_max = 0;
    if (o.precond == 1 && !W.direct && !W.d32 && !W.tree) {
        if (!h->ic.perm) OT_TRY(ic_alloc(h->ic, n));
        bool changed = false;
        OT_TRY(chol_assemble(h->chol, W, S, 0.0, &changed, st));
        OT_TRY(ic_factor(h->ic, h->chol, h->ic_tau, kPivotEps, st));
        W.ic = &h->ic;
    }
    pc.mark("factor");
    int cg = 0;
    SolveStats ss;
    // a PCG solve that misses its tolerance by more than kPcgFail switches this iteration (and,
    // through direct_mode, the following ones) to the LDL^T branch when its fill is acceptable
    auto solve = [&](const Rhs &R, double tol, double *du, double *dv, double *ds, double *dp) -> Error {
        W.fp64_fallback = o.linear_solver != 0;  // in auto mode a failed solve escalates to LDL^T
        OT_TRY(newton_solve(W, S, R, tol, o.max_cg, o.precision, du, dv, ds, dp, &ss, st));
        cg += ss.cg_iters;
        if (ss.direct) h->direct_cg_last = std::max(h->direct_cg_last, ss.cg_iters);
        if (W.ic && !W.direct) h->ic_cg_max = std::max(h->ic_cg_max, ss.cg_iters);
        const bool late_d32 = W.d32 && n > kDenseMaxN;   // already the strongest solver here
        if (!W.direct && !W.tree && !late_d32 && o.linear_solver == 0 && !(ss.relres <= kPcgFail * tol)) {
            OT_TRY(enable_direct());
            if (W.direct || (W.d32 && n > kDenseMaxN)) {
                h->direct_mode = true;
                h->psi_min = S.psi;
                if (W.d32) h->d32_escalated = true;
                OT_TRY(newton_solve(W, S, R, tol, o.max_cg, o.precision, du, dv, ds, dp, &ss, st));
            } else if (o.precision == 1) {  // fill over budget: FP64 PCG as the last resort
                OT_TRY(newton_solve(W, S, R, tol, o.max_cg, 0, du, dv, ds, dp, &ss, st));
                cg += ss.cg_iters;
            }
        }
        return ok();
    };
    OT_TRY(corrector_r3(W, S, 0.0, nullptr, nullptr, st));  // r3 = -p s
    Rhs R{W.r1a, W.r1b, W.r2, W.r3};
    OT_TRY(solve(R, o.cg_tol_pred, W.du, W.dv, W.ds, W.dp));
    OT_TRY(step_lengths(W, S, W.dp, W.ds, o.step_scale, st));
    OT_TRY(read_scalars(W, hs, st));
    const double apa = step_of(hs[SC_AP], o.step_scale), asa = step_of(hs[SC_AS], o.step_scale);
    OT_TRY(trial_complementarity(W, S, W.dp, W.ds, apa, asa, st));
    OT_TRY(read_scalars(W, hs, st));
    const double mu_aff = hs[SC_MUAFF] / psi;
    const double sigma = std::min(1.0, std::max(0.0, std::pow(mu_aff / mu, 3.0)));
    OT_TRY(corrector_r3(W, S, sigma * mu, W.dp, W.ds, st));
    double *d_du = W.du2, *d_dv = W.dv2, *d_ds = W.ds2, *d_dp = W.dp2;  // current direction
    double *c_du = W.du3, *c_dv = W.dv3, *c_ds = W.ds3, *c_dp = W.dp3;  // corrector scratch
    OT_TRY(solve(R, o.cg_tol_pred, d_du, d_dv, d_ds, d_dp));
    OT_TRY(step_lengths(W, S, d_dp, d_ds, o.step_scale, st));
    OT_TRY(read_scalars(W, hs, st));
    double ap = step_of(hs[SC_AP], o.step_scale), as = step_of(hs[SC_AS], o.step_scale);
    int ncorr = 0;
    for (int k = 0; k < o.max_corr; ++k) {
        if (std::min(ap, as) >= 1.0) break;
        const double tp = std::min(1.0, ap + kAlphaBoost), ts = std::min(1.0, as + kAlphaBoost);
        OT_TRY(centrality_r3(W, S, d_dp, d_ds, tp, ts, kBetaMin * sigma * mu, kBetaMax * sigma * mu, st));
        Rhs Rc{nullptr, nullptr, nullptr, W.r3};
        OT_TRY(solve(Rc, o.cg_tol_corr, c_du, c_dv, c_ds, c_dp));
        OT_TRY(add_direction(W, S, c_dp, c_ds, c_du, c_dv, d_dp, d_ds, d_du, d_dv, st));
        OT_TRY(step_lengths(W, S, c_dp, c_ds, o.step_scale, st));
        OT_TRY(read_scalars(W, hs, st));
        const double ap2 = step_of(hs[SC_AP], o.step_scale), as2 = step_of(hs[SC_AS], o.step_scale);
        if (std::min(ap2, as2) >= kAcceptGain * std::min(ap, as)) {
            std::swap(d_du, c_du); std::swap(d_dv, c_dv); std::swap(d_ds, c_ds); std::swap(d_dp, c_dp);
            ap = ap2;
            as = as2;
            ++ncorr;
        } else {
            break;
        }
    }
    pc.mark("newton");
    OT_TRY(take_step(W, S, h->u, h->v, d_dp, d_ds, d_du, d_dv, ap, as, st));
    OT_TRY(read_scalars(W, hs, st));
    const double mu_new = hs[SC_PSNEW] / psi;
    if (!std::isfinite(mu_new) || !(mu_new > 0)) return fail(OT_ERR_NUMERIC, "non-finite or non-positive mu");

    // ---- pricing (Section 3.4) and support update (Section 3.2)
    const int32_t kadd = o.add_max > 0 ? o.add_max : m;
    int32_t added = 0;
    PriceStats ps;
    pc.mark("step");
    // Section 3.4: the heuristic set J between full refreshes (every jset_refresh-th iteration)
    const int refresh = o.jset_refresh > 0 ? o.jset_refresh : 3;
    const bool use_j = o.jset_cmax > 0 && (h->iter % refresh) != refresh - 1;
    OT_TRY(price_support(h, S, kadd, &added, &ps, use_j));
    pc.mark("price");
    {
        count_below_kernel<<<1, 256, 0, st>>>(h->pcount, h->pd, -o.tol * (1.0 + cmax_red), h->pstrong);
        OT_LAUNCHED();
        OT_CUDA(cudaMemcpyAsync(&h->strong, h->pstrong, sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    // grow first: growing reallocates the work arrays, the removal flags included
    OT_TRY(ensure_capacity(h, S.psi + added));
    int64_t removed = 0;
    const bool removing = mu_new <= o.rm_mu_frac * h->mu0;
    if (removing) OT_TRY(removal_flags(S, m, n, h->a_s, h->b_s, o.rm_p_frac, m, W.flag, &removed, st));
    Support &S0 = h->S[h->cur];
    Support &T = h->S[1 - h->cur];
    pc.mark("remove");
    OT_TRY(merge_support(S0, removing ? W.flag : nullptr, h->pi, h->pj, added, std::sqrt(mu_new), m, n, T, st,
                         o.new_col_rule == 1 ? h->a_s : nullptr, o.new_col_rule == 1 ? h->b_s : nullptr));
    h->cur = 1 - h->cur;
    OT_TRY(support_costs(W, h->cd, T, st));
    OT_CUDA(cudaStreamSynchronize(st));
    pc.mark("merge");

    // the drop tolerance schedule of the incomplete factor (reading of Section 4.2)
    if (h->ic_cg_max > kIcManyCg) h->ic_tau = std::max(h->ic_tau * 0.1, kIcTauFloor);
    h->iter++;
    h->cg_total += cg;
    inf.alpha_p = ap;
    inf.alpha_s = as;
    inf.sigma = sigma;
    inf.ncorr = ncorr;
    inf.cg_iters = cg;
    inf.added = added;
    inf.removed = removed;
    if (o.verbose >= 2) fprintf(stderr, "   phases(ms):%s\n", pc.line.c_str());
    if (o.verbose >= 2 && W.ic)
        fprintf(stderr, "   incomplete Cholesky: %d colours, %lld entries, drop tolerance %.1e, most CG %d\n",
                h->ic.ncolors, (long long)h->ic.nnzL, h->ic.tau, h->ic_cg_max);
    if (o.verbose)
        fprintf(stderr, "it %3d psi %8lld mu %.3e crit %.3e ap %.3f as %.3f sig %.2e corr %d cg %d %s +%d -%lld\n",
                inf.iter, (long long)inf.psi, mu, crit, ap, as, sigma, ncorr, cg, inf.direct ? "LDL" : "PCG", added,
                (long long)removed);
    if (info) *info = inf;
    return ok();
}

int record(ot_ipm *h, const Error &e) {
    if (e.code != OT_OK) h->err = e.msg;
    return e.code;
}

// Explicit pairs join the support: validated, deduplicated and stripped of the pairs already in
// it on the host, then merged (at most what the support buffers hold).  *added (may be NULL)
// receives the number merged.
Error add_pairs(ot_ipm *h, const int32_t *pi, const int32_t *pj, int64_t count, cudaStream_t st, int64_t *added) {
    const int m = h->m, n = h->n;
    if (added) *added = 0;
    Support &A = h->S[h->cur];
    Support &B = h->S[1 - h->cur];
    std::vector<int32_t> si(A.psi), sj(A.psi);
    OT_CUDA(cudaMemcpyAsync(si.data(), A.i, sizeof(int32_t) * A.psi, cudaMemcpyDeviceToHost, st));
    OT_CUDA(cudaMemcpyAsync(sj.data(), A.j, sizeof(int32_t) * A.psi, cudaMemcpyDeviceToHost, st));
    OT_CUDA(cudaStreamSynchronize(st));
    std::vector<int64_t> have(A.psi);
    for (int64_t e = 0; e < A.psi; ++e) have[e] = (int64_t)si[e] * n + sj[e];  // sorted by (i, j)
    std::vector<int64_t> add;
    add.reserve(count);
    for (int64_t t = 0; t < count; ++t) {
        const int32_t i = pi[t], j = pj[t];
        if (i < 0 || i >= m || j < 0 || j >= n) return fail(OT_ERR_ARG, "warm pairs: index out of range");
        add.push_back((int64_t)i * n + j);
    }
    std::sort(add.begin(), add.end());
    add.erase(std::unique(add.begin(), add.end()), add.end());
    std::vector<int32_t> ni, nj;
    const int64_t room = std::min(A.cap, B.cap) - A.psi;
    for (int64_t key : add) {
        if ((int64_t)ni.size() >= room) break;
        if (std::binary_search(have.begin(), have.end(), key)) continue;
        ni.push_back((int32_t)(key / n));
        nj.push_back((int32_t)(key % n));
    }
    const int64_t k = (int64_t)ni.size();
    if (k == 0) return ok();
    DevTemp<int32_t> di, dj;
    DevTemp<uint8_t> keep;
    OT_TRY(di.alloc(k, st)); OT_TRY(dj.alloc(k, st));
    OT_TRY(keep.alloc(std::max<int64_t>(A.psi, 1), st));
    OT_CUDA(cudaMemcpyAsync(di.p, ni.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, st));
    OT_CUDA(cudaMemcpyAsync(dj.p, nj.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, st));
    OT_CUDA(cudaMemsetAsync(keep.p, 0, std::max<int64_t>(A.psi, 1), st));
    OT_TRY(merge_support(A, keep.p, di.p, dj.p, k, 1.0, m, n, B, st));
    h->cur = 1 - h->cur;
    if (added) *added = k;
    return ok();
}

Error warm_pairs(ot_ipm *h, const ot_options &o, cudaStream_t st) {
    int64_t k = 0;
    OT_TRY(add_pairs(h, o.warm_i, o.warm_j, o.warm_npairs, st, &k));
    h->warm_added += k;
    return ok();
}

// Pairs of the north-west-corner coupling of the scaled masses, sources and targets in index order
// (a feasible transportation plan: a staircase of at most m + n - 1 pairs; equal partial sums
// advance both sides).
void nw_corner_pairs(const std::vector<double> &a, const std::vector<double> &b, std::vector<int32_t> &I,
                     std::vector<int32_t> &J) {
    const size_t m = a.size(), n = b.size();
    double A = 0.0, B = 0.0;
    size_t i = 0, j = 0;
    if (m && n) { A = a[0]; B = b[0]; }
    while (i < m && j < n) {
        I.push_back((int32_t)i);
        J.push_back((int32_t)j);
        if (A < B) { if (++i < m) A += a[i]; }
        else if (B < A) { if (++j < n) B += b[j]; }
        else {
            if (++i < m) A += a[i];
            if (++j < n) B += b[j];
        }
    }
}

// Initial support (Section 3.2 end), in S[cur]: {c_ij <= init_cost} plus every row's and column's
// cheapest pair; when that support graph splits into several components (point sets that do not
// overlap, where the restricted problem would be infeasible), the north-west-corner coupling's
// pairs join it, which makes the restricted problem feasible.
Error complete_feasible(ot_ipm *h, cudaStream_t st) {
    bool one = true;
    OT_TRY(support_connected(h->W, h->S[h->cur], &one, st));
    if (one) return ok();
    std::vector<int32_t> I, J;
    nw_corner_pairs(h->as_host, h->bs_host, I, J);
    OT_TRY(ensure_capacity(h, h->S[h->cur].psi + (int64_t)I.size()));
    return add_pairs(h, I.data(), J.data(), (int64_t)I.size(), st, nullptr);
}

Error cold_support(ot_ipm *h, cudaStream_t st) {
    int32_t *ii = nullptr, *jj = nullptr;
    int64_t psi0 = 0;
    OT_TRY(initial_support(h->cd, h->opt.init_cost, &ii, &jj, &psi0, st));
    Error e = ensure_capacity(h, psi0);
    Support &S = h->S[h->cur];
    if (e.code == OT_OK) {
        cudaMemcpyAsync(S.i, ii, sizeof(int32_t) * psi0, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(S.j, jj, sizeof(int32_t) * psi0, cudaMemcpyDeviceToDevice, st);
        cudaStreamSynchronize(st);
    }
    cudaFree(ii);
    cudaFree(jj);
    OT_TRY(e);
    S.psi = psi0;
    OT_TRY(rebuild_views(S, h->m, h->n, st));
    return complete_feasible(h, st);
}

// Warm start: the pricing scan with the predicted duals shifted by init_cost selects the pairs of
// least predicted reduced cost c_ij - u_i - v_j < init_cost outside the cold support, and they
// join it (the cold rule is the same test with u = v = 0).
Error warm_support(ot_ipm *h, const ot_options &o, cudaStream_t st) {
    const int m = h->m, n = h->n;
    Support &A = h->S[h->cur];
    Support &B = h->S[1 - h->cur];
    // at most what the support buffers hold beyond the cold support (the workspace is sized after)
    const int64_t want = o.warm_count > 0 ? o.warm_count : 2LL * (m + n);
    const int32_t K = (int32_t)std::min<int64_t>(want, std::min(A.cap, B.cap) - A.psi);
    if (K <= 0) return ok();
    std::vector<double> hu(o.warm_u, o.warm_u + m), hv(o.warm_v, o.warm_v + n);
    for (int i = 0; i < m; ++i) {
        if (!std::isfinite(hu[i])) return fail(OT_ERR_ARG, "warm_u: non-finite value");
        hu[i] += o.init_cost;
    }
    for (int j = 0; j < n; ++j)
        if (!std::isfinite(hv[j])) return fail(OT_ERR_ARG, "warm_v: non-finite value");
    DevTemp<double> du, dv, dd;
    DevTemp<int32_t> wi, wj, wc;
    DevTemp<uint8_t> keep;
    OT_TRY(du.alloc(m, st)); OT_TRY(dv.alloc(n, st)); OT_TRY(dd.alloc(K, st));
    OT_TRY(wi.alloc(K, st)); OT_TRY(wj.alloc(K, st)); OT_TRY(wc.alloc(1, st));
    OT_TRY(keep.alloc(std::max<int64_t>(A.psi, 1), st));
    OT_CUDA(cudaMemcpyAsync(du.p, hu.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st));
    OT_CUDA(cudaMemcpyAsync(dv.p, hv.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
    OT_CUDA(cudaMemsetAsync(keep.p, 0, std::max<int64_t>(A.psi, 1), st));
    PriceInput in;
    in.m = m;
    in.n = n;
    in.sx = h->sx; in.sy = h->sy; in.tx = h->tx; in.ty = h->ty;
    in.u = du.p;
    in.v = dv.p;
    in.sup_i = A.i;
    in.sup_j = A.j;
    in.row_ptr = A.row_ptr;
    in.psi = A.psi;
    in.kmax = K;
    in.precision = o.precision;
    in.kind = h->cd.kind;
    in.C = h->C;
    in.origin_x = h->ox;
    in.origin_y = h->oy;
    in.num_sms = h->num_sms;
    OT_TRY(price_topk(in, wi.p, wj.p, dd.p, wc.p, nullptr, st));
    int32_t k = 0;
    OT_CUDA(cudaMemcpyAsync(&k, wc.p, sizeof(k), cudaMemcpyDeviceToHost, st));
    OT_CUDA(cudaStreamSynchronize(st));
    if (k <= 0) return ok();
    OT_TRY(merge_support(A, keep.p, wi.p, wj.p, k, 1.0, m, n, B, st));
    h->cur = 1 - h->cur;
    h->warm_added += k;
    return ok();
}

// Duals in the caller's indexing (host buffers, either may be NULL).  Points removed by the
// presolve get c-transform duals when `complete`, else 0.
Error caller_duals(ot_ipm *h, double *u_out, double *v_out, bool complete) {
    cudaStream_t st = h->st;
    if (!h->presolved) {
        if (u_out) OT_CUDA(cudaMemcpyAsync(u_out, h->u, sizeof(double) * h->m, cudaMemcpyDeviceToHost, st));
        if (v_out) OT_CUDA(cudaMemcpyAsync(v_out, h->v, sizeof(double) * h->n, cudaMemcpyDeviceToHost, st));
        OT_CUDA(cudaStreamSynchronize(st));
        return ok();
    }
    if (!u_out && !v_out) return ok();
    const int m0 = h->m0, n0 = h->n0;
    DevTemp<double> uf, vf;
    OT_TRY(uf.alloc(m0, st));
    OT_TRY(vf.alloc(n0, st));
    OT_CUDA(cudaMemsetAsync(uf.p, 0, sizeof(double) * m0, st));
    OT_CUDA(cudaMemsetAsync(vf.p, 0, sizeof(double) * n0, st));
    scatter_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(h->m, 256), 1024)), 256, 0, st>>>(
        h->m, h->d_src_map, h->u, uf.p);
    OT_LAUNCHED();
    scatter_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(h->n, 256), 1024)), 256, 0, st>>>(
        h->n, h->d_dst_map, h->v, vf.p);
    OT_LAUNCHED();
    if (complete) {
        std::vector<int32_t> ri, rj;
        for (int i = 0; i < m0; ++i) if (h->src_inv[i] < 0) ri.push_back(i);
        for (int j = 0; j < n0; ++j) if (h->dst_inv[j] < 0) rj.push_back(j);
        CostDev cf = h->cd;
        cf.m = m0;
        cf.n = n0;
        if (cf.kind == OT_COST_DENSE) cf.C = h->fC;
        else { cf.sx = h->fsx; cf.sy = h->fsy; cf.tx = h->ftx; cf.ty = h->fty; }
        DevTemp<int32_t> dri, drj;
        OT_TRY(dri.alloc((int64_t)ri.size(), st));
        OT_TRY(drj.alloc((int64_t)rj.size(), st));
        if (!ri.empty()) {
            OT_CUDA(cudaMemcpyAsync(dri.p, ri.data(), sizeof(int32_t) * ri.size(), cudaMemcpyHostToDevice, st));
            complete_u_kernel<<<(unsigned)ri.size(), 256, 0, st>>>(cf, dri.p, h->n, h->d_dst_map, h->v, uf.p);
            OT_LAUNCHED();
        }
        if (!rj.empty()) {
            OT_CUDA(cudaMemcpyAsync(drj.p, rj.data(), sizeof(int32_t) * rj.size(), cudaMemcpyHostToDevice, st));
            complete_v_kernel<<<(unsigned)rj.size(), 256, 0, st>>>(cf, drj.p, uf.p, vf.p);
            OT_LAUNCHED();
        }
        OT_CUDA(cudaStreamSynchronize(st));  // the host index lists above must outlive the copies
    }
    if (u_out) OT_CUDA(cudaMemcpyAsync(u_out, uf.p, sizeof(double) * m0, cudaMemcpyDeviceToHost, st));
    if (v_out) OT_CUDA(cudaMemcpyAsync(v_out, vf.p, sizeof(double) * n0, cudaMemcpyDeviceToHost, st));
    OT_CUDA(cudaStreamSynchronize(st));
    return ok();
}

// Support indices to the caller's indexing (host arrays, in place).
void caller_pairs(const ot_ipm *h, int32_t *i, int32_t *j, int64_t k) {
    if (!h->presolved) return;
    for (int64_t e = 0; e < k; ++e) {
        if (i) i[e] = h->src_map[i[e]];
        if (j) j[e] = h->dst_map[j[e]];
    }
}

Error create_impl(const ot_problem *P, const ot_options *O, ot_ipm *h);
Error do_step(ot_ipm *h, ot_iter_info *info);

constexpr int kMsMinPoints = 256;             // no coarser level below this many points per side
constexpr int64_t kMsMaxCells = 1LL << 26;    // bound of the coarse lattice

// Multiscale warm start (see ot_options.multiscale): solve the 2x2-binned problem (recursively
// coarser itself), interpolate its duals at the points, and hand them to the warm start.  A coarse
// solve that fails leaves the cold start.
Error multiscale_start(ot_ipm *h, const std::vector<double> &as, const std::vector<double> &bs,
                       const std::vector<int32_t> &hx, const std::vector<int32_t> &hy,
                       const std::vector<int32_t> &gx, const std::vector<int32_t> &gy, cudaStream_t st) {
    ot_options &o = h->opt;
    const int m = h->m, n = h->n;
    if (o.multiscale <= 0 || h->cd.kind == OT_COST_DENSE || (o.warm_u && o.warm_v) || m < kMsMinPoints ||
        n < kMsMinPoints)
        return ok();
    int ox = INT32_MAX, oy = INT32_MAX, xmax = INT32_MIN, ymax = INT32_MIN;
    for (int i = 0; i < m; ++i) { ox = std::min(ox, hx[i]); oy = std::min(oy, hy[i]); xmax = std::max(xmax, hx[i]); ymax = std::max(ymax, hy[i]); }
    for (int j = 0; j < n; ++j) { ox = std::min(ox, gx[j]); oy = std::min(oy, gy[j]); xmax = std::max(xmax, gx[j]); ymax = std::max(ymax, gy[j]); }
    const int W = (xmax - ox) / 2 + 1, H = (ymax - oy) / 2 + 1;
    if ((int64_t)W * H > kMsMaxCells) return ok();
    // cells: masses summed, coordinates = cell index
    std::vector<int32_t> slat((size_t)W * H, -1), tlat((size_t)W * H, -1);
    std::vector<double> ca, cb;
    std::vector<int32_t> csx, csy, ctx, cty;
    for (int i = 0; i < m; ++i) {
        const int bx = (hx[i] - ox) / 2, by = (hy[i] - oy) / 2;
        int32_t &c = slat[(size_t)by * W + bx];
        if (c < 0) { c = (int32_t)ca.size(); ca.push_back(0.0); csx.push_back(bx); csy.push_back(by); }
        ca[c] += as[i];
    }
    for (int j = 0; j < n; ++j) {
        const int bx = (gx[j] - ox) / 2, by = (gy[j] - oy) / 2;
        int32_t &c = tlat[(size_t)by * W + bx];
        if (c < 0) { c = (int32_t)cb.size(); cb.push_back(0.0); ctx.push_back(bx); cty.push_back(by); }
        cb[c] += bs[j];
    }
    ot_problem cp{};
    cp.m = (int32_t)ca.size();
    cp.n = (int32_t)cb.size();
    cp.a = ca.data();
    cp.b = cb.data();
    cp.cost = h->cd.kind;
    cp.src_x = csx.data(); cp.src_y = csy.data(); cp.dst_x = ctx.data(); cp.dst_y = cty.data();
    ot_options co = o;
    co.multiscale = o.multiscale - 1;
    // the coarse duals only guide the fine start: relative tolerance ms_tol on every test
    co.tol = o.ms_tol > 0 ? o.ms_tol : std::max(o.tol, 1e-4);
    double cmass = 0.0;
    for (double x : ca) cmass += x;
    co.feas_l1 = co.tol * cmass;
    co.max_iter = std::max(o.max_iter, 200);
    co.warm_u = co.warm_v = nullptr;
    co.warm_i = co.warm_j = nullptr;
    co.warm_npairs = 0;
    co.warm_count = 0;
    co.add_max = 0;
    co.stream = st;
    ot_ipm *hc = new (std::nothrow) ot_ipm();
    if (!hc) return fail(OT_ERR_OOM, "multiscale: host allocation failed");
    Error e = create_impl(&cp, &co, hc);
    while (e.code == OT_OK && !hc->done) e = do_step(hc, nullptr);
    if (e.code == OT_OK) {
        const double scale = h->cd.kind == OT_COST_SQEUCLID ? 4.0 : 2.0;
        e = [&]() -> Error {
            DevTemp<int32_t> dsl, dtl;
            DevTemp<double> wu, wv;
            OT_TRY(dsl.alloc((int64_t)W * H, st));
            OT_TRY(dtl.alloc((int64_t)W * H, st));
            OT_TRY(wu.alloc(m, st));
            OT_TRY(wv.alloc(n, st));
            OT_CUDA(cudaMemcpyAsync(dsl.p, slat.data(), sizeof(int32_t) * slat.size(), cudaMemcpyHostToDevice, st));
            OT_CUDA(cudaMemcpyAsync(dtl.p, tlat.data(), sizeof(int32_t) * tlat.size(), cudaMemcpyHostToDevice, st));
            upsample_kernel<<<(unsigned)std::min<int64_t>(ceil_div(m, 256), 1024), 256, 0, st>>>(
                m, h->sx, h->sy, ox, oy, W, H, dsl.p, hc->u, scale, wu.p);
            OT_LAUNCHED();
            upsample_kernel<<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 1024), 256, 0, st>>>(
                n, h->tx, h->ty, ox, oy, W, H, dtl.p, hc->v, scale, wv.p);
            OT_LAUNCHED();
            h->ms_u.resize(m);
            h->ms_v.resize(n);
            OT_CUDA(cudaMemcpyAsync(h->ms_u.data(), wu.p, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
            OT_CUDA(cudaMemcpyAsync(h->ms_v.data(), wv.p, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
            OT_CUDA(cudaStreamSynchronize(st));
            return ok();
        }();
        if (e.code == OT_OK) {
            o.warm_u = h->ms_u.data();
            o.warm_v = h->ms_v.data();
            if (o.warm_count <= 0) o.warm_count = (int32_t)std::min<int64_t>(10LL * (m + n), INT32_MAX);
            h->ms_levels = 1 + hc->ms_levels;
        }
    }
    const bool cuda_failed = e.code == OT_ERR_CUDA;
    ot_ipm_destroy(hc);
    if (cuda_failed) return e;
    return ok();
}

Error create_impl(const ot_problem *P, const ot_options *O, ot_ipm *h) {
    if (!P || P->m <= 0 || P->n <= 0 || !P->a || !P->b) return fail(OT_ERR_ARG, "problem: sizes or masses missing");
    const int32_t m0 = P->m, n0 = P->n;
    if ((uint64_t)m0 * (uint64_t)n0 > (1ull << 32)) return fail(OT_ERR_ARG, "problem: m*n exceeds 2^32");
    if (O) h->opt = *O; else ot_options_default(&h->opt);
    ot_options &o = h->opt;
    if (!(o.tol > 0) || o.max_iter < 0 || o.max_cg <= 0 || o.max_corr < 0 || !(o.step_scale > 0 && o.step_scale < 1) ||
        (o.precision != 0 && o.precision != 1) || o.jset_refresh < 0 || !std::isfinite(o.jset_cmax) ||
        o.precond < 0 || o.precond > 1 || !(o.ic_tau >= 0 && o.ic_tau < 1) || o.tc_update < -1 || o.tc_update > 1 ||
        !(o.direct_cg_tol >= 0 && o.direct_cg_tol < 1))
        return fail(OT_ERR_ARG, "options: out of range");
    if (P->cost < 0 || P->cost > OT_COST_DENSE) return fail(OT_ERR_ARG, "problem: unknown cost kind");
    const bool dense = P->cost == OT_COST_DENSE;
    if (dense && !P->C) return fail(OT_ERR_ARG, "problem: dense cost without C");
    if (dense && (uint64_t)m0 * (uint64_t)n0 > (1ull << 30)) return fail(OT_ERR_ARG, "problem: dense C above 2^30 entries");
    const bool on_dev = P->inputs_on_device != 0;
    // host copies of the masses and coordinates (device inputs are read back: m + n values)
    std::vector<double> A(m0), B(n0);
    auto fetch = [&](void *dst, const void *src, size_t bytes) -> Error {
        if (on_dev) OT_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
        else memcpy(dst, src, bytes);
        return ok();
    };
    OT_TRY(fetch(A.data(), P->a, sizeof(double) * m0));
    OT_TRY(fetch(B.data(), P->b, sizeof(double) * n0));
    double sa = 0, sb = 0;
    for (int i = 0; i < m0; ++i) {
        if (!(A[i] >= 0) || !std::isfinite(A[i])) return fail(OT_ERR_ARG, "problem: negative or non-finite mass in a");
        sa += A[i];
    }
    for (int j = 0; j < n0; ++j) {
        if (!(B[j] >= 0) || !std::isfinite(B[j])) return fail(OT_ERR_ARG, "problem: negative or non-finite mass in b");
        sb += B[j];
    }
    if (!(sa > 0) || std::fabs(sa - sb) > 1e-12 * sa) return fail(OT_ERR_ARG, "problem: sum(a) != sum(b)");
    // coordinates (caller's indexing)
    std::vector<int32_t> X0(m0, 0), Y0(m0, 0), G0(n0, 0), H0(n0, 0);
    if (!dense) {
        const bool have = P->src_x && P->src_y && P->dst_x && P->dst_y;
        if (!have && (P->src_w <= 0 || P->dst_w <= 0 || m0 % P->src_w || n0 % P->dst_w))
            return fail(OT_ERR_ARG, "problem: no coordinates and no valid grid widths");
        if (have) {
            OT_TRY(fetch(X0.data(), P->src_x, sizeof(int32_t) * m0));
            OT_TRY(fetch(Y0.data(), P->src_y, sizeof(int32_t) * m0));
            OT_TRY(fetch(G0.data(), P->dst_x, sizeof(int32_t) * n0));
            OT_TRY(fetch(H0.data(), P->dst_y, sizeof(int32_t) * n0));
        } else {
            for (int i = 0; i < m0; ++i) { X0[i] = i % P->src_w; Y0[i] = i / P->src_w; }
            for (int j = 0; j < n0; ++j) { G0[j] = j % P->dst_w; H0[j] = j / P->dst_w; }
        }
    }
    // zero-mass presolve: only points with positive mass enter the solve
    for (int i = 0; i < m0; ++i) if (A[i] > 0) h->src_map.push_back(i);
    for (int j = 0; j < n0; ++j) if (B[j] > 0) h->dst_map.push_back(j);
    const int32_t m = (int32_t)h->src_map.size(), n = (int32_t)h->dst_map.size();
    h->m0 = m0;
    h->n0 = n0;
    h->presolved = m < m0 || n < n0;
    h->src_inv.assign(m0, -1);
    h->dst_inv.assign(n0, -1);
    for (int r = 0; r < m; ++r) h->src_inv[h->src_map[r]] = r;
    for (int r = 0; r < n; ++r) h->dst_inv[h->dst_map[r]] = r;
    h->m = m;
    h->n = n;
    h->sigma_f = (double)m / sa;
    std::vector<double> as(m), bs(n);
    double f2 = 0;
    for (int i = 0; i < m; ++i) { as[i] = A[h->src_map[i]] * h->sigma_f; f2 += as[i] * as[i]; }
    for (int j = 0; j < n; ++j) { bs[j] = B[h->dst_map[j]] * (sa / sb) * h->sigma_f; f2 += bs[j] * bs[j]; }
    h->fnorm = std::sqrt(f2);
    h->as_host = as;
    h->bs_host = bs;
    std::vector<int32_t> hx(m), hy(m), gx(n), gy(n);
    for (int i = 0; i < m; ++i) { hx[i] = X0[h->src_map[i]]; hy[i] = Y0[h->src_map[i]]; }
    for (int j = 0; j < n; ++j) { gx[j] = G0[h->dst_map[j]]; gy[j] = H0[h->dst_map[j]]; }
    int xmin = INT32_MAX, xmax = INT32_MIN, ymin = INT32_MAX, ymax = INT32_MIN;
    for (int i = 0; i < m0; ++i) { xmin = std::min(xmin, X0[i]); xmax = std::max(xmax, X0[i]); ymin = std::min(ymin, Y0[i]); ymax = std::max(ymax, Y0[i]); }
    for (int j = 0; j < n0; ++j) { xmin = std::min(xmin, G0[j]); xmax = std::max(xmax, G0[j]); ymin = std::min(ymin, H0[j]); ymax = std::max(ymax, H0[j]); }
    if (xmin <= -(1 << 14) || ymin <= -(1 << 14) || xmax >= (1 << 14) || ymax >= (1 << 14))
        return fail(OT_ERR_ARG, "problem: coordinates must satisfy |x|, |y| < 2^14");
    h->ox = (int32_t)(((int64_t)xmin + xmax) / 2);
    h->oy = (int32_t)(((int64_t)ymin + ymax) / 2);

    int dev;
    OT_CUDA(cudaGetDevice(&dev));
    h->device = dev;
    OT_CUDA(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
    {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    }
    if (o.stream) {
        h->st = (cudaStream_t)o.stream;
    } else {
        OT_CUDA(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    cudaStream_t st = h->st;
    OT_CUDA(cudaMalloc((void **)&h->a_s, sizeof(double) * m));
    OT_CUDA(cudaMalloc((void **)&h->b_s, sizeof(double) * n));
    OT_CUDA(cudaMalloc((void **)&h->u, sizeof(double) * m));
    OT_CUDA(cudaMalloc((void **)&h->v, sizeof(double) * n));
    OT_CUDA(cudaMalloc((void **)&h->sx, sizeof(int32_t) * m));
    OT_CUDA(cudaMalloc((void **)&h->sy, sizeof(int32_t) * m));
    OT_CUDA(cudaMalloc((void **)&h->tx, sizeof(int32_t) * n));
    OT_CUDA(cudaMalloc((void **)&h->ty, sizeof(int32_t) * n));
    OT_CUDA(cudaMalloc((void **)&h->pi, sizeof(int32_t) * std::max(m, 1)));
    OT_CUDA(cudaMalloc((void **)&h->pj, sizeof(int32_t) * std::max(m, 1)));
    OT_CUDA(cudaMalloc((void **)&h->pd, sizeof(double) * std::max(m, 1)));
    OT_CUDA(cudaMalloc((void **)&h->pcount, sizeof(int32_t)));
    OT_CUDA(cudaMalloc((void **)&h->pstrong, sizeof(int)));
    OT_CUDA(cudaMalloc((void **)&h->rowmin, sizeof(unsigned long long) * m));
    OT_CUDA(cudaMalloc((void **)&h->lbv, sizeof(double)));
    if (o.add_max > m) o.add_max = m;
    h->ic_tau = o.ic_tau > 0 ? o.ic_tau : 1e-2;
    OT_CUDA(cudaMemcpyAsync(h->a_s, as.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st));
    OT_CUDA(cudaMemcpyAsync(h->b_s, bs.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
    OT_CUDA(cudaMemcpyAsync(h->sx, hx.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
    OT_CUDA(cudaMemcpyAsync(h->sy, hy.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
    OT_CUDA(cudaMemcpyAsync(h->tx, gx.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
    OT_CUDA(cudaMemcpyAsync(h->ty, gy.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
    if (h->presolved) {
        // the caller's points and index maps stay on the device for the dual completion
        OT_CUDA(cudaMalloc((void **)&h->d_src_map, sizeof(int32_t) * m));
        OT_CUDA(cudaMalloc((void **)&h->d_dst_map, sizeof(int32_t) * n));
        OT_CUDA(cudaMemcpyAsync(h->d_src_map, h->src_map.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
        OT_CUDA(cudaMemcpyAsync(h->d_dst_map, h->dst_map.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
        if (!dense) {
            OT_CUDA(cudaMalloc((void **)&h->fsx, sizeof(int32_t) * m0));
            OT_CUDA(cudaMalloc((void **)&h->fsy, sizeof(int32_t) * m0));
            OT_CUDA(cudaMalloc((void **)&h->ftx, sizeof(int32_t) * n0));
            OT_CUDA(cudaMalloc((void **)&h->fty, sizeof(int32_t) * n0));
            OT_CUDA(cudaMemcpyAsync(h->fsx, X0.data(), sizeof(int32_t) * m0, cudaMemcpyHostToDevice, st));
            OT_CUDA(cudaMemcpyAsync(h->fsy, Y0.data(), sizeof(int32_t) * m0, cudaMemcpyHostToDevice, st));
            OT_CUDA(cudaMemcpyAsync(h->ftx, G0.data(), sizeof(int32_t) * n0, cudaMemcpyHostToDevice, st));
            OT_CUDA(cudaMemcpyAsync(h->fty, H0.data(), sizeof(int32_t) * n0, cudaMemcpyHostToDevice, st));
        }
    }
    if (dense) {
        // the caller's matrix on the device (validated there), then its kept rows and columns
        const int64_t cnt = (int64_t)m0 * n0;
        OT_CUDA(cudaMalloc((void **)&h->fC, sizeof(double) * cnt));
        OT_CUDA(cudaMemcpyAsync(h->fC, P->C, sizeof(double) * cnt,
                                on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        int *bad = nullptr;
        OT_CUDA(cudaMalloc((void **)&bad, sizeof(int)));
        int hbad = 0;
        cudaMemsetAsync(bad, 0, sizeof(int), st);
        check_dense_kernel<<<(unsigned)std::min<int64_t>(ceil_div(cnt, 256), 4LL * h->num_sms), 256, 0, st>>>(
            cnt, h->fC, bad);
        g_launches.fetch_add(1);
        cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
        const cudaError_t ce = cudaStreamSynchronize(st);
        cudaFree(bad);
        if (ce != cudaSuccess) return fail(OT_ERR_CUDA, cudaGetErrorString(ce));
        if (hbad) return fail(OT_ERR_ARG, "problem: C has a negative or non-finite entry");
        if (h->presolved) {
            OT_CUDA(cudaMalloc((void **)&h->C, sizeof(double) * (int64_t)m * n));
            gather_dense_kernel<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)m * n, 256), 4LL * h->num_sms), 256, 0,
                                  st>>>(m, n, n0, h->d_src_map, h->d_dst_map, h->fC, h->C);
            OT_LAUNCHED();
        } else {
            h->C = h->fC;
            h->fC = nullptr;
        }
    }
    h->cd.kind = P->cost;
    h->cd.m = m;
    h->cd.n = n;
    h->cd.sx = h->sx; h->cd.sy = h->sy; h->cd.tx = h->tx; h->cd.ty = h->ty;
    h->cd.C = h->C;
    if (h->presolved) {
        // warm-start inputs are in the caller's indexing: keep what concerns the kept points
        if (o.warm_u && o.warm_v) {
            h->warm_ur.resize(m);
            h->warm_vr.resize(n);
            for (int r = 0; r < m; ++r) h->warm_ur[r] = o.warm_u[h->src_map[r]];
            for (int r = 0; r < n; ++r) h->warm_vr[r] = o.warm_v[h->dst_map[r]];
            o.warm_u = h->warm_ur.data();
            o.warm_v = h->warm_vr.data();
        }
        if (o.warm_i && o.warm_j && o.warm_npairs > 0) {
            for (int64_t t = 0; t < o.warm_npairs; ++t) {
                const int32_t i = o.warm_i[t], j = o.warm_j[t];
                if (i < 0 || i >= m0 || j < 0 || j >= n0) return fail(OT_ERR_ARG, "warm pairs: index out of range");
                if (h->src_inv[i] < 0 || h->dst_inv[j] < 0) continue;
                h->warm_ir.push_back(h->src_inv[i]);
                h->warm_jr.push_back(h->dst_inv[j]);
            }
            o.warm_i = h->warm_ir.data();
            o.warm_j = h->warm_jr.data();
            o.warm_npairs = (int64_t)h->warm_ir.size();
        }
    }

    OT_TRY(multiscale_start(h, as, bs, hx, hy, gx, gy, st));

    // initial support (Section 3.2 end) and Mehrotra's starting point
    int32_t *ii = nullptr, *jj = nullptr;
    int64_t psi0 = 0;
    OT_TRY(initial_support(h->cd, o.init_cost, &ii, &jj, &psi0, st));
    const int64_t cap = std::max<int64_t>(2 * psi0, psi0 + 8LL * m);
    Error e = support_alloc(h->S[0], cap, m, n);
    if (e.code == OT_OK) e = support_alloc(h->S[1], cap, m, n);
    if (e.code == OT_OK) {
        cudaMemcpyAsync(h->S[0].i, ii, sizeof(int32_t) * psi0, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(h->S[0].j, jj, sizeof(int32_t) * psi0, cudaMemcpyDeviceToDevice, st);
        cudaStreamSynchronize(st);
    }
    cudaFree(ii);
    cudaFree(jj);
    OT_TRY(e);
    h->S[0].psi = psi0;
    OT_TRY(rebuild_views(h->S[0], m, n, st));
    const bool want_warm = (o.warm_u && o.warm_v) || (o.warm_i && o.warm_j && o.warm_npairs > 0);
    OT_TRY(newton_alloc(h->W, m, n, h->S[h->cur].cap, h->num_sms));
    h->W.verbose = h->opt.verbose;
    h->W.direct_cg_tol = h->opt.direct_cg_tol;
    OT_TRY(complete_feasible(h, st));
    OT_TRY(chol_alloc(h->chol, n));
    int cgs = 0;
    double crit_cold = INFINITY;
    if (want_warm) {
        // the cold starting point first: a warm start is kept only when its point is better
        OT_TRY(support_costs(h->W, h->cd, h->S[h->cur], st));
        OT_TRY(mehrotra_start(h->W, h->S[h->cur], h->a_s, h->b_s, h->u, h->v, o.precision, o.cg_tol_pred,
                              20 * o.max_cg, &cgs, st));
        h->cg_total += cgs;
        OT_TRY(start_crit(h, &crit_cold));
        if (o.warm_u && o.warm_v) OT_TRY(warm_support(h, o, st));
        if (o.warm_i && o.warm_j && o.warm_npairs > 0) OT_TRY(warm_pairs(h, o, st));
        h->warm_active = true;
    }
    OT_TRY(support_costs(h->W, h->cd, h->S[h->cur], st));
    const bool warm = o.warm_u && o.warm_v && o.warm_mode == 1;
    if (warm) {
        OT_CUDA(cudaMemcpyAsync(h->u, o.warm_u, sizeof(double) * m, cudaMemcpyHostToDevice, st));
        OT_CUDA(cudaMemcpyAsync(h->v, o.warm_v, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    }
    OT_TRY(mehrotra_start(h->W, h->S[h->cur], h->a_s, h->b_s, h->u, h->v, o.precision, o.cg_tol_pred, 20 * o.max_cg,
                          &cgs, st, warm));
    h->cg_total += cgs;
    if (want_warm) {
        double crit_warm = INFINITY;
        OT_TRY(start_crit(h, &crit_warm));
        if (!(crit_warm < crit_cold)) OT_TRY(cold_restart(h));
    }
    OT_CUDA(cudaStreamSynchronize(st));
    return ok();
}

}  // namespace

// ======================================================================== C ABI
extern "C" {

void ot_options_default(ot_options *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->tol = 1e-6;
    o->feas_l1 = 1e-8;
    o->cg_tol_pred = 1e-6;
    o->cg_tol_corr = 1e-3;
    o->max_iter = 200;
    o->max_cg = 1000;
    o->max_corr = 3;
    o->step_scale = 0.995;
    o->precision = 1;
    o->linear_solver = 0;
    o->init_cost = 2.0;
    o->rm_mu_frac = 1e-3;
    o->rm_p_frac = 1e-3;
    o->add_max = 0;
    o->new_col_rule = 1;
    o->jset_cmax = 0.0;
    o->jset_refresh = 3;
    o->multiscale = 0;
    o->ms_tol = 0.0;
    o->precond = 0;
    o->ic_tau = 0.0;
    o->tc_update = 0;
    o->direct_cg_tol = 0.0;
    o->verbose = 0;
    o->stream = nullptr;
}

int ot_ipm_create(const ot_problem *prob, const ot_options *opt, ot_ipm_t **out) {
    if (!out) { set_thread_error("ot_ipm_create: out is NULL"); return OT_ERR_ARG; }
    *out = nullptr;
    ot_ipm *h = new (std::nothrow) ot_ipm();
    if (!h) { set_thread_error("ot_ipm_create: host allocation failed"); return OT_ERR_OOM; }
    const auto t0 = std::chrono::steady_clock::now();
    Error e = create_impl(prob, opt, h);
    h->create_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (e.code != OT_OK) {
        set_thread_error(e.msg.c_str());
        ot_ipm_destroy(h);
        return e.code;
    }
    *out = h;
    return OT_OK;
}

int ot_ipm_step(ot_ipm_t *h, ot_iter_info *info) {
    if (!h) return OT_ERR_ARG;
    if (h->done) {
        if (info) { memset(info, 0, sizeof(*info)); info->done = 1; info->iter = h->iter; }
        return OT_OK;
    }
    return record(h, do_step(h, info));
}

int ot_ipm_solve(ot_ipm_t *h, ot_result *res) {
    if (!h) return OT_ERR_ARG;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, h->st);
    int rc = OT_OK;
    ot_iter_info inf{};
    while (!h->done) {
        rc = ot_ipm_step(h, &inf);
        if (rc != OT_OK) break;
    }
    cudaEventRecord(e1, h->st);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (res) {
        memset(res, 0, sizeof(*res));
        res->status = rc;
        double hs[SC_COUNT];
        Error e = residuals(h->W, h->S[h->cur], h->a_s, h->b_s, h->u, h->v, h->st);
        if (e.code == OT_OK) e = read_scalars(h->W, hs, h->st);
        if (e.code == OT_OK) {
            double lb = h->last_lb;
            if (!h->done) {
                Error e2 = lower_bound(h, &lb);
                if (e2.code != OT_OK) lb = NAN;
            }
            const double ctp = hs[SC_CP];
            res->obj = ctp / h->sigma_f;
            res->lower_bound = lb / h->sigma_f;
            res->rel_gap = (ctp - lb) / (1.0 + std::fabs(ctp));
            res->r1_l1 = (hs[SC_R1A_L1] + hs[SC_R1B_L1]) / h->sigma_f;
            res->mu = hs[SC_PS] / (double)h->S[h->cur].psi;
        } else if (rc == OT_OK) {
            rc = record(h, e);
            res->status = rc;
        }
        res->iters = h->iter;
        res->cg_iters = (int32_t)h->cg_total;
        res->direct_iters = h->direct_total;
        res->max_fill = h->max_fill;
        res->psi = h->S[h->cur].psi;
        res->seconds = ms * 1e-3;
        res->warm_added = h->warm_added;
        res->warm_restarts = h->warm_restarts;
        res->create_seconds = h->create_seconds;
        res->ms_levels = h->ms_levels;
    }
    return rc;
}

int ot_ipm_solve_batch(ot_ipm_t *const *hs, int32_t count, ot_result *res, int32_t workers) {
    if (!hs || !res || count < 0) {
        set_thread_error("ot_ipm_solve_batch: invalid argument");
        return OT_ERR_ARG;
    }
    for (int32_t i = 0; i < count; ++i)
        if (!hs[i]) {
            set_thread_error("ot_ipm_solve_batch: NULL handle");
            return OT_ERR_ARG;
        }
    if (count == 0) return OT_OK;
    const int nw = std::max(1, std::min<int32_t>(workers > 0 ? workers : kBatchWorkers, count));
    // One queue, largest instance first, drained by nw host threads (one stream per handle).  The
    // mixed solve of one instance leaves the GPU partly idle (its factorisation is a chain of
    // latency-bound launches, its refinement CG waits on host checks), so a second instance in
    // flight fills the gaps; more than two contend for the SMs the chains wait on.
    std::vector<int32_t> order(count);
    for (int32_t i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        return (int64_t)hs[x]->m * hs[x]->n > (int64_t)hs[y]->m * hs[y]->n;
    });
    std::atomic<size_t> next{0};
    auto run = [&](int32_t i) {
        cudaSetDevice(hs[i]->device);
        std::memset(&res[i], 0, sizeof(ot_result));
        res[i].status = ot_ipm_solve(hs[i], &res[i]);
    };
    auto drain = [&]() {
        for (;;) {
            const size_t q = next.fetch_add(1);
            if (q >= order.size()) break;
            run(order[q]);
        }
    };
    std::vector<std::thread> pool;
    pool.reserve(nw - 1);
    for (int t = 1; t < nw; ++t) pool.emplace_back(drain);
    drain();
    for (auto &t : pool) t.join();
    for (int32_t i = 0; i < count; ++i)
        if (res[i].status != OT_OK) {
            set_thread_error("ot_ipm_solve_batch: an instance failed (see its ot_result.status)");
            return res[i].status;
        }
    return OT_OK;
}

int ot_ipm_get_solution(ot_ipm_t *h, int32_t *i, int32_t *j, double *p, int64_t cap, int64_t *nnz, double *u,
                        double *v) {
    if (!h || !nnz) return OT_ERR_ARG;
    const Support &S = h->S[h->cur];
    *nnz = S.psi;
    if (cap < S.psi) { h->err = "ot_ipm_get_solution: buffer too small"; return OT_ERR_BUF_TOO_SMALL; }
    if ((!i || !j || !p) && S.psi > 0) return OT_ERR_ARG;
    Error e = ok();
    double *tmp = nullptr;
    if (cudaMalloc((void **)&tmp, sizeof(double) * std::max<int64_t>(S.psi, 1)) != cudaSuccess) return OT_ERR_OOM;
    scale_copy_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(S.psi, 256), 1024)), 256, 0, h->st>>>(
        S.psi, S.p, 1.0 / h->sigma_f, tmp);
    g_launches.fetch_add(1);
    cudaMemcpyAsync(i, S.i, sizeof(int32_t) * S.psi, cudaMemcpyDeviceToHost, h->st);
    cudaMemcpyAsync(j, S.j, sizeof(int32_t) * S.psi, cudaMemcpyDeviceToHost, h->st);
    cudaMemcpyAsync(p, tmp, sizeof(double) * S.psi, cudaMemcpyDeviceToHost, h->st);
    cudaError_t ce = cudaStreamSynchronize(h->st);
    cudaFree(tmp);
    if (ce != cudaSuccess) return record(h, fail(OT_ERR_CUDA, cudaGetErrorString(ce)));
    caller_pairs(h, i, j, S.psi);
    e = caller_duals(h, u, v, true);
    return record(h, e);
}

int ot_ipm_get_state(ot_ipm_t *h, int32_t *i, int32_t *j, double *p, double *s, int64_t cap, int64_t *psi,
                     double *u, double *v) {
    if (!h || !psi) return OT_ERR_ARG;
    const Support &S = h->S[h->cur];
    *psi = S.psi;
    if (cap < S.psi) { h->err = "ot_ipm_get_state: buffer too small"; return OT_ERR_BUF_TOO_SMALL; }
    if (i) cudaMemcpyAsync(i, S.i, sizeof(int32_t) * S.psi, cudaMemcpyDeviceToHost, h->st);
    if (j) cudaMemcpyAsync(j, S.j, sizeof(int32_t) * S.psi, cudaMemcpyDeviceToHost, h->st);
    if (p) cudaMemcpyAsync(p, S.p, sizeof(double) * S.psi, cudaMemcpyDeviceToHost, h->st);
    if (s) cudaMemcpyAsync(s, S.s, sizeof(double) * S.psi, cudaMemcpyDeviceToHost, h->st);
    cudaError_t ce = cudaStreamSynchronize(h->st);
    if (ce != cudaSuccess) return record(h, fail(OT_ERR_CUDA, cudaGetErrorString(ce)));
    caller_pairs(h, i, j, S.psi);
    return record(h, caller_duals(h, u, v, false));
}

int ot_ipm_newton_direction(ot_ipm_t *h, int32_t solver, double cg_tol, int32_t max_cg, double *du, double *dv,
                            double *dp, double *ds, int64_t cap, int32_t *cg_iters) {
    if (!h) return OT_ERR_ARG;
    if (solver < OT_LS_PCG64 || solver > OT_LS_TREE || !(cg_tol > 0) || max_cg <= 0)
        return record(h, fail(OT_ERR_ARG, "ot_ipm_newton_direction: bad solver, tolerance or iteration limit"));
    Support &S = h->S[h->cur];
    if (cap < S.psi) return record(h, fail(OT_ERR_BUF_TOO_SMALL, "ot_ipm_newton_direction: buffer too small"));
    Newton &W = h->W;
    cudaStream_t st = h->st;
    const int n = h->n;
    Error e = [&]() -> Error {
        OT_TRY(residuals(W, S, h->a_s, h->b_s, h->u, h->v, st));
        OT_TRY(schur_setup(W, S, st));
        W.direct = nullptr;
        W.dense = nullptr;
        W.d32 = nullptr;
        W.ic = nullptr;
        W.tree = nullptr;
        if (solver == OT_LS_DENSE32) {
            if (n > kDense32LateMaxN) return fail(OT_ERR_UNSUPPORTED, "FP32 dense factor: n above its limit");
            if (!h->d32.A) { OT_TRY(d32_alloc(h->d32, n)); h->d32.tc_mode = h->opt.tc_update; }
            OT_TRY(d32_assemble(h->d32, W, S, st));
            OT_TRY(d32_factor(h->d32, (float)kPivotEps, st));
            W.d32 = &h->d32;
        } else if (solver == OT_LS_DENSE64) {
            if (n > kDenseMaxN) return fail(OT_ERR_UNSUPPORTED, "FP64 dense factor: n above its limit");
            if (!h->dense.A) OT_TRY(dense_alloc(h->dense, n));
            bool changed = false;
            OT_TRY(chol_assemble(h->chol, W, S, 0.0, &changed, st));
            OT_CUDA(cudaMemsetAsync(h->dense.err, 0, sizeof(int), st));
            OT_TRY(dense_factor(h->dense, h->chol, kPivotEps, st));
            W.direct = &h->chol;
            W.dense = &h->dense;
        } else if (solver == OT_LS_SPARSE) {
            bool changed = false;
            OT_TRY(chol_assemble(h->chol, W, S, 0.0, &changed, st));
            if (changed || !h->chol.have_symbolic) OT_TRY(chol_symbolic(h->chol, st));
            OT_TRY(chol_numeric(h->chol, kPivotEps, st));
            W.direct = &h->chol;
        } else if (solver == OT_LS_TREE) {
            bool forest = false;
            OT_TRY(forest_setup(h, S, &forest, st));
            if (!forest) return fail(OT_ERR_UNSUPPORTED, "forest solver: the support graph has a cycle");
            W.tree = &h->tree;
        } else if (solver == OT_LS_IC) {
            if (!h->ic.perm) OT_TRY(ic_alloc(h->ic, n));
            bool changed = false;
            OT_TRY(chol_assemble(h->chol, W, S, 0.0, &changed, st));
            OT_TRY(ic_factor(h->ic, h->chol, 1e-2, kPivotEps, st));
            W.ic = &h->ic;
        }
        W.fp64_fallback = false;
        OT_TRY(corrector_r3(W, S, 0.0, nullptr, nullptr, st));   // predictor: r3 = -p s
        Rhs R{W.r1a, W.r1b, W.r2, W.r3};
        SolveStats ss;
        OT_TRY(newton_solve(W, S, R, cg_tol, max_cg, solver == OT_LS_MIXED ? 1 : 0, W.du, W.dv, W.ds, W.dp, &ss,
                            st));
        std::vector<double> hdu(du ? h->m : 0), hdv(dv ? n : 0);
        if (du) OT_CUDA(cudaMemcpyAsync(hdu.data(), W.du, sizeof(double) * h->m, cudaMemcpyDeviceToHost, st));
        if (dv) OT_CUDA(cudaMemcpyAsync(hdv.data(), W.dv, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        if (dp) OT_CUDA(cudaMemcpyAsync(dp, W.dp, sizeof(double) * S.psi, cudaMemcpyDeviceToHost, st));
        if (ds) OT_CUDA(cudaMemcpyAsync(ds, W.ds, sizeof(double) * S.psi, cudaMemcpyDeviceToHost, st));
        OT_CUDA(cudaStreamSynchronize(st));
        // to the caller's indexing (points removed by the presolve: 0)
        if (du) {
            std::fill(du, du + h->m0, 0.0);
            for (int r = 0; r < h->m; ++r) du[h->presolved ? h->src_map[r] : r] = hdu[r];
        }
        if (dv) {
            std::fill(dv, dv + h->n0, 0.0);
            for (int r = 0; r < n; ++r) dv[h->presolved ? h->dst_map[r] : r] = hdv[r];
        }
        if (cg_iters) *cg_iters = ss.cg_iters;
        return ok();
    }();
    W.direct = nullptr;
    W.dense = nullptr;
    W.d32 = nullptr;
    W.ic = nullptr;
    W.tree = nullptr;
    return record(h, e);
}

int ot_ipm_set_state(ot_ipm_t *h, const int32_t *i, const int32_t *j, const double *p, const double *s, int64_t psi,
                     const double *u, const double *v, int32_t reset_mu0) {
    if (!h || psi <= 0 || !i || !j || !p || !s || !u || !v) return OT_ERR_ARG;
    for (int64_t e = 0; e < psi; ++e) {
        if (i[e] < 0 || i[e] >= h->m0 || j[e] < 0 || j[e] >= h->n0 || !(p[e] > 0) || !(s[e] > 0))
            return record(h, fail(OT_ERR_ARG, "ot_ipm_set_state: entry out of range or nonpositive"));
        if (e > 0 && ((int64_t)i[e] * h->n0 + j[e]) <= ((int64_t)i[e - 1] * h->n0 + j[e - 1]))
            return record(h, fail(OT_ERR_ARG, "ot_ipm_set_state: pairs not sorted by (i, j) or repeated"));
        if (h->src_inv[i[e]] < 0 || h->dst_inv[j[e]] < 0)
            return record(h, fail(OT_ERR_ARG, "ot_ipm_set_state: pair on a point with zero mass"));
    }
    std::vector<int32_t> ri, rj;
    std::vector<double> ru, rv;
    if (h->presolved) {
        // to the solve's indexing (the maps are increasing, so the (i, j) order is kept)
        ri.resize(psi);
        rj.resize(psi);
        for (int64_t e = 0; e < psi; ++e) { ri[e] = h->src_inv[i[e]]; rj[e] = h->dst_inv[j[e]]; }
        ru.resize(h->m);
        rv.resize(h->n);
        for (int r = 0; r < h->m; ++r) ru[r] = u[h->src_map[r]];
        for (int r = 0; r < h->n; ++r) rv[r] = v[h->dst_map[r]];
        i = ri.data();
        j = rj.data();
        u = ru.data();
        v = rv.data();
    }
    Error e = ensure_capacity(h, psi);
    if (e.code != OT_OK) return record(h, e);
    Support &S = h->S[h->cur];
    cudaMemcpyAsync(S.i, i, sizeof(int32_t) * psi, cudaMemcpyHostToDevice, h->st);
    cudaMemcpyAsync(S.j, j, sizeof(int32_t) * psi, cudaMemcpyHostToDevice, h->st);
    cudaMemcpyAsync(S.p, p, sizeof(double) * psi, cudaMemcpyHostToDevice, h->st);
    cudaMemcpyAsync(S.s, s, sizeof(double) * psi, cudaMemcpyHostToDevice, h->st);
    cudaMemcpyAsync(h->u, u, sizeof(double) * h->m, cudaMemcpyHostToDevice, h->st);
    cudaMemcpyAsync(h->v, v, sizeof(double) * h->n, cudaMemcpyHostToDevice, h->st);
    S.psi = psi;
    e = rebuild_views(S, h->m, h->n, h->st);
    if (e.code == OT_OK) e = support_costs(h->W, h->cd, S, h->st);
    cudaError_t ce = cudaStreamSynchronize(h->st);
    if (e.code == OT_OK && ce != cudaSuccess) e = fail(OT_ERR_CUDA, cudaGetErrorString(ce));
    if (reset_mu0) h->mu0 = -1.0;
    h->done = false;
    h->strong = 1;
    return record(h, e);
}

int ot_ipm_ic_apply(ot_ipm_t *h, double tau, const double *b, double *x) {
    if (!h || !b || !x || !(tau >= 0)) return OT_ERR_ARG;
    Newton &W = h->W;
    cudaStream_t st = h->st;
    const int n = h->n;
    Error e = [&]() -> Error {
        Support &S = h->S[h->cur];
        OT_TRY(schur_setup(W, S, st));
        if (!h->ic.perm) OT_TRY(ic_alloc(h->ic, n));
        bool changed = false;
        OT_TRY(chol_assemble(h->chol, W, S, 0.0, &changed, st));
        OT_TRY(ic_factor(h->ic, h->chol, tau, kPivotEps, st));
        std::vector<double> hb(n), hx(n);
        for (int r = 0; r < n; ++r) hb[r] = b[h->presolved ? h->dst_map[r] : r];
        DevTemp<double> db, dx;
        OT_TRY(db.alloc(n, st));
        OT_TRY(dx.alloc(n, st));
        OT_CUDA(cudaMemcpyAsync(db.p, hb.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
        OT_TRY(ic_apply(h->ic, db.p, dx.p, st));
        OT_CUDA(cudaMemcpyAsync(hx.data(), dx.p, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        OT_CUDA(cudaStreamSynchronize(st));
        std::fill(x, x + h->n0, 0.0);
        for (int r = 0; r < n; ++r) x[h->presolved ? h->dst_map[r] : r] = hx[r];
        return ok();
    }();
    return record(h, e);
}

double ot_ipm_mass_scale(const ot_ipm_t *h) { return h ? h->sigma_f : 0.0; }

void ot_ipm_destroy(ot_ipm_t *h) {
    if (!h) return;
    if (h->st) cudaStreamSynchronize(h->st);
    support_free(h->S[0]);
    support_free(h->S[1]);
    newton_free(h->W);
    chol_free(h->chol);
    dense_free(h->dense);
    d32_free(h->d32);
    jset_free(h->jset);
    ic_free(h->ic);
    tree_free(h->tree);
    void *ptrs[] = {h->a_s, h->b_s, h->C, h->sx, h->sy, h->tx, h->ty, h->u, h->v, h->pi, h->pj, h->pd,
                    h->pcount, h->pstrong, h->rowmin, h->lbv, h->d_src_map, h->d_dst_map, h->fsx, h->fsy,
                    h->ftx, h->fty, h->fC};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->own_stream && h->st) cudaStreamDestroy(h->st);
    delete h;
}

const char *ot_ipm_last_error(const ot_ipm_t *h) { return h ? h->err.c_str() : "null handle"; }

const char *ot_last_error(void) { return t_last_error.c_str(); }

int ot_price_topk(int32_t m, int32_t n, const int32_t *sx, const int32_t *sy, const int32_t *tx, const int32_t *ty,
                  const double *u, const double *v, const int32_t *sup_i, const int32_t *sup_j, int64_t psi,
                  int32_t kmax, int32_t precision, int32_t *out_i, int32_t *out_j, double *out_d,
                  int32_t *out_count, void *stream) {
    if (m <= 0 || n <= 0 || kmax < 0 || psi < 0 || !sx || !sy || !tx || !ty || !u || !v || !out_i || !out_j ||
        !out_count || (psi > 0 && (!sup_i || !sup_j)) || (precision != 0 && precision != 1)) {
        set_thread_error("ot_price_topk: invalid argument");
        return OT_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    PriceInput in;
    in.m = m; in.n = n;
    in.sx = sx; in.sy = sy; in.tx = tx; in.ty = ty;
    in.u = u; in.v = v;
    in.sup_i = sup_i; in.sup_j = sup_j; in.psi = psi;
    in.kmax = kmax;
    in.precision = precision;
    Error e = coord_origin(m, n, sx, sy, tx, ty, &in.origin_x, &in.origin_y, st);
    if (e.code == OT_OK) e = price_topk(in, out_i, out_j, out_d, out_count, nullptr, st);
    if (e.code != OT_OK) set_thread_error(e.msg.c_str());
    return e.code;
}

int ot_price_topk_ex(int32_t m, int32_t n, const int32_t *sx, const int32_t *sy, const int32_t *tx,
                     const int32_t *ty, const double *u, const double *v, const int32_t *sup_i, const int32_t *sup_j,
                     int64_t psi, int32_t kmax, int32_t precision, int32_t *out_i, int32_t *out_j, double *out_d,
                     int32_t *out_count, const ot_price_opts *opts, void *stream) {
    ot_price_opts po{};
    if (opts) po = *opts;
    const bool dense = po.cost == OT_COST_DENSE;
    if (m <= 0 || n <= 0 || kmax < 0 || psi < 0 || po.cost < OT_COST_SQEUCLID || po.cost > OT_COST_DENSE ||
        (dense ? !po.C : (!sx || !sy || !tx || !ty)) || !u || !v || !out_i || !out_j || !out_count ||
        (psi > 0 && (!sup_i || !sup_j)) || (precision != 0 && precision != 1) || po.scan_rows < 0 ||
        !std::isfinite(po.jset_cmax)) {
        set_thread_error("ot_price_topk_ex: invalid argument");
        return OT_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    PriceInput in;
    in.m = m; in.n = n;
    in.sx = sx; in.sy = sy; in.tx = tx; in.ty = ty;
    in.u = u; in.v = v;
    in.sup_i = sup_i; in.sup_j = sup_j; in.psi = psi;
    in.kmax = kmax;
    in.precision = precision;
    in.kind = po.cost;
    in.C = po.C;
    in.rows = po.scan_rows;
    JSet J;
    Error e = ok();
    if (!dense) e = coord_origin(m, n, sx, sy, tx, ty, &in.origin_x, &in.origin_y, st);
    if (e.code == OT_OK && po.jset_cmax > 0) {
        e = jset_build(po.cost, m, n, sx, sy, tx, ty, po.C, po.jset_cmax, &J, st);
        in.ji = J.i; in.jj = J.j; in.jn = J.n; in.jlim = J.lim; in.jcmax = J.cmax;
    }
    if (e.code == OT_OK) e = price_topk(in, out_i, out_j, out_d, out_count, nullptr, st);
    if (J.i) {
        cudaStreamSynchronize(st);
        jset_free(J);
    }
    if (e.code != OT_OK) set_thread_error(e.msg.c_str());
    return e.code;
}

int64_t ot_kernel_launches(void) { return g_launches.load(); }

void ot_kernel_timing_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_kt.mu);
    g_kt.on = on != 0;
    for (int k = 0; k < KT_COUNT; ++k) { g_kt.ms[k] = 0; g_kt.count[k] = 0; g_kt.work[k] = 0; }
}

int ot_kernel_timing_read(double *ms, int64_t *count, double *work, int32_t cap) {
    if (!ms || !count || cap < KT_COUNT) return OT_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_kt.mu);
    for (int k = 0; k < KT_COUNT; ++k) {
        for (auto &pr : g_kt.pending[k]) {
            cudaEventSynchronize(pr.second);
            float t = 0;
            cudaEventElapsedTime(&t, pr.first, pr.second);
            g_kt.ms[k] += t;
            g_kt.count[k] += 1;
            g_kt.pool.push_back(pr.first);
            g_kt.pool.push_back(pr.second);
        }
        g_kt.pending[k].clear();
        ms[k] = g_kt.ms[k];
        count[k] = g_kt.count[k];
        if (work) work[k] = g_kt.work[k];
    }
    return KT_COUNT;
}

int ot_abi_struct_sizes(int64_t *out, int32_t count) {
    if (!out || count < 4) return OT_ERR_ARG;
    out[0] = sizeof(ot_problem);
    out[1] = sizeof(ot_options);
    out[2] = sizeof(ot_iter_info);
    out[3] = sizeof(ot_result);
    return 4;
}

}  // extern "C"
