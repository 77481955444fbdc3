// Forest solver of the Newton system by the Euler-tour technique (see tree.cuh).
#include "tree.cuh"
#include "primitives.cuh"

#include <algorithm>

namespace ot {
namespace {

constexpr int kT = 256;

inline unsigned grid_for_count(int64_t count) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(count, kT), 4096));
}

#define TS_LOOP(var, count) \
    for (int64_t var = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; var < (count); var += (int64_t)gridDim.x * blockDim.x)

// arc a: pair e = a / 2, a even: source -> target, a odd: target -> source (nodes: rows 0..m-1,
// columns m..m+n-1); key (from, to)
__global__ void arc_keys_kernel(int64_t arcs, int m, int nn, const int32_t *__restrict__ si,
                                const int32_t *__restrict__ sj, uint64_t *__restrict__ key, uint32_t *__restrict__ val) {
    TS_LOOP(a, arcs) {
        const int64_t e = a >> 1;
        const int x = si[e], y = m + sj[e];
        const int from = (a & 1) ? y : x, to = (a & 1) ? x : y;
        key[a] = (uint64_t)from * (uint64_t)nn + (uint64_t)to;
        val[a] = (uint32_t)a;
    }
}

__global__ void arc_pos_kernel(int64_t arcs, const uint32_t *__restrict__ order, int32_t *__restrict__ pos) {
    TS_LOOP(p, arcs) pos[order[p]] = (int32_t)p;
}

// first sorted position of every node's arcs (v in [0, nn])
__global__ void node_start_kernel(int64_t arcs, int nn, const uint64_t *__restrict__ key, int32_t *__restrict__ start) {
    TS_LOOP(v, (int64_t)nn + 1) {
        const uint64_t target = (uint64_t)v * (uint64_t)nn;
        int64_t lo = 0, hi = arcs;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (key[mid] < target) lo = mid + 1; else hi = mid;
        }
        start[v] = (int32_t)lo;
    }
}

// successor of x -> y: the arc after y -> x in y's list (cyclically); every component's tour is
// cut before it returns to the first arc of its root (its smallest node)
__global__ void succ_kernel(int64_t arcs, int m, const int32_t *__restrict__ si, const int32_t *__restrict__ sj,
                            const uint32_t *__restrict__ order, const int32_t *__restrict__ pos,
                            const int32_t *__restrict__ start, const int32_t *__restrict__ labels,
                            int32_t *__restrict__ succ) {
    TS_LOOP(a, arcs) {
        const int64_t e = a >> 1;
        const int y = (a & 1) ? si[e] : m + sj[e];   // head of arc a
        const int pt = pos[a ^ 1];                     // y -> x in y's list
        const int pn = pt + 1 < start[y + 1] ? pt + 1 : start[y];
        int32_t s = (int32_t)order[pn];
        // the tour of y's component starts at the root's first arc: the arc leading there ends it
        if (labels[y] == y && pn == start[y]) s = -1;
        succ[a] = s;
    }
}

__global__ void jump_init_kernel(int64_t arcs, const int32_t *__restrict__ succ, const double *__restrict__ w,
                                 int32_t *__restrict__ nxt, double *__restrict__ val) {
    TS_LOOP(a, arcs) {
        nxt[a] = succ[a];
        val[a] = w ? w[a] : 1.0;
    }
}

// one round of pointer jumping: val[a] += val[nxt[a]], nxt[a] = nxt[nxt[a]] (double-buffered)
__global__ void jump_kernel(int64_t arcs, const int32_t *__restrict__ nxt, const double *__restrict__ val,
                            int32_t *__restrict__ nxt2, double *__restrict__ val2) {
    TS_LOOP(a, arcs) {
        const int32_t q = nxt[a];
        if (q >= 0) {
            val2[a] = val[a] + val[q];
            nxt2[a] = nxt[q];
        } else {
            val2[a] = val[a];
            nxt2[a] = -1;
        }
    }
}

// arcs ranked (count from the arc to its tour's end): the one of a twin pair ranked higher comes
// first in the tour and points down; it is its head's down arc
__global__ void down_kernel(int64_t arcs, int m, const int32_t *__restrict__ si, const int32_t *__restrict__ sj,
                            const double *__restrict__ rnk, int32_t *__restrict__ down) {
    TS_LOOP(a, arcs) {
        if (rnk[a] > rnk[a ^ 1]) {
            const int64_t e = a >> 1;
            const int y = (a & 1) ? si[e] : m + sj[e];
            down[y] = (int32_t)a;
        }
    }
}

__global__ void fill_int_kernel(int64_t count, int32_t v, int32_t *__restrict__ x) {
    TS_LOOP(k, count) x[k] = v;
}

// weights of the subtree-sum pass: b of the head on every down arc
__global__ void w_subtree_kernel(int nn, const int32_t *__restrict__ down, const double *__restrict__ b,
                                 double *__restrict__ w) {
    TS_LOOP(v, nn) if (down[v] >= 0) w[down[v]] = b[v];
}

// f_v = sum of b over v's subtree = S[down_v] - S[up_v] (suffix sums); delta_v = f_v / theta of
// v's parent edge; weights of the path pass: +delta on the down arc, -delta on the up arc
__global__ void w_path_kernel(int nn, const int32_t *__restrict__ down, const double *__restrict__ S,
                              const double *__restrict__ theta, double *__restrict__ f, double *__restrict__ w) {
    TS_LOOP(v, nn) {
        const int32_t a = down[v];
        if (a < 0) { f[v] = 0.0; continue; }
        const double fv = S[a] - S[a ^ 1];
        const double d = fv / theta[a >> 1];
        f[v] = d;
        w[a] = d;
        w[a ^ 1] = -d;
    }
}

// phi_v = sum of delta over the path root -> v = delta_v - T[down_v] (the tour's total is 0);
// dv_j = -phi_{m+j}
__global__ void phi_kernel(int m, int n, const int32_t *__restrict__ down, const double *__restrict__ T,
                           const double *__restrict__ delta, double *__restrict__ dv) {
    TS_LOOP(j, n) {
        const int v = m + (int)j;
        const int32_t a = down[v];
        const double phi = a < 0 ? 0.0 : delta[v] - T[a];
        dv[j] = -phi;
    }
}

__global__ void rhs_nodes_kernel(int m, int n, const double *__restrict__ rhs, double *__restrict__ b) {
    TS_LOOP(v, (int64_t)m + n) b[v] = v < m ? 0.0 : -rhs[v - m];
}

__global__ void zero_kernel(int64_t count, double *__restrict__ x) {
    TS_LOOP(k, count) x[k] = 0.0;
}

template <typename T>
Error tdalloc(T **p, int64_t count) {
    OT_CUDA(cudaMalloc((void **)p, sizeof(T) * (size_t)std::max<int64_t>(count, 1)));
    return ok();
}
template <typename T>
void tdfree(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

// suffix sums of w along the tours (w == nullptr: all ones) into T.val
Error suffix_sums(TreeSolver &T, const double *w, cudaStream_t st) {
    const int64_t arcs = 2 * T.psi;
    const unsigned g = grid_for_count(arcs);
    jump_init_kernel<<<g, kT, 0, st>>>(arcs, T.succ, w, T.nxt, T.val);
    OT_LAUNCHED();
    for (int r = 0; r < T.rounds; ++r) {
        jump_kernel<<<g, kT, 0, st>>>(arcs, T.nxt, T.val, T.nxt2, T.val2);
        OT_LAUNCHED();
        std::swap(T.nxt, T.nxt2);
        std::swap(T.val, T.val2);
    }
    return ok();
}

}  // namespace

Error tree_alloc(TreeSolver &T, int32_t m, int32_t n, int64_t cap) {
    tree_free(T);
    T.m = m;
    T.n = n;
    T.cap = cap;
    const int64_t nn = (int64_t)m + n, arcs = 2 * cap;
    OT_TRY(tdalloc(&T.order, arcs));
    OT_TRY(tdalloc(&T.node_start, nn + 1));
    OT_TRY(tdalloc(&T.succ, arcs));
    OT_TRY(tdalloc(&T.succ2, arcs));
    OT_TRY(tdalloc(&T.nxt, arcs));
    OT_TRY(tdalloc(&T.nxt2, arcs));
    OT_TRY(tdalloc(&T.val, arcs));
    OT_TRY(tdalloc(&T.val2, arcs));
    OT_TRY(tdalloc(&T.down, nn));
    OT_TRY(tdalloc(&T.f, nn));
    OT_TRY(tdalloc(&T.phi, nn));
    OT_TRY(tdalloc(&T.b, nn));
    return ok();
}

void tree_free(TreeSolver &T) {
    tdfree(T.order); tdfree(T.node_start); tdfree(T.succ); tdfree(T.succ2); tdfree(T.nxt); tdfree(T.nxt2);
    tdfree(T.val); tdfree(T.val2); tdfree(T.down); tdfree(T.f); tdfree(T.phi); tdfree(T.b);
    T = TreeSolver();
}

Error tree_build(TreeSolver &T, const Support &S, const int32_t *labels, cudaStream_t st) {
    const int m = T.m, n = T.n, nn = m + n;
    if (S.psi > T.cap) OT_TRY(tree_alloc(T, m, n, std::max<int64_t>(S.psi, (int64_t)(1.5 * T.cap))));
    T.psi = S.psi;
    const int64_t arcs = 2 * S.psi;
    T.rounds = 0;
    while ((1LL << T.rounds) < arcs) ++T.rounds;
    const unsigned g = grid_for_count(arcs), gn = grid_for_count((int64_t)nn + 1);
    DevTemp<uint64_t> key;
    DevTemp<int32_t> pos;
    OT_TRY(key.alloc(arcs, st));
    OT_TRY(pos.alloc(arcs, st));
    arc_keys_kernel<<<g, kT, 0, st>>>(arcs, m, nn, S.i, S.j, key.p, T.order);
    OT_LAUNCHED();
    int bits = 1;
    while (bits < 64 && (((uint64_t)nn * (uint64_t)nn - 1) >> bits)) ++bits;
    OT_TRY(radix_sort_pairs(key.p, T.order, arcs, bits, st));
    arc_pos_kernel<<<g, kT, 0, st>>>(arcs, T.order, pos.p);
    OT_LAUNCHED();
    node_start_kernel<<<gn, kT, 0, st>>>(arcs, nn, key.p, T.node_start);
    OT_LAUNCHED();
    succ_kernel<<<g, kT, 0, st>>>(arcs, m, S.i, S.j, T.order, pos.p, T.node_start, labels, T.succ);
    OT_LAUNCHED();
    OT_TRY(suffix_sums(T, nullptr, st));   // ranks
    fill_int_kernel<<<gn, kT, 0, st>>>(nn, -1, T.down);
    OT_LAUNCHED();
    down_kernel<<<g, kT, 0, st>>>(arcs, m, S.i, S.j, T.val, T.down);
    OT_LAUNCHED();
    T.ready = true;
    return ok();
}

Error tree_solve(TreeSolver &T, const Support &S, const double *theta, const double *rhs, double *dv,
                 cudaStream_t st) {
    if (!T.ready || T.psi != S.psi) return fail(OT_ERR_ARG, "tree_solve: structure not built for this support");
    const int m = T.m, n = T.n, nn = m + n;
    const int64_t arcs = 2 * T.psi;
    const unsigned g = grid_for_count(arcs), gn = grid_for_count(nn);
    DevTemp<double> w;
    OT_TRY(w.alloc(arcs, st));
    rhs_nodes_kernel<<<gn, kT, 0, st>>>(m, n, rhs, T.b);
    OT_LAUNCHED();
    zero_kernel<<<g, kT, 0, st>>>(arcs, w.p);
    OT_LAUNCHED();
    w_subtree_kernel<<<gn, kT, 0, st>>>(nn, T.down, T.b, w.p);
    OT_LAUNCHED();
    OT_TRY(suffix_sums(T, w.p, st));
    // T.val: subtree suffix sums; f = delta per node, path weights into w
    w_path_kernel<<<gn, kT, 0, st>>>(nn, T.down, T.val, theta, T.f, w.p);
    OT_LAUNCHED();
    OT_TRY(suffix_sums(T, w.p, st));
    phi_kernel<<<grid_for_count(n), kT, 0, st>>>(m, n, T.down, T.val, T.f, dv);
    OT_LAUNCHED();
    return ok();
}

}  // namespace ot
