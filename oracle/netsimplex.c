/*
 * Oracle O1 -- plain primal network simplex for the Kantorovich transportation LP.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls this
 * file; only the tests, the smoke check and the CPU-baseline leg of the benchmark do.
 *
 * Problem (Section 2, eqs. feasible_region / OT_problem / kantorovichlp):
 *     min sum_ij c_ij p_ij   s.t.  sum_j p_ij = a_i,  sum_i p_ij = b_j,  p >= 0,
 * read as a min-cost flow on the complete bipartite graph of Section 2.2 (sources i send
 * a_i, sinks j receive b_j).  Any vertex of the feasible region is a spanning forest of at
 * most m+n-1 arcs (Section 2.2), which is what a simplex basis is.
 *
 * Textbook method (Ahuja, Magnanti & Orlin, "Network Flows", ch. 11), written plainly:
 *   - an artificial root R joined to every node by an artificial arc of cost BIG gives the
 *     initial feasible spanning tree (source i -> R carries a_i, R -> sink j carries b_j);
 *   - node potentials phi make every tree arc's reduced cost c - phi_tail + phi_head zero;
 *   - entering arc: block search over the m*n real arcs (most negative reduced cost in the
 *     first block, scanned cyclically, that contains a negative one);
 *   - leaving arc: the last blocking arc met when the pivot cycle is walked along the
 *     entering arc's orientation starting at the apex (Cunningham's strongly feasible tree
 *     rule, which rules out cycling);
 *   - after each pivot the tree is rebuilt by a breadth-first search from R (O(m+n)).
 * Costs are evaluated on the fly, never stored (kinds below), except the dense kind.
 *
 * Outputs: the real tree arcs with their flows (a basic optimal coupling), the potentials
 * u_i = phi_i and v_j = -phi_{m+j} (so that c_ij - u_i - v_j is the reduced cost), and
 * the objective.  For integer costs every potential is an exact integer in double.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { K_SQEUCLID = 0, K_EUCLID = 1, K_L1 = 2, K_LINF = 3, K_DENSE = 4 };

typedef struct {
    int m, n, kind;
    const double *C;                 /* dense, row-major m x n (kind == K_DENSE) */
    const double *sx, *sy, *tx, *ty; /* coordinates (grid kinds) */
} cost_t;

static double cost_ij(const cost_t *c, int i, int j) {
    if (c->kind == K_DENSE) return c->C[(int64_t)i * c->n + j];
    double dx = c->sx[i] - c->tx[j], dy = c->sy[i] - c->ty[j];
    switch (c->kind) {
    case K_SQEUCLID: return dx * dx + dy * dy;
    case K_EUCLID: return sqrt(dx * dx + dy * dy);
    case K_L1: return fabs(dx) + fabs(dy);
    default: return fabs(dx) > fabs(dy) ? fabs(dx) : fabs(dy);
    }
}

typedef struct {
    int m, n, N, root, narc;
    int *tail, *head;       /* per tree arc */
    double *flow, *cost;    /* per tree arc */
    int *parent, *parc, *depth, *queue, *adj_start, *adj_fill, *adj;
    double *pot;
} tree_t;

static void rebuild(tree_t *t) {
    int N = t->N;
    memset(t->adj_start, 0, sizeof(int) * (N + 1));
    for (int k = 0; k < t->narc; ++k) { t->adj_start[t->tail[k] + 1]++; t->adj_start[t->head[k] + 1]++; }
    for (int v = 0; v < N; ++v) t->adj_start[v + 1] += t->adj_start[v];
    memcpy(t->adj_fill, t->adj_start, sizeof(int) * N);
    for (int k = 0; k < t->narc; ++k) { t->adj[t->adj_fill[t->tail[k]]++] = k; t->adj[t->adj_fill[t->head[k]]++] = k; }
    for (int v = 0; v < N; ++v) t->parent[v] = -2;
    int qh = 0, qt = 0;
    t->queue[qt++] = t->root;
    t->parent[t->root] = -1; t->parc[t->root] = -1; t->depth[t->root] = 0; t->pot[t->root] = 0.0;
    while (qh < qt) {
        int p = t->queue[qh++];
        for (int e = t->adj_start[p]; e < t->adj_start[p + 1]; ++e) {
            int k = t->adj[e];
            int w = t->tail[k] == p ? t->head[k] : t->tail[k];
            if (t->parent[w] != -2) continue;
            t->parent[w] = p; t->parc[w] = k; t->depth[w] = t->depth[p] + 1;
            /* tree arc reduced cost c - phi_tail + phi_head = 0 */
            t->pot[w] = (t->tail[k] == w) ? t->pot[p] + t->cost[k] : t->pot[p] - t->cost[k];
            t->queue[qt++] = w;
        }
    }
}

/* Returns 0 on success, 1 on allocation failure, 2 on a pivot without a blocking arc,
 * 3 when the pivot cap is reached. */
int ot_oracle_netsimplex(int m, int n, int kind, const double *C,
                         const double *sx, const double *sy, const double *tx, const double *ty,
                         const double *a, const double *b,
                         int *tree_i, int *tree_j, double *tree_p, int *ntree,
                         double *u, double *v, double *obj, int64_t *pivots_out,
                         int64_t block, int64_t max_pivots) {
    cost_t cs = {m, n, kind, C, sx, sy, tx, ty};
    tree_t t;
    t.m = m; t.n = n; t.N = m + n + 1; t.root = m + n; t.narc = m + n;
    int N = t.N, A = t.narc;
    t.tail = malloc(sizeof(int) * A); t.head = malloc(sizeof(int) * A);
    t.flow = malloc(sizeof(double) * A); t.cost = malloc(sizeof(double) * A);
    t.parent = malloc(sizeof(int) * N); t.parc = malloc(sizeof(int) * N);
    t.depth = malloc(sizeof(int) * N); t.queue = malloc(sizeof(int) * N);
    t.adj_start = malloc(sizeof(int) * (N + 1)); t.adj_fill = malloc(sizeof(int) * N);
    t.adj = malloc(sizeof(int) * 2 * A); t.pot = malloc(sizeof(double) * N);
    int *path_y = malloc(sizeof(int) * N), *path_x = malloc(sizeof(int) * N);
    int rc = 0;
    if (!t.tail || !t.head || !t.flow || !t.cost || !t.parent || !t.parc || !t.depth || !t.queue ||
        !t.adj_start || !t.adj_fill || !t.adj || !t.pot || !path_y || !path_x) { rc = 1; goto done; }

    /* BIG exceeds the cost of any simple path through real arcs. */
    double cmax = 0.0;
    if (kind == K_DENSE) {
        for (int64_t q = 0; q < (int64_t)m * n; ++q) if (C[q] > cmax) cmax = C[q];
    } else {
        for (int i = 0; i < m; ++i) for (int j = 0; j < n; j += (n > 64 ? n / 64 : 1)) {
            double c = cost_ij(&cs, i, j); if (c > cmax) cmax = c;
        }
        /* exact bound for grid kinds: diameter of the bounding box */
        double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
        for (int i = 0; i < m; ++i) { x0 = fmin(x0, sx[i]); x1 = fmax(x1, sx[i]); y0 = fmin(y0, sy[i]); y1 = fmax(y1, sy[i]); }
        for (int j = 0; j < n; ++j) { x0 = fmin(x0, tx[j]); x1 = fmax(x1, tx[j]); y0 = fmin(y0, ty[j]); y1 = fmax(y1, ty[j]); }
        double dx = x1 - x0, dy = y1 - y0;
        double bound = dx * dx + dy * dy + dx + dy + 1.0;
        if (bound > cmax) cmax = bound;
    }
    double BIG = (double)(m + n + 1) * (cmax + 1.0);

    for (int i = 0; i < m; ++i) {
        if (a[i] > 0.0) { t.tail[i] = i; t.head[i] = t.root; }
        else { t.tail[i] = t.root; t.head[i] = i; }
        t.flow[i] = fabs(a[i]); t.cost[i] = BIG;
    }
    for (int j = 0; j < n; ++j) {
        t.tail[m + j] = t.root; t.head[m + j] = m + j; t.flow[m + j] = b[j]; t.cost[m + j] = BIG;
    }
    rebuild(&t);

    int64_t total = (int64_t)m * n;
    if (block <= 0) { block = (int64_t)sqrt((double)total); if (block < 10) block = 10; }
    if (block > total) block = total;
    /* integer costs give integer potentials and reduced costs: any negative one is <= -1 */
    int integral = kind != K_EUCLID;
    if (kind == K_DENSE) {
        for (int64_t q = 0; q < total && integral; ++q) if (C[q] != floor(C[q])) integral = 0;
    } else {
        for (int i = 0; i < m && integral; ++i) if (sx[i] != floor(sx[i]) || sy[i] != floor(sy[i])) integral = 0;
        for (int j = 0; j < n && integral; ++j) if (tx[j] != floor(tx[j]) || ty[j] != floor(ty[j])) integral = 0;
    }
    double eps = integral ? 0.5 : 1e-10 * (1.0 + cmax);
    int64_t next = 0, piv = 0;
    for (;;) {
        /* block search for the entering arc */
        int64_t best = -1; double bestrc = -eps; int64_t scanned = 0;
        while (scanned < total) {
            int64_t lim = scanned + block < total ? block : total - scanned;
            for (int64_t q = 0; q < lim; ++q) {
                int64_t e = next + q; if (e >= total) e -= total;
                int i = (int)(e / n), j = (int)(e % n);
                double r = cost_ij(&cs, i, j) - t.pot[i] + t.pot[m + j];
                if (r < bestrc) { bestrc = r; best = e; }
            }
            next += lim; if (next >= total) next -= total;
            scanned += lim;
            if (best >= 0) break;
        }
        if (best < 0) break; /* optimal */
        if (piv >= max_pivots) { rc = 3; goto done; }
        int xi = (int)(best / n), yj = (int)(best % n);
        int x = xi, y = m + yj;
        /* paths to the apex */
        int ny = 0, nx = 0, p = y, q = x;
        while (t.depth[p] > t.depth[q]) { path_y[ny++] = p; p = t.parent[p]; }
        while (t.depth[q] > t.depth[p]) { path_x[nx++] = q; q = t.parent[q]; }
        while (p != q) { path_y[ny++] = p; p = t.parent[p]; path_x[nx++] = q; q = t.parent[q]; }
        /* ratio test */
        double delta = INFINITY;
        for (int s = 0; s < ny; ++s) { int w = path_y[s], k = t.parc[w];
            if (t.tail[k] != w && t.flow[k] < delta) delta = t.flow[k]; }
        for (int s = 0; s < nx; ++s) { int w = path_x[s], k = t.parc[w];
            if (t.head[k] != w && t.flow[k] < delta) delta = t.flow[k]; }
        if (!(delta < INFINITY)) { rc = 2; goto done; }
        /* leaving arc: last blocking arc along the orientation starting at the apex */
        int leave = -1;
        for (int s = 0; s < ny; ++s) { int w = path_y[s], k = t.parc[w];
            if (t.tail[k] != w && t.flow[k] == delta) leave = k; }
        if (leave < 0) {
            for (int s = 0; s < nx; ++s) { int w = path_x[s], k = t.parc[w];
                if (t.head[k] != w && t.flow[k] == delta) { leave = k; break; } }
        }
        /* augment */
        for (int s = 0; s < ny; ++s) { int w = path_y[s], k = t.parc[w];
            t.flow[k] += (t.tail[k] == w) ? delta : -delta; }
        for (int s = 0; s < nx; ++s) { int w = path_x[s], k = t.parc[w];
            t.flow[k] += (t.head[k] == w) ? delta : -delta; }
        t.tail[leave] = x; t.head[leave] = y; t.flow[leave] = delta; t.cost[leave] = cost_ij(&cs, xi, yj);
        rebuild(&t);
        ++piv;
    }
    {
        int cnt = 0; double o = 0.0;
        for (int k = 0; k < A; ++k) {
            if (t.tail[k] == t.root || t.head[k] == t.root) continue;
            int i = t.tail[k], j = t.head[k] - m;
            if (tree_i) { tree_i[cnt] = i; tree_j[cnt] = j; tree_p[cnt] = t.flow[k]; }
            o += t.cost[k] * t.flow[k];
            ++cnt;
        }
        *ntree = cnt; *obj = o; *pivots_out = piv;
        for (int i = 0; i < m; ++i) u[i] = t.pot[i];
        for (int j = 0; j < n; ++j) v[j] = -t.pot[m + j];
    }
done:
    free(t.tail); free(t.head); free(t.flow); free(t.cost); free(t.parent); free(t.parc);
    free(t.depth); free(t.queue); free(t.adj_start); free(t.adj_fill); free(t.adj); free(t.pot);
    free(path_y); free(path_x);
    return rc;
}
