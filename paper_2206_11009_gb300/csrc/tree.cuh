// Exact solver of the Newton system when the support graph is a forest (Section 4.3: near
// optimality the support approaches a forest, Theorem 2, and the system then needs no fill).
//
// With phi_i = du_i for sources and phi_{m+j} = -dv_j for targets, the normal equations
// [M V; V^T N] [du; dv] = [beta1; beta2] become the Laplacian L phi = b of the support graph with
// edge weights theta (b_i = beta1_i, b_{m+j} = -beta2_j).  On a tree rooted at r, summing the
// equations over the subtree of a node y with parent x gives theta_xy (phi_y - phi_x) = f_y, the
// sum of b over the subtree, so phi_y = phi_r + sum over the path r -> y of f / theta.
//
// GPU form (Euler-tour technique): every pair gives two arcs; the arcs sorted by (from, to) give
// each node's adjacency, the successor of x -> y in the tour is the arc after y -> x in y's list,
// and every component's tour is cut at its smallest node (its root).  Pointer jumping (log2 of the
// tour length rounds) ranks the arcs; an arc before its twin points down the tree.  Subtree sums
// and path sums are then suffix sums over the tour (again by pointer jumping) of b placed on the
// down arcs, and of +f/theta on the down arcs and -f/theta on the up arcs.
#pragma once

#include "common.cuh"
#include "support.cuh"

namespace ot {

struct TreeSolver {
    int32_t m = 0, n = 0;
    int64_t psi = 0, cap = 0;
    bool ready = false;                 // structure built for the current support
    int rounds = 0;                     // pointer-jumping rounds (ceil log2 of the longest tour)
    uint32_t *order = nullptr;          // arcs sorted by (from, to)
    int32_t *node_start = nullptr;      // (m + n + 1) offsets into `order`
    int32_t *succ = nullptr, *succ2 = nullptr;  // tour successor (-1 at a tour's end), scratch
    int32_t *nxt = nullptr, *nxt2 = nullptr;
    double *val = nullptr, *val2 = nullptr;
    int32_t *down = nullptr;            // per node: its down arc (-1 at roots)
    double *f = nullptr;                // per node: subtree sum
    double *phi = nullptr;              // per node: potential
    double *b = nullptr;                // per node: right-hand side
};

Error tree_alloc(TreeSolver &T, int32_t m, int32_t n, int64_t cap);
void tree_free(TreeSolver &T);

// Structure of the current support (a forest: psi == m + n - #components); labels[v] = the
// smallest node of v's component (union-find roots over rows 0..m-1 and columns m..m+n-1).
Error tree_build(TreeSolver &T, const Support &S, const int32_t *labels, cudaStream_t st);

// dv = S_M^+ rhs through the tree Laplacian with b = (0, -rhs); theta per support entry (CSR
// order).  rhs must sum to zero on every component; dv is determined up to a constant per
// component (the caller projects it).
Error tree_solve(TreeSolver &T, const Support &S, const double *theta, const double *rhs, double *dv,
                 cudaStream_t st);

}  // namespace ot
