// Direct branch (Sections 4.2-4.3): assembled Schur complement S_M, minimum-degree ordering,
// LDL^T factorisation in FP64 with the "small pivot -> infinity" rule, triangular solves.
#pragma once

#include <vector>

#include "common.cuh"
#include "newton.cuh"
#include "support.cuh"

namespace ot {

struct Chol {
    int32_t n = 0;
    // assembled S_M (off-diagonal, CSR, both triangles) + diagonal
    int64_t nnzA = 0, capA = 0;
    int32_t *Ap = nullptr, *Aj = nullptr;
    double *Ax = nullptr;
    double *Adiag = nullptr;            // S_jj (cancellation-free form)
    // sparsification (drop tolerance): kept flags and kept-only row sums
    int64_t capE = 0;
    uint8_t *keep = nullptr;
    double *exd = nullptr;              // per entry: sum of the OTHER kept theta of its row
    double *Mt = nullptr;               // per row: sum of kept theta
    double drop = 0.0;                  // drop tolerance used by the current assembly
    int64_t *a2l = nullptr;             // per A entry: position in Lx (lower part) or -1
    // symbolic (device)
    int64_t nnzL = 0, capL = 0;
    int32_t *perm = nullptr, *iperm = nullptr;
    int32_t *Lp = nullptr, *Li = nullptr;    // CSC of strictly lower L (permuted indices)
    int32_t *Rp = nullptr, *Rj = nullptr;    // CSR of strictly lower L
    int64_t *Rpos = nullptr;                 // Lx position of (row, Rj)
    double *Lx = nullptr, *D = nullptr, *dperm = nullptr;
    double *z = nullptr, *x = nullptr, *y = nullptr;
    int *done = nullptr;
    unsigned *counter = nullptr;
    unsigned *bar = nullptr;             // grid barrier of the level-scheduled kernels
    int32_t *lvl_ptr = nullptr, *lvl_cols = nullptr;
    int nlev = 0, cap_lev = 0, max_width = 0;
    int *err = nullptr;
    bool have_symbolic = false;
    double fill_pct = 0.0;              // nnz(L) / n^2 * 100
    int64_t max_nnzL = 0;               // symbolic gives up beyond this (too much fill)
    // host copy of the pattern used by the current symbolic analysis
    std::vector<int32_t> hAp, hAj;
    // ordering reused while the pattern does not grow much
    std::vector<int32_t> hperm;
    int64_t perm_nnzA = 0, perm_nnzL = 0;
};

// Dense LDL^T of the assembled S_M (moderate n, a sizeable fraction of the factor dense).
struct DenseLDL {
    int32_t n = 0;
    double *A = nullptr;      // n x n column-major; strictly lower part holds L after dense_factor
    double *LD = nullptr;     // n x 64 panel scratch (L21 D1)
    double *Linv = nullptr;   // n x 64: inverses of the unit lower diagonal blocks
    double *D = nullptr, *d0 = nullptr, *z = nullptr, *part = nullptr;
    unsigned *bar = nullptr;
    int *err = nullptr;
};

Error dense_alloc(DenseLDL &M, int32_t n);
void dense_free(DenseLDL &M);
// factor the matrix assembled in C (chol_assemble with drop = 0); +inf pivots as in chol_numeric
Error dense_factor(DenseLDL &M, const Chol &C, double eps, cudaStream_t st);
// x = S^+ b (one cooperative launch); b and x distinct device vectors of length n
Error dense_solve(DenseLDL &M, const double *b, double *x, cudaStream_t st);

Error chol_alloc(Chol &C, int32_t n);
void chol_free(Chol &C);

// Assemble the Schur complement of the support graph with its negligible pairs dropped: a pair
// whose theta is below drop x (largest theta of its source row) is left out (drop = 0: the exact
// S_M = N - V^T M^-1 V).  Off-diagonal part by rows of V; diagonal by the cancellation-free form
// over the kept pairs, so every connected component still has S e = 0.  Sets *pattern_changed.
Error chol_assemble(Chol &C, Newton &W, const Support &S, double drop, bool *pattern_changed, cudaStream_t st);

// Minimum-degree ordering and the pattern of L (host), uploaded to the device.  Returns
// OT_ERR_UNSUPPORTED when nnz(L) would exceed C.max_nnzL (the caller keeps using PCG).
Error chol_symbolic(Chol &C, cudaStream_t st);

// Numeric LDL^T of the assembled S_M; pivots d <= eps * S_jj become +infinity.
Error chol_numeric(Chol &C, double eps, cudaStream_t st);

// x = S_M^+ b through L D L^T (+inf pivots ground one node per component), b and x device
// vectors of length n (natural order), one cooperative launch.  Errors of the launch's bounded
// barrier are reported by the next chol_numeric / by the caller reading C.err.
Error chol_solve(Chol &C, const double *b, double *x, cudaStream_t st);

}  // namespace ot
