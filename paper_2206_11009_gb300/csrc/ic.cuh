// Incomplete Cholesky preconditioner with a drop tolerance for the Schur complement S_M
// (Section 4.2: the iterative phase preconditions CG with an incomplete Cholesky factor whose drop
// tolerance is lowered when CG needs too many iterations).
//
// GPU form: the factor keeps the pattern of S_M without the entries the drop test removes on
// their own value (|S_rs| < tau sqrt(S_rr S_ss)) and without fill, in a multicolour order -- the
// targets greedily coloured so that no two neighbours in that pattern share a colour, colours in
// sequence -- so that every row of one colour depends only on rows of earlier colours: the
// factorisation and both triangular solves proceed one colour at a time with all rows of the
// colour in parallel.  Within the pattern, an entry l_rs is dropped when
// |l_rs d_s| < tau sqrt(S_rr S_ss).  A pivot
// d_r <= eps S_rr becomes +infinity (the alternative of Section 4.2), which grounds one node per
// connected component of the singular S_M.
#pragma once

#include <vector>

#include "chol.cuh"
#include "common.cuh"

namespace ot {

struct IncChol {
    int32_t n = 0;
    int ncolors = 0;
    std::vector<int32_t> hcolor_ptr;       // first new index of each colour (host), ncolors + 1
    int32_t *perm = nullptr;               // new index -> target
    // strictly lower L by rows (new indices), with the position of each entry's value in the
    // assembled S_M (Chol::Ax); strictly upper U = L^T by rows with the position in Lx
    int32_t *Lp = nullptr, *Lj = nullptr;
    int64_t *Lsrc = nullptr;
    double *Lx = nullptr;
    int32_t *Up = nullptr, *Uj = nullptr;
    int64_t *Upos = nullptr;
    double *D = nullptr;                   // pivots (new order); +inf for grounded rows
    double *Ad = nullptr;                  // S_rr (new order)
    double *y = nullptr;                   // work vector (new order)
    int64_t nnzL = 0, capL = 0;
    double tau = 0.0;
    int32_t *dropped = nullptr;            // entries dropped by the last factorisation (device)
};

Error ic_alloc(IncChol &F, int32_t n);
void ic_free(IncChol &F);

// Colour the pattern of the assembled S_M (C.hAp / C.hAj on the host), build L's pattern and
// factor C's values (exact S_M: assembled with drop 0).
Error ic_factor(IncChol &F, const Chol &C, double tau, double eps, cudaStream_t st);

// x = (L D L^T)^+ b (the grounded rows of D^-1 are 0), b and x device vectors in target order.
Error ic_apply(const IncChol &F, const double *b, double *x, cudaStream_t st);

}  // namespace ot
