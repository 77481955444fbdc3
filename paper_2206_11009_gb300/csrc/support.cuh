// Support bookkeeping (Sections 3.2-3.3): initial support, removal, merge of new pairs, and the
// CSR (by source) / CSC (by target) views used by every per-iteration kernel.
#pragma once

#include "common.cuh"

namespace ot {

// Costs of the problem, evaluated on the device.
struct CostDev {
    int32_t kind = OT_COST_SQEUCLID;
    int32_t m = 0, n = 0;
    const int32_t *sx = nullptr, *sy = nullptr, *tx = nullptr, *ty = nullptr;
    const double *C = nullptr;  // dense row-major (OT_COST_DENSE)
};

__device__ __forceinline__ double cost_at(const CostDev &c, int i, int j) {
    if (c.kind == OT_COST_DENSE) return c.C[(int64_t)i * c.n + j];
    const int dx = c.sx[i] - c.tx[j], dy = c.sy[i] - c.ty[j];
    switch (c.kind) {
    case OT_COST_SQEUCLID: return (double)(dx * dx + dy * dy);
    case OT_COST_EUCLID: return __dsqrt_rn((double)(dx * dx + dy * dy));
    case OT_COST_L1: return (double)(abs(dx) + abs(dy));
    default: return (double)max(abs(dx), abs(dy));
    }
}

// Sorted support of size psi with capacity cap (structure of arrays on the device).
struct Support {
    int64_t psi = 0, cap = 0;
    int32_t *i = nullptr, *j = nullptr;   // sorted by (i, j)
    double *p = nullptr, *s = nullptr;
    int32_t *row_ptr = nullptr;           // m+1
    int32_t *col_ptr = nullptr;           // n+1
    int32_t *col_perm = nullptr;          // CSR index of the k-th entry in (j, i) order
    int32_t *col_row = nullptr;           // source of the k-th entry in (j, i) order
};

// Initial support: {c_ij <= thr} plus every row's and every column's cheapest pair (ties:
// smaller index).  Returns the pairs (device, sorted by (i, j)) in freshly allocated buffers
// owned by the caller (cudaFree), count in *psi.
Error initial_support(const CostDev &c, double thr, int32_t **out_i, int32_t **out_j, int64_t *psi,
                      cudaStream_t st);

// Rebuild row_ptr, col_ptr, col_perm, col_row for the current (i, j) arrays.
Error rebuild_views(Support &S, int32_t m, int32_t n, cudaStream_t st);

// Removal (reading of Section 3.2): flag[e] = 1 for the pairs that leave -- candidates
// p < rm_p_frac*min(a_i, b_j) with theta < 1, except the edges of a maximum-weight spanning
// forest of the support graph (weights p, ties by jlin), so the support stays connected; at most
// kmax leave, smallest (p, jlin) first.  *count (host) receives the number flagged.
Error removal_flags(const Support &S, int32_t m, int32_t n, const double *a_s, const double *b_s,
                    double rm_p_frac, int32_t kmax, uint8_t *flag, int64_t *count, cudaStream_t st);

// New support = (S without flagged) merged with the k new pairs (ni, nj) at p = s = p_new, or,
// with a_cap / b_cap (device masses) given, at p = min(p_new, a_i, b_j) and s = p_new^2 / p.
// Writes into T (capacity >= result size) and rebuilds T's views.  S and T must differ.
Error merge_support(const Support &S, const uint8_t *flag, const int32_t *ni, const int32_t *nj,
                    int64_t k, double p_new, int32_t m, int32_t n, Support &T, cudaStream_t st,
                    const double *a_cap = nullptr, const double *b_cap = nullptr);

}  // namespace ot
