// Pricing (Section 3.4) + support enlargement selection (Section 3.2): internal API.
// Cost kinds: the squared Euclidean distance and the distances of Section 5.1 from integer
// coordinates, or an explicit matrix (always priced in FP64).
#pragma once

#include "common.cuh"

namespace ot {

struct PriceInput {
    int32_t m = 0, n = 0;
    const int32_t *sx = nullptr, *sy = nullptr, *tx = nullptr, *ty = nullptr;  // device
    const double *u = nullptr, *v = nullptr;                                   // device
    const int32_t *sup_i = nullptr, *sup_j = nullptr;  // device, sorted by (i, j)
    const int32_t *row_ptr = nullptr;                  // device (m+1); nullptr: built here
    int64_t psi = 0;
    int32_t kmax = 0;
    int32_t precision = 1;  // 1: FP32 scan + FP64 recheck; 0: FP64 scan
    int32_t origin_x = 0, origin_y = 0;  // coordinate shift applied before the FP32 form
    int32_t num_sms = 0;
    int32_t rows = 0;       // rows per scan tile (8..256); 0: chosen from the problem size
    int32_t kind = OT_COST_SQEUCLID;   // ot_cost_kind
    const double *C = nullptr;         // OT_COST_DENSE: device, m x n row-major
    // Heuristic set J of Section 3.4: when jn >= 0 only the jn listed pairs (ji, jj) are priced;
    // the support pairs inside J are those with integer cost key < jlim (point costs) or with
    // C_ij < jcmax (explicit matrix).
    const int32_t *ji = nullptr, *jj = nullptr;
    int64_t jn = -1;
    long long jlim = 0;
    double jcmax = 0.0;
};

// The pairs of J = {(i, j) : c_ij < cmax} (Section 3.4), sorted by (i, j), in device buffers
// owned by the struct (jset_free).  lim: the integer cost key bound (c_ij < cmax <=> key < lim;
// the key is dx^2 + dy^2 for the squared and Euclidean distances, |dx| + |dy| for L1,
// max(|dx|, |dy|) for L-infinity).
struct JSet {
    int32_t *i = nullptr, *j = nullptr;
    int64_t n = 0;
    long long lim = 0;
    double cmax = 0.0;
};
long long jset_limit(int kind, double cmax);
Error jset_build(int kind, int32_t m, int32_t n, const int32_t *sx, const int32_t *sy, const int32_t *tx,
                 const int32_t *ty, const double *C, double cmax, JSet *out, cudaStream_t st);
void jset_free(JSet &J);

struct PriceStats {
    uint64_t gathered = 0;   // pairs rechecked in FP64
    uint32_t valid = 0;      // candidates with d < 0 outside the support
    uint32_t selected = 0;
    float err_bound = 0.f;   // proven |d_fp32 - d_fp64| bound used for the window
};

// Selection written to out_i/out_j/out_d (capacity kmax, device) and *out_count (device).
// One host synchronisation (to size the candidate buffer).  Stats filled when non-null.
Error price_topk(const PriceInput &in, int32_t *out_i, int32_t *out_j, double *out_d,
                 int32_t *out_count, PriceStats *stats, cudaStream_t st);

// Integer origin (midpoint of the bounding box of all points), device inputs, host result.
Error coord_origin(int32_t m, int32_t n, const int32_t *sx, const int32_t *sy, const int32_t *tx,
                   const int32_t *ty, int32_t *ox, int32_t *oy, cudaStream_t st);

// row_ptr[i] = first support index with sup_i >= i (i in [0, m]); sup_i sorted.
Error build_row_ptr(const int32_t *sup_i, int64_t psi, int32_t m, int32_t *row_ptr, cudaStream_t st);

}  // namespace ot
