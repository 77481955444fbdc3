// Pricing (Section 3.4) + support enlargement selection (Section 3.2): internal API.
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
};

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
