// FP32 dense LDL^T of S_M with an explicit inverse factor, used as the preconditioner of an FP64
// conjugate-gradient refinement of the Newton system (Section 4's normal equations, solved in
// mixed precision).
//
// S_M = N - V^T M^-1 V has non-positive off-diagonal entries and exactly zero row sums (S_M e = 0,
// Section 4.1), so every Schur complement met during elimination has them too.  The pivot of the
// column being eliminated is therefore minus the sum of its remaining off-diagonal entries, and no
// step of the factorisation, of the inverse of the unit lower factor (L^-1 >= 0) or of the
// assembly ever subtracts quantities of opposite sign: the FP32 factors are accurate entry by
// entry however wide the spread of theta.  A component's last node gets an exact zero pivot and
// becomes +infinity (grounded), as Section 4.2 prescribes for the singular pivots.
#pragma once

#include "common.cuh"
#include "newton.cuh"
#include "support.cuh"

namespace ot {

struct Dense32 {
    int32_t n = 0, ld = 0;       // ld: column stride (n rounded up to a multiple of 32)
    float *A = nullptr;          // ld x n column-major; strictly lower part: S_M, then L
    float *X = nullptr;          // ld x n; lower part with the unit diagonal: L^-1
    float *LD = nullptr;         // 3 x ld x 64 panel scratch (L21 D1), panels in turn
    float *L0 = nullptr;         // 64 x 64: the next panel's rows of L21, until the next diagonal kernel stores them
    float *Linv = nullptr;       // ld x 64: inverse diagonal blocks, block k in rows k..k+63
    float *D = nullptr;          // n pivots (+inf: grounded)
    float *d0 = nullptr;         // n diagonal entries of S_M (the reference of the pivot rule)
    float *csum = nullptr;       // partial sums of the next panel's columns below its diagonal block
    float *w = nullptr;          // n
    float *part = nullptr;       // (n / 64) x ld partial sums of the forward product
    float eps = 0.f;
    cudaGraphExec_t graph = nullptr;  // the factorisation's launch sequence for this n
    int64_t graph_nodes = 0;
    // bulk update on the tensor cores (split TF32, tcgen05): tc_mode 1 = on, -1 = the FP32 SIMT
    // update, 0 = on from n = 8192 (read when the launch sequence is built); split operands,
    // double-buffered by panel
    int tc_mode = 0;
    bool use_tc = false;
    float *tc = nullptr;
    int *tc_err = nullptr;      // a bounded wait of the tensor-core update gave up (device)
    int *tc_err_host = nullptr; // pinned copy, read at the next factorisation
};

Error d32_alloc(Dense32 &F, int32_t n);
void d32_free(Dense32 &F);

// Strictly lower part of S_M (from theta, M^-1 and N of the Newton workspace) into F.A, and the
// diagonal into F.d0.  Off-diagonal sums are accumulated in 64-bit fixed point (scaled by the
// column's N_j), so the result does not depend on the order of the atomic additions.
Error d32_assemble(Dense32 &F, const Newton &W, const Support &S, cudaStream_t st);

// F.A <- L (unit, strictly lower), F.D <- D, F.X <- L^-1; pivots d <= eps * d0 become +infinity.
// The launch sequence (five kernels per 64-column panel) is captured once into a CUDA graph.
Error d32_factor(Dense32 &F, float eps, cudaStream_t st);

// z = L^-T D^+ L^-1 r: two triangular matrix-vector products with L^-1 (FP32 arithmetic, FP64
// vectors in and out; r and z distinct device vectors of length n).
Error d32_apply(Dense32 &F, const double *r, double *z, cudaStream_t st);

}  // namespace ot
