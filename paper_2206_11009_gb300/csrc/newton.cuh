// Newton direction through the Schur complement S_M of the normal equations (Sections 3-4).
#pragma once

#include "common.cuh"
#include "support.cuh"

namespace ot {

// Device scalars written by reductions (indices into Newton::scal).
enum Scalar : int {
    SC_R1A_SQ = 0, SC_R1A_L1, SC_R1B_SQ, SC_R1B_L1, SC_R2SQ, SC_PS, SC_CP, SC_CSQ, SC_CMAX,
    SC_AP, SC_AS,            // raw minimum ratios -x/dx over dx < 0 (+inf when none)
    SC_MUAFF, SC_PSNEW, SC_SUM_A, SC_SUM_B, SC_NORM_A, SC_NORM_B, SC_ONECOMP,
    SC_PCG_ITERS, SC_PCG_RELRES,
    SC_RZ0, SC_RZ1,          // ping-pong r.z of the refinement CG (alpha, beta formed on the device)
    SC_COUNT
};

// Per-iteration device work arrays (allocated by the solver, sized by capacity).
struct Newton {
    int32_t m = 0, n = 0;
    int64_t cap = 0;
    int num_sms = 0;
    // entry arrays (CSR order)
    double *c = nullptr, *theta = nullptr, *excl = nullptr, *r2 = nullptr, *r3 = nullptr, *g = nullptr;
    double *dp = nullptr, *ds = nullptr, *dp2 = nullptr, *ds2 = nullptr, *dp3 = nullptr, *ds3 = nullptr;
    float *theta32 = nullptr;
    double *theta_col = nullptr;
    float *theta32_col = nullptr;
    uint8_t *flag = nullptr;
    // rows (m)
    double *r1a = nullptr, *beta1 = nullptr, *M = nullptr, *Minv = nullptr, *du = nullptr, *du2 = nullptr,
           *du3 = nullptr, *w64 = nullptr;
    float *Minv32 = nullptr, *w32 = nullptr;
    // cols (n)
    double *r1b = nullptr, *beta2 = nullptr, *N = nullptr, *Dinv = nullptr, *Sdiag = nullptr, *rhs = nullptr,
           *dv = nullptr,
           *dv2 = nullptr, *dv3 = nullptr, *res64 = nullptr, *y64 = nullptr;
    double *x64 = nullptr, *r64 = nullptr, *z64 = nullptr, *p64 = nullptr, *q64 = nullptr;
    float *Dinv32 = nullptr, *b32 = nullptr, *x32 = nullptr, *r32 = nullptr, *z32 = nullptr, *p32 = nullptr,
          *q32 = nullptr;
    // components (m + n nodes)
    int32_t *parent = nullptr;
    double *comp_sum = nullptr, *comp_cnt = nullptr;
    // reductions
    double *part = nullptr;  // [16][kMaxPartBlocks]
    double *scal = nullptr;  // [SC_COUNT]
    double *hscal = nullptr; // [2][SC_COUNT] pinned host copies
    cudaEvent_t ev_scal = nullptr, ev_scal2[2] = {nullptr, nullptr};
    unsigned *bar = nullptr;
    int *err = nullptr;
    int pcg_grid = 0;
    bool onecomp = true;       // the support graph is connected (set by schur_setup)
    int verbose = 0;           // >= 3: one line per PCG launch (support size, iterations, device ms)
    double last_pcg_ms = 0.0;
    double *pcg_pb = nullptr;     // second direction buffer of the PCG (fp64 / fp32)
    float *pcg_pb32 = nullptr;
    int *pcg_bnd = nullptr;       // grid PCG: first row (then first column) of each lane group
    int64_t pcg_bnd_cap = 0;      // entries per half of pcg_bnd
    double pcg_bytes_per_iter = 0.0;
    int pcg_cluster = 0;       // CTAs of the FP32 cluster PCG (0: not available on this device)
    int pcg_cluster_smem = 0;  // dynamic shared memory of one of its CTAs
    // direct branch: when set, S_M x = rhs is solved by its LDL^T factorisation (chol.cuh)
    struct Chol *direct = nullptr;
    struct DenseLDL *dense = nullptr;   // when set (with direct), solve with the dense factor
    // when set (and direct is not): FP64 CG preconditioned by the FP32 dense factorisation
    struct Dense32 *d32 = nullptr;
    // when set (and neither of the above): FP64 CG preconditioned by the incomplete Cholesky factor
    // (ic.cuh), stopped at the CG tolerance of the solve
    struct IncChol *ic = nullptr;
    // when set: the support is a forest and the Newton system is solved exactly on the tree
    // (tree.cuh); takes precedence over every other solver
    struct TreeSolver *tree = nullptr;
    int fallbacks = 0;        // mixed-precision solves redone in FP64
    double direct_cg_tol = 0.0;  // > 0: target of the factor-preconditioned CG (else min(tol, 1e-10))
    bool fp64_fallback = true;  // redo a failed mixed-precision solve with FP64 PCG
};

constexpr int kMaxPartBlocks = 2048;

Error newton_alloc(Newton &W, int32_t m, int32_t n, int64_t cap, int num_sms);
Error newton_grow(Newton &W, int64_t cap);
void newton_free(Newton &W);

// Costs of the support pairs into W.c.
Error support_costs(Newton &W, const CostDev &cd, const Support &S, cudaStream_t st);

// r1 = f - A p, r2 = c - A^T y - s, and the sums behind mu, norms and c^T p (eq. redsystem).
Error residuals(Newton &W, const Support &S, const double *a_s, const double *b_s, const double *u,
                const double *v, cudaStream_t st);

// theta = p/s, M, N, M^-1, Jacobi diagonal of S_M (cancellation-free), column-order copies;
// connected components of the support graph.
Error schur_setup(Newton &W, const Support &S, cudaStream_t st);

// Number of connected components of the support graph, from the labels schur_setup left in
// W.parent (one host read).
Error support_components(Newton &W, int64_t *ncomp, cudaStream_t st);

// *one = whether the support graph is connected (every row has a pair; columns are compared).
Error support_connected(Newton &W, const Support &S, bool *one, cudaStream_t st);

// Which right-hand side pieces to use in newton_solve.
struct Rhs {
    const double *r1a, *r1b, *r2, *r3;  // nullptr = zero
};

struct SolveStats {
    int cg_iters = 0;
    double relres = 0.0;
    int refinements = 0;
    int direct = 0;
};

// Direction (du, dv, ds, dp) of eq. normalequationsipm for the given right-hand sides.
// precision 0: FP64 PCG; 1: FP32 PCG inside FP64 iterative refinement.
Error newton_solve(Newton &W, const Support &S, const Rhs &rhs, double cg_tol, int max_cg, int precision,
                   double *du, double *dv, double *ds, double *dp, SolveStats *stats, cudaStream_t st);

// Minimum ratios -p/dp (dp < 0) and -s/ds (ds < 0) into scal[SC_AP], scal[SC_AS]; the step
// lengths are min(1, scale * ratio) (the scale is applied by the caller).
Error step_lengths(Newton &W, const Support &S, const double *dp, const double *ds, double scale,
                   cudaStream_t st);

// scal[SC_MUAFF] = sum (p + ap dp)(s + as ds)
Error trial_complementarity(Newton &W, const Support &S, const double *dp, const double *ds, double ap,
                            double as, cudaStream_t st);

// r3 = sigma mu - p s - dpa dsa   (Mehrotra corrector)
Error corrector_r3(Newton &W, const Support &S, double sigma_mu, const double *dpa, const double *dsa,
                   cudaStream_t st);

// Gondzio centrality corrector target: r3 = clip(v, lo, hi) - v, floored at -hi,
// v = (p + tp dp)(s + ts ds)
Error centrality_r3(Newton &W, const Support &S, const double *dp, const double *ds, double tp, double ts,
                    double lo, double hi, cudaStream_t st);

// x += y on the direction arrays (entries psi, rows m, cols n)
Error add_direction(Newton &W, const Support &S, double *dp, double *ds, double *du, double *dv,
                    const double *dp2, const double *ds2, const double *du2, const double *dv2, cudaStream_t st);

// p += ap dp, s += as ds, u += as du, v += as dv; scal[SC_PSNEW] = p^T s
Error take_step(Newton &W, Support &S, double *u, double *v, const double *dp, const double *ds,
                const double *du, const double *dv, double ap, double as, cudaStream_t st);

// Mehrotra's starting point on the restricted problem (Theta = I): writes S.p, S.s, u, v.
Error mehrotra_start(Newton &W, Support &S, const double *a_s, const double *b_s, double *u, double *v,
                     int precision, double cg_tol, int max_cg, int *cg_iters, cudaStream_t st,
                     bool warm_duals = false);

// Read the scalars back (synchronises the stream).
Error read_scalars(Newton &W, double *host, cudaStream_t st);

}  // namespace ot
