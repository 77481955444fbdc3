/*
 * ot_ipm.h -- C ABI of the GB300 (sm_103a) hybrid interior-point / column-generation solver
 * for the Kantorovich optimal-transport linear program.
 *
 * Method: Zanetti & Gondzio, "An Interior-Point-Inspired algorithm for Linear Programs arising
 * in Discrete Optimal Transport" (arXiv:2206.11009).  Section numbers below refer to it.
 *
 * Conventions shared by every entry point
 *   - Return value: an ot_status code; OT_OK == 0.  On failure the handle (when there is one)
 *     keeps a message readable with ot_ipm_last_error(); nothing is left half-written in the
 *     caller's output buffers except where stated.
 *   - Ownership: the caller owns every pointer it passes; the library copies what it needs and
 *     never keeps or frees a caller pointer.  A handle owns all device memory it allocates and
 *     releases it in ot_ipm_destroy().
 *   - Indices are 0-based.  Source i in [0, m), target j in [0, n).  The column of the LP
 *     that carries the flow p_ij is jlin = i + j*m (column-major vec(P), Section 2.1).
 *   - Masses a, b: nonnegative doubles with sum(a) == sum(b) up to a relative 1e-12 (b is then
 *     rescaled by sum(a)/sum(b)); otherwise OT_ERR_ARG.
 *   - Device pointers (the ot_price_* / ot_ipm_*_dev entry points) must live on the current
 *     CUDA device; `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   - Host-buffer entry points synchronise the handle's stream before returning.
 */
#ifndef OT_IPM_H
#define OT_IPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OT_OK = 0,
    OT_ERR_ARG = 1,           /* invalid argument (sizes, masses, null pointers, options)     */
    OT_ERR_CUDA = 2,          /* a CUDA runtime call failed                                   */
    OT_ERR_OOM = 3,           /* device allocation failed                                      */
    OT_ERR_MAXITER = 4,       /* iteration limit reached before the stopping test held        */
    OT_ERR_NUMERIC = 5,       /* NaN/Inf or breakdown in mu, step length or a linear solve    */
    OT_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up (grid barrier)            */
    OT_ERR_BUF_TOO_SMALL = 7, /* caller buffer too small; the needed size is still returned   */
    OT_ERR_UNSUPPORTED = 8    /* valid request this build does not implement                  */
} ot_status;

/* Cost c_ij between source point i and target point j (Section 5.1 lists the L1, Euclidean
 * and L-infinity pixel distances; the squared Euclidean distance is the default here). */
typedef enum {
    OT_COST_SQEUCLID = 0,     /* (dx)^2 + (dy)^2, computed on the fly, never stored           */
    OT_COST_EUCLID = 1,       /* sqrt(dx^2 + dy^2)                                            */
    OT_COST_L1 = 2,           /* |dx| + |dy|                                                  */
    OT_COST_LINF = 3,         /* max(|dx|, |dy|)                                              */
    OT_COST_DENSE = 4         /* explicit matrix C (tests and small problems)                 */
} ot_cost_kind;

/* Problem statement (Section 2: a in R^m_+, b in R^n_+, cost matrix C in R^{m x n}_+).
 * The pointers are HOST pointers unless inputs_on_device is set, in which case every one of them
 * (a, b, the coordinates, C) is a device pointer on the current device.  ot_ipm_create copies
 * what it needs and keeps no caller pointer.
 *
 * Zero masses (input handling; the paper does not discuss them): a source i with a_i = 0 or a
 * target j with b_j = 0 carries no flow in any feasible coupling, so it is removed before the
 * solve (presolve).  Every entry point below still speaks in the caller's indices: couplings are
 * reported on the original (i, j), and ot_ipm_get_solution completes the duals of removed points
 * by the c-transform (u_i = min_j c_ij - v_j over the kept targets, then v_j = min_i c_ij - u_i
 * over all sources), which keeps (u, v) dual feasible wherever the solve's duals are. */
typedef struct {
    int32_t m, n;
    const double *a;          /* m source masses                                              */
    const double *b;          /* n target masses                                              */
    int32_t cost;             /* ot_cost_kind                                                 */
    /* point coordinates for the distance kinds: integers with |x|,|y| < 2^14.  When all four
     * are NULL the points are pixel grids: source i sits at (i mod src_w, i div src_w), target j
     * at (j mod dst_w, j div dst_w) (m = src_w*src_h, n = dst_w*dst_h). */
    const int32_t *src_x, *src_y, *dst_x, *dst_y;
    int32_t src_w, dst_w;
    const double *C;          /* OT_COST_DENSE only: m x n row-major, C[i*n + j], finite, >= 0,  */
                              /* m*n <= 2^30                                                  */
    int32_t inputs_on_device; /* 0: host pointers; 1: device pointers (see above)             */
} ot_problem;

typedef struct {
    double tol;               /* 1e-6: feasibility and optimality tolerance (Section 5.2)     */
    double feas_l1;           /* 1e-8: ||f - A p||_1 bound in the caller's mass units         */
    double cg_tol_pred;       /* 1e-6: PCG relative residual for predictors (Section 5.2)     */
    double cg_tol_corr;       /* 1e-3: PCG relative residual for correctors (Section 5.2)     */
    int32_t max_iter;         /* 200 (Section 5.2)                                            */
    int32_t max_cg;           /* 1000 CG iterations per call (Section 5.2)                    */
    int32_t max_corr;         /* 3 centrality correctors (Section 5.2)                        */
    double step_scale;        /* 0.995 (Section 3.3)                                          */
    int32_t precision;        /* 0: plain FP64 everywhere; 1: FP32 scan + FP64 recheck and    */
                              /*    FP32 PCG + FP64 iterative refinement                      */
    int32_t linear_solver;    /* 0: PCG then switch to the sparse LDL^T (Section 4.2-4.3)     */
                              /* 1: PCG only; 2: LDL^T only                                  */
    double init_cost;         /* 2.0: initial support {c_ij <= init_cost} (Section 3.2 end)   */
    double rm_mu_frac;        /* 1e-3: removal phase once mu <= rm_mu_frac * mu_0             */
    double rm_p_frac;         /* 1e-3: remove when p < rm_p_frac*min(a_i,b_j) and theta < 1   */
    int32_t add_max;          /* 0 = m: pairs added per pricing (end of Section 3.2)          */
    int32_t verbose;          /* 0: silent; 1: one line per iteration on stderr               */
    void *stream;             /* cudaStream_t to run on; NULL = a stream the handle creates   */
    /* Warm start (not in the paper; its conclusion names a better starting support as future
     * work).  warm_u (m) and warm_v (n): predicted duals, HOST pointers, the caller's cost units;
     * NULL (either) = cold start.  The initial support then also holds the warm_count pairs
     * outside {c_ij <= init_cost} with the least c_ij - u_i - v_j below init_cost, selected by
     * the pricing scan (ties by jlin); 0 = 2(m+n).  warm_mode 0: only the support is warm (the
     * starting point is Mehrotra's, computed on it); 1: the starting point also takes warm_u,
     * warm_v as its duals, with slacks max(c_ij - u_i - v_j, 0) before Mehrotra's balancing. */
    const double *warm_u;
    const double *warm_v;
    int32_t warm_count;
    int32_t warm_mode;
    /* Warm start by explicit pairs: warm_i, warm_j (HOST, warm_npairs entries, any order,
     * duplicates allowed) join the cold support; pairs already in it are skipped.  Used with or
     * without warm_u / warm_v (their pairs are added first). */
    const int32_t *warm_i;
    const int32_t *warm_j;
    int64_t warm_npairs;
    /* New pairs from pricing start at p = s = sqrt(mu) (Section 3.2): new_col_rule 0.  1: p =
     * min(sqrt(mu), a_i, b_j) and s = mu / p (still p s = mu, but a pair never enters with more
     * flow than its smaller mass; masses in the solver's scaling, sum(a) = m). */
    int32_t new_col_rule;
    /* Launch shapes (chosen by the autotuner; 0 = the library's rule).  scan_rows: source rows
     * per pricing-scan tile, 8..256.  dense32_max_n: largest n for which the mixed-precision
     * path preconditions every iteration with the FP32 dense factorisation (0 = 8192; at most
     * 65536, where its two n x n factors take 2 x 4 n^2 bytes = 34 GB; -1: never). */
    int32_t scan_rows;
    int32_t dense32_max_n;
    /* Largest n for which the direct branch factors S_M densely in FP64 (at most 8192; 0 = 8192,
     * -1: never, the sparse LDL^T of Section 4.2 instead). */
    int32_t dense_max_n;
    /* Heuristic pricing set of Section 3.4: jset_cmax > 0 prices only the pairs of
     * J = {(i, j) : c_ij < jset_cmax} (listed once, on the first such iteration), except on every
     * jset_refresh-th iteration (iterations jset_refresh-1, 2*jset_refresh-1, ...), which prices all
     * m*n pairs; 0 = 3 (the paper refreshes every 3 or 4 iterations).  jset_cmax <= 0: every
     * iteration prices all pairs.  The stopping test's certificate always covers all pairs. */
    double jset_cmax;
    int32_t jset_refresh;
    /* Multiscale warm start (not in the paper; its conclusion names a better starting support as
     * future work): multiscale = L > 0 first solves the problem coarsened by binning the points
     * into 2 x 2 cells (cell masses summed), itself with L - 1 coarser levels, to relative
     * tolerance ms_tol (0 = max(tol, 1e-4); also the coarse ||f - A p||_1 bound relative to the
     * total mass); its duals, interpolated bilinearly at the points and
     * scaled by the cost's degree (x4 for the squared distance, x2 for the others), are used as
     * warm_u, warm_v (warm_count 0 then means 10(m+n), warm_mode as given).  Skipped for explicit
     * cost matrices, for caller-given warm_u / warm_v, and below 256 points per side.  Runs inside
     * ot_ipm_create (ot_result.create_seconds). */
    int32_t multiscale;
    double ms_tol;
    /* Preconditioner of the iterative phase (Section 4.2).  0: the library's choice (mixed
     * precision: the FP32 dense factorisation for n <= 8192, Jacobi PCG otherwise; FP64: Jacobi
     * PCG).  1: incomplete Cholesky with a drop tolerance -- the factor keeps S_M's pattern in a
     * multicolour order (every colour's rows in parallel), drops l_rs when |l_rs d_s| <
     * tau sqrt(S_rr S_ss) and grounds pivots d_r <= 1e-12 S_rr -- preconditioning an FP64 CG to the
     * PCG tolerance; tau starts at ic_tau (0 = 1e-2) and is divided by 10 (down to 1e-6) after an
     * iteration whose solves needed more than 200 CG iterations.  The switch to the direct branch
     * (Section 4.3) is unchanged. */
    int32_t precond;
    double ic_tau;
    /* Bulk update of the FP32 dense factorisation: 1 = on the tensor cores (tcgen05 MMAs in split
     * TF32, a = a_hi + a_lo, three products per term, FP32 accumulation in tensor memory: FP32
     * accuracy; operands pre-split per panel, fetched by bulk copies; persistent warp-specialised
     * CTAs with two accumulators), -1 = the FP32 SIMT update with the fused panel step, 0 = the
     * tensor cores from n = 8192 on, SIMT below (the default; measured per factorisation:
     * n = 16384 75 ms against 93 ms, n = 4096 2.9 ms either way). */
    int32_t tc_update;
    /* Relative residual at which the CG preconditioned by a factorisation (the FP32 dense factor,
     * the direct branch) stops: 0 = min(CG tolerance, 1e-10) (near-exact Newton directions);
     * > 0: max(direct_cg_tol, min(CG tolerance, 1e-10)). */
    double direct_cg_tol;
} ot_options;

/* One outer iteration (Section 3.4's commented listing). */
typedef struct {
    int32_t iter;             /* iteration index                                              */
    int64_t psi;              /* support size before the support update                       */
    double mu;                /* p^T s / psi before the step                                  */
    double crit;              /* stopping measure before the step                             */
    double alpha_p, alpha_s;  /* step lengths taken                                           */
    double sigma;             /* centring parameter                                           */
    int32_t ncorr;            /* centrality correctors accepted                               */
    int32_t cg_iters;         /* CG iterations in this iteration (all solves)                 */
    int32_t direct;           /* 1 if the Newton systems were solved by LDL^T                 */
    int64_t added, removed;   /* support changes                                              */
    int32_t done;             /* 1 when the stopping test held (no step was taken)            */
} ot_iter_info;

typedef struct {
    int32_t status;           /* ot_status of the solve                                       */
    double obj;               /* c^T p (caller's units)                                       */
    double lower_bound;       /* c-transform bound a^T u~ + b^T v <= OPT (caller's units)     */
    double rel_gap;           /* (obj - lower_bound) / (1 + |obj|)                            */
    double r1_l1;             /* ||f - A p||_1 (caller's units)                               */
    double mu;
    int32_t iters, cg_iters, direct_iters;
    int64_t psi;              /* final support size                                           */
    double max_fill;          /* max nnz(L)/n^2 * 100 over direct iterations (Table 3's fill)  */
    double seconds;           /* device time of the solve (CUDA events)                       */
    int64_t warm_added;       /* pairs the warm start added to the initial support            */
    int32_t warm_restarts;    /* 1 when a warm start lost ground (mu over twice its first value */
                              /* by iteration 5) and the solve restarted from the cold support */
    double create_seconds;    /* wall time of ot_ipm_create (initial support, starting point,    */
                              /* coarse solves of the multiscale warm start), synchronised      */
    int32_t ms_levels;        /* coarse levels solved by the multiscale warm start              */
} ot_result;

typedef struct ot_ipm ot_ipm_t;

/* Fill *opt with the paper's defaults (Section 5.2) and this library's readings. */
void ot_options_default(ot_options *opt);

/* Validate and copy the problem to the device, presolve zero masses, build the initial support
 * (Section 3.2 end) and the initial point.  On success *out owns all device state.  Errors:
 * OT_ERR_ARG (sizes, masses, coordinates, a negative or non-finite C), OT_ERR_OOM, OT_ERR_CUDA. */
int ot_ipm_create(const ot_problem *prob, const ot_options *opt, ot_ipm_t **out);

/* One outer iteration: residuals, stopping test, predictor-corrector Newton direction,
 * step, pricing, support update (Section 3.4's listing).  info may be NULL.  Returns OT_OK
 * (info->done tells whether the stopping test held), or an error status. */
int ot_ipm_step(ot_ipm_t *h, ot_iter_info *info);

/* Iterate to the stopping test (or max_iter) and fill *res (may be NULL). */
int ot_ipm_solve(ot_ipm_t *h, ot_result *res);

/* Solve `count` independent instances (handles from ot_ipm_create, each with its own stream)
 * with `workers` host threads (0 = 2) drawing from one queue, largest instance (m * n) first.
 * res[i] receives instance i's result and status.  Returns OT_OK when every instance
 * succeeded, else the first failing status.  Handles must be distinct and must not be used by
 * other threads meanwhile. */
int ot_ipm_solve_batch(ot_ipm_t *const *handles, int32_t count, ot_result *res, int32_t workers);

/* Copy the current coupling (support pairs and their flows, caller's units) and the duals u, v
 * into caller HOST buffers of capacity cap.  *nnz receives the support size even when cap is
 * too small (then OT_ERR_BUF_TOO_SMALL and nothing else is written).  u (m), v (n) may be NULL. */
int ot_ipm_get_solution(ot_ipm_t *h, int32_t *i, int32_t *j, double *p, int64_t cap,
                        int64_t *nnz, double *u, double *v);

/* Full iterate in the solver's internal scaling (masses scaled by m'/sum(a), m' the number of
 * sources with positive mass): support pairs sorted by (i, j), p, s, and u, v (entries of points
 * removed by the presolve are 0).  Same buffer rules as ot_ipm_get_solution.  Used for
 * checkpoints and to compare single steps with a reference. */
int ot_ipm_get_state(ot_ipm_t *h, int32_t *i, int32_t *j, double *p, double *s, int64_t cap,
                     int64_t *psi, double *u, double *v);

/* Replace the iterate (host buffers, internal scaling).  Pairs must be distinct, in range,
 * sorted by (i, j) and free of points removed by the presolve; p, s > 0 (u, v entries of removed
 * points are ignored).  Resets the iteration counter's mu_0 reference only if reset_mu0 != 0. */
int ot_ipm_set_state(ot_ipm_t *h, const int32_t *i, const int32_t *j, const double *p,
                     const double *s, int64_t psi, const double *u, const double *v,
                     int32_t reset_mu0);


/* Linear solvers of the Newton system (ot_ipm_newton_direction). */
enum {
    OT_LS_PCG64 = 0,    /* Jacobi PCG in FP64 (Section 4.2, matrix-free S_M)                      */
    OT_LS_MIXED = 1,    /* Jacobi PCG in FP32 inside FP64 iterative refinement                     */
    OT_LS_DENSE32 = 2,  /* FP64 CG preconditioned by the FP32 dense LDL^T of S_M (n <= 16384)      */
    OT_LS_DENSE64 = 3,  /* FP64 dense LDL^T with the infinite-pivot rule (Section 4.3, n <= 8192)  */
    OT_LS_SPARSE = 4,   /* FP64 sparse LDL^T, fill-reducing order, no dropping (Section 4.3)       */
    OT_LS_IC = 5,       /* FP64 CG preconditioned by the incomplete Cholesky factor, drop tolerance */
                        /* 1e-2 (Section 4.2; ot_options.precond 1)                                 */
    OT_LS_TREE = 6      /* exact solve on a forest support (Section 4.3, Theorem 2): the normal     */
                        /* equations as a tree Laplacian, by the Euler-tour technique; used         */
                        /* automatically whenever the support is a forest (linear_solver != 1);     */
                        /* OT_ERR_UNSUPPORTED when the support has a cycle                           */
};

/* The predictor direction (du, dv, dp, ds) of the normal equations (Section 3, eq. redsystem with
 * r3 = -P S e; Schur complement S_M of Section 4) at the handle's current iterate -- after
 * ot_ipm_set_state or any step -- computed with the chosen linear solver.  Iterative solvers stop
 * at ||S_M dv - rhs|| <= cg_tol ||rhs|| or after max_cg iterations; the direct ones refine with
 * FP64 CG to the same tolerance.  dv is returned with mean zero on every connected component of
 * the support graph.  Outputs are HOST buffers owned by the caller (any may be NULL): du (m),
 * dv (n), dp and ds (cap >= the support size, entries in ot_ipm_get_state order).  The iterate
 * and the support are not changed.  Errors: OT_ERR_ARG, OT_ERR_BUF_TOO_SMALL, OT_ERR_UNSUPPORTED
 * (n above the dense factor's limit, sparse fill over budget), OT_ERR_CUDA, OT_ERR_TIMEOUT. */
int ot_ipm_newton_direction(ot_ipm_t *h, int32_t solver, double cg_tol, int32_t max_cg, double *du, double *dv,
                            double *dp, double *ds, int64_t cap, int32_t *cg_iters);

/* The incomplete Cholesky preconditioner (Section 4.2; the factor of ot_options.precond 1, see
 * there) of S_M at the handle's current iterate, with drop tolerance tau >= 0, applied to b:
 * x = L^-T D^-1 L^-1 b (grounded pivots contribute 0).  b and x are HOST buffers of n entries in
 * the caller's target indexing (entries of targets removed by the presolve: ignored / 0).  The
 * iterate is not changed.  The parity hook of the factor.  Errors: OT_ERR_ARG, OT_ERR_CUDA. */
int ot_ipm_ic_apply(ot_ipm_t *h, double tau, const double *b, double *x);

/* Internal scale factor sigma_f = m / sum(a) (masses are multiplied by it). */
double ot_ipm_mass_scale(const ot_ipm_t *h);

/* Release everything the handle owns.  NULL is accepted. */
void ot_ipm_destroy(ot_ipm_t *h);

/* Message of the last failure on this handle ("" if none).  Valid until the next call. */
const char *ot_ipm_last_error(const ot_ipm_t *h);

/* Message of the last failure of a handle-less entry point on the calling thread. */
const char *ot_last_error(void);

/* ---------------------------------------------------------------------------------------
 * Pricing (Section 3.4, with the support enlargement of Section 3.2) on device buffers.
 *
 * Computes d_ij = c_ij - u_i - v_j for ALL m*n pairs of a squared-Euclidean point set, costs
 * evaluated on the fly from integer coordinates, and selects the pairs outside the support
 * with d_ij < 0, at most kmax of them, smallest first.  The selected SET is exactly the one of
 * this rule: d_ij = (c_ij - u_i) - v_j in IEEE float64 round-to-nearest in that order (no
 * fusion); order by (d_ij, jlin = i + j*m) ascending; keep the first min(kmax, #candidates).
 * precision 1 scans in FP32 and rechecks every pair inside a proven error window in FP64;
 * precision 0 scans in FP64.  Both return the same set.
 *
 *   sx, sy (m) / tx, ty (n): int32 coordinates, |value| < 2^14      (device)
 *   u (m), v (n): float64 duals                                      (device)
 *   sup_i, sup_j (psi): support pairs sorted by (i, j), distinct     (device, may be NULL if psi==0)
 *   out_i, out_j, out_d (kmax): selected pairs in (d, jlin) order    (device, caller-owned)
 *   out_count: number selected (device int32)
 * Scratch is allocated from the stream-ordered pool and released before return.
 * Errors: OT_ERR_ARG (sizes, m*n > 2^32, null pointers), OT_ERR_OOM, OT_ERR_CUDA.
 * ------------------------------------------------------------------------------------- */
int ot_price_topk(int32_t m, int32_t n, const int32_t *sx, const int32_t *sy,
                  const int32_t *tx, const int32_t *ty, const double *u, const double *v,
                  const int32_t *sup_i, const int32_t *sup_j, int64_t psi, int32_t kmax,
                  int32_t precision, int32_t *out_i, int32_t *out_j, double *out_d,
                  int32_t *out_count, void *stream);

/* Options of ot_price_topk_ex (zero-initialise, then set what differs). */
typedef struct {
    int32_t cost;        /* ot_cost_kind; the distance kinds use the coordinates (Section 5.1),    */
                         /* OT_COST_DENSE uses C (and always scans in FP64)                         */
    int32_t scan_rows;   /* 0: the library's rule; else 8..256 source rows per scan tile            */
    double jset_cmax;    /* > 0: only the pairs with c_ij < jset_cmax are priced (the set J of       */
                         /* Section 3.4, listed inside the call); <= 0: all m*n pairs                 */
    const double *C;     /* OT_COST_DENSE: m x n row-major costs (device); NULL otherwise           */
} ot_price_opts;

/* ot_price_topk for any cost kind, with an explicit scan tile height and the heuristic set J.
 * The selection rule is the same with c_ij the chosen cost: d_ij = (c_ij - u_i) - v_j in IEEE
 * float64 (the Euclidean distance is the correctly rounded square root of the integer dx^2 + dy^2),
 * candidates outside the support with d_ij < 0 (and, with jset_cmax > 0, c_ij < jset_cmax), order
 * (d_ij, jlin), first min(kmax, #candidates).  precision 1 scans the distance kinds in FP32 with a
 * proven error window and rechecks in FP64.  opts may be NULL (squared cost, full scan).  The
 * coordinates may be NULL for OT_COST_DENSE.  Errors as ot_price_topk. */
int ot_price_topk_ex(int32_t m, int32_t n, const int32_t *sx, const int32_t *sy,
                     const int32_t *tx, const int32_t *ty, const double *u, const double *v,
                     const int32_t *sup_i, const int32_t *sup_j, int64_t psi, int32_t kmax,
                     int32_t precision, int32_t *out_i, int32_t *out_j, double *out_d,
                     int32_t *out_count, const ot_price_opts *opts, void *stream);

/* ot_price_topk without any device allocation.  The paper has no counterpart: this exists for
 * callers that cannot allocate device memory while they run -- for example a serving process
 * that reserved its whole memory budget at start-up, where a further cudaMalloc would fail or
 * evict its caches, or a loop that must not pay the implicit device-wide synchronisation an
 * allocation or release can cause.
 *
 * Same arguments, outputs and selection as ot_price_topk.  All temporary buffers come from one
 * fixed 24 MiB array in device memory, declared statically in the library.  The array belongs to
 * the library's device module, which CUDA loads on a device when it is first needed (lazy
 * loading): in practice at the first call of this function on that device, which can then fail
 * with OT_ERR_CUDA if the device has no 24 MiB left.  A caller that reserves its memory budget at
 * start-up should therefore make one call on every device it uses before it reserves; from then
 * on the device holds those 24 MiB until the process exits.  Every call looks up the array's
 * device address (with the calling thread's current device); make the first call on a device
 * before any stream capture.  Limits: m, n <= 16384, and the candidate set the selection has to
 * recheck must fit the array (about 400k pairs); beyond either limit the call returns OT_ERR_ARG
 * or OT_ERR_BUF_TOO_SMALL with a message (ot_last_error) and changes no output.  Every call on a
 * device uses the same array and leaves its contents behind (each call clears what it needs), so
 * calls that overlap on the GPU -- on two streams, or from two threads -- race and must be
 * serialised by the caller.  The call synchronises its stream twice (to size the candidate set)
 * before it returns.  No cudaMalloc, cudaFree or allocating library routine is called. */
int ot_price_topk_noalloc(int32_t m, int32_t n, const int32_t *sx, const int32_t *sy,
                          const int32_t *tx, const int32_t *ty, const double *u, const double *v,
                          const int32_t *sup_i, const int32_t *sup_j, int64_t psi, int32_t kmax,
                          int32_t precision, int32_t *out_i, int32_t *out_j, double *out_d,
                          int32_t *out_count, void *stream);

/* Number of kernels this library launched since load (for launch accounting). */
int64_t ot_kernel_launches(void);

/* Opt-in timing of the library's main kernels with CUDA events recorded on the stream each one
 * is launched on.  enable(1) clears the totals and starts recording; read() resolves the events
 * (synchronising on them) and writes, per kernel id, the total milliseconds, the launch count and
 * (work != NULL) the algorithmic work of those launches: FP32 operations for the pricing scan
 * (4 per pair for the squared cost, 6 for L1 / L-infinity, 8 for the Euclidean distance; pairs
 * of the J list only when it is used), bytes for the PCG (per CG iteration: theta, index and
 * gathered vector entry per support pair in both passes, plus the row/column vectors), FP64 flops
 * for the LDL^T numeric factorisation (n^3/3 when dense), bytes for the LDL^T solves (L read
 * twice), FP32 flops for the FP32 dense factorisation with its inverse factor (n^3/3 + n^3/3) and
 * bytes for its application (the triangle of L^-1 read twice), and bytes for the FP64 CG that
 * refines a factor-preconditioned solve (per iteration: theta, index and gathered vector entry
 * per support pair in the row and the column pass, the per-row and per-column vectors, the
 * step's update of x and r, and -- with the FP32 dense factor, whose CG runs as one persistent
 * launch that includes the factor's application -- the triangle of L^-1 read twice):
 *   0 pricing scan (histogram pass)   1 pricing scan (gather pass)   2 FP64 recheck
 *   3 PCG FP64 (persistent kernel)    4 PCG FP32                     5 LDL^T numeric (FP64)
 *   6 LDL^T solve (FP64)              7 FP32 dense LDL^T + L^-1      8 FP32 dense apply
 *   9 FP64 refinement CG operator (S_M p and the step)
 * cap >= 10.  Returns the number of ids written, or OT_ERR_ARG.  Not thread-safe. */
void ot_kernel_timing_enable(int32_t on);
int ot_kernel_timing_read(double *ms, int64_t *count, double *work, int32_t cap);

/* ---- Warm-start network (not in the paper; its conclusion names a better starting support as
 * future work).  A convolutional network maps the two marginals of a k x k image pair to predicted
 * dual potentials, which ot_options.warm_u / warm_v turn into extra initial pairs:
 *   input  x (B, 2, k, k): log(a m / sum a), log(b m / sum b), NCHW, FP32
 *   blocks l = 0..3: h <- silu(rmsnorm_c(conv3x3(h; W_l, b_l, dilation 2^l)) * g_l), 2->32->32->32->32
 *   head:  y = conv3x3(h; W_4, b_4), 32 -> 2: the predicted (u, v) / k^2
 * Convolutions take BF16 operands and accumulate in FP32; those of the three 32 -> 32 blocks
 * (forward, data gradient, weight gradient) are implicit GEMMs on the tensor cores (tcgen05, FP32
 * accumulators in tensor memory), the 2 -> 32 and 32 -> 2 ones run on the FP32 pipes.  Parameters
 * (FP32, the flat order: per layer W[cout][cin][3][3], b[cout], then g[cout] for the normalised
 * blocks) are the caller's at creation.  All x / y / target / gradient pointers are DEVICE
 * pointers; one handle is one stream's state and is not thread-safe.  ot_cnn_forward and
 * ot_cnn_backward synchronise the stream once at the end: a tensor-core kernel whose bounded wait
 * gave up is reported there as OT_ERR_TIMEOUT. */
typedef struct ot_cnn ot_cnn_t;

/* Number of parameters for `channels` hidden channels (only 32 is built; -1 otherwise). */
int64_t ot_cnn_param_count(int32_t channels);

/* Copy the parameters (HOST, ot_cnn_param_count entries) to a new handle on `stream` (NULL =
 * legacy default stream).  Errors: OT_ERR_ARG, OT_ERR_UNSUPPORTED (channels != 32), OT_ERR_OOM. */
int ot_cnn_create(int32_t channels, const float *params, void *stream, ot_cnn_t **out);

/* Parameters to a HOST buffer of capacity cap (OT_ERR_BUF_TOO_SMALL if cap is short). */
int ot_cnn_get_params(ot_cnn_t *c, float *params, int64_t cap);

/* y (B, 2, k, k) = network(x); keeps the activations for ot_cnn_loss / ot_cnn_backward.  y may be
 * NULL (the prediction stays in the handle).  1 <= batch <= 4096. */
int ot_cnn_forward(ot_cnn_t *c, int32_t batch, int32_t k, const float *x, float *y);

/* Gauge-invariant squared error of the last forward against target (B, 2, k, k) (the pair
 * (u + t, v - t) is the same potential pair, so the best t per image is removed first); dy
 * (device, B*2*k*k) receives its gradient with respect to y, *loss (host) its value. */
int ot_cnn_loss(ot_cnn_t *c, const float *target, float *dy, float *loss);

/* Gradients of sum(dy * y) for the last forward: grad (device, param count, overwritten) and,
 * when dx is not NULL, with respect to x. */
int ot_cnn_backward(ot_cnn_t *c, const float *dy, float *grad, float *dx);

/* One Adam step (step >= 1 is the bias-correction count) on the FP32 parameters. */
int ot_cnn_adam(ot_cnn_t *c, const float *grad, float lr, float beta1, float beta2, float eps, int32_t step);

const char *ot_cnn_last_error(const ot_cnn_t *c);   /* NULL: the calling thread's last error  */
void ot_cnn_destroy(ot_cnn_t *c);                    /* NULL-safe                               */

/* sizeof(ot_problem), sizeof(ot_options), sizeof(ot_iter_info), sizeof(ot_result) written to
 * out[0..3] (count >= 4), so bindings can check their struct layouts.  Returns 4. */
int ot_abi_struct_sizes(int64_t *out, int32_t count);

#ifdef __cplusplus
}
#endif
#endif /* OT_IPM_H */
