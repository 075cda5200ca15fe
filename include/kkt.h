/*
 * kkt.h -- C ABI of the GB300 KKT library.
 *
 * The library computes the Newton (KKT) step of a primal-dual interior-point
 * method on a dynamic nonlinear program with the two hybrid sparse solvers of
 * Pacaud & Shin, "GPU-accelerated dynamic nonlinear optimization with
 * ExaModels and MadNLP" (arXiv 2403.15913):
 *
 *   Lifted-KKT (Sec. IV-A, Eq. liftedkkt): Cholesky of the condensed matrix
 *       K_D = W + Sigma_x + delta_x I + J^T diag(D) J, then Richardson
 *       refinement on the original system (Sec. V-B);
 *   HyKKT (Sec. IV-B, Eq. hykkt, Eq. schurcomp): Cholesky of
 *       K_gamma = W + Sigma_x + delta_x I + gamma J^T J and conjugate
 *       gradients on S_gamma = J K_gamma^{-1} J^T.
 *
 * Every solve returns the solution of
 *
 *     [ W + Sigma_x + delta_x I    J^T ] [dx]   [r_x]
 *     [ J                          -C  ] [dy] = [r_y]          (K_orig)
 *
 * i.e. the condensed system Eq. (kkt:condensed) with the variable-bound
 * barrier terms folded into Sigma_x; C = 0 for the equality-constrained
 * system and C = D^{-1} for the relaxed problem of Eq. (problemrelaxation).
 * Callers pass r = -F_mu (Eq. newtonstep).
 *
 * Conventions for every function below:
 *  - Pointers named d_* are DEVICE memory (current CUDA device); all others
 *    are HOST memory.  The caller owns every buffer it passes; the library
 *    owns the context and all of its workspace.
 *  - Integer arrays are int32, floating-point arrays float64 (FP64).
 *  - Work is enqueued on the given stream; functions that return a value the
 *    host needs (status, step info) synchronise that stream before returning.
 *    One context is used by one stream at a time.
 *  - Functions return a kkt_status; they never abort the process and never
 *    trap on the device.  kkt_last_error() gives a message for the last error
 *    of a context.
 */
#ifndef KKT_GB300_H
#define KKT_GB300_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KKT_CONVERGED = 1,      /* kkt_ipm_step: the optimality error is <= tol   */
    KKT_OK = 0,
    KKT_ERR_ARG = -1,       /* invalid argument (sizes, NULL, bad pattern)    */
    KKT_ERR_OOM = -2,       /* device allocation failed                      */
    KKT_ERR_CUDA = -3,      /* a CUDA runtime call failed                     */
    KKT_ERR_NOT_SPD = -4,   /* non-positive pivot: kkt_info.failed_col is set */
    KKT_ERR_MAXIT = -5,     /* CG or refinement hit its iteration limit       */
    KKT_ERR_STALL = -6,     /* refinement stopped improving (eta stagnated)   */
    KKT_ERR_TIMEOUT = -7,   /* a dependency wait of the dataflow triangular
                               solves (staged_solve 2, 3) gave up after one
                               second: the solution is invalid; the solve
                               state is reset, so the next call starts clean */
    KKT_ERR_STATE = -8,     /* call out of order (e.g. solve before factor)   */
    KKT_ERR_INTERNAL = -9   /* a consistency check of the analysis' index
                               maps failed on the host (a library bug)       */
} kkt_status;

typedef enum { KKT_LIFTED = 0, KKT_HYKKT = 1 } kkt_scheme;

typedef struct kkt_ctx kkt_ctx;

/* Options.  Fill with kkt_default_options() and change what you need. */
typedef struct {
    int scheme;          /* KKT_LIFTED or KKT_HYKKT                            */
    /* symbolic analysis (pinned nested dissection, Sec. V-B) */
    int leaf_size;       /* ND components this small are ordered by minimum
                            degree (default 8)                                */
    int relax_cols;      /* relaxed amalgamation: max merged width (32);
                            0 keeps fundamental supernodes                    */
    int relax_zeros;     /* max explicit zeros in a merged panel (128)        */
    int max_width;       /* supernodes wider than this are cut (32);
                            0 or anything above 64 means 64                   */
    /* numerics */
    double delta;        /* Lifted-KKT: D = 1/delta when factor gets D = NULL
                            (default 1e-8)                                    */
    double gamma;        /* HyKKT gamma (default 1e4; the paper uses 1e7)     */
    double tol_refine;   /* stop refinement at eta <= tol_refine (1e-10)      */
    double tol_cg;       /* CG stops at ||res||_2 <= tol_cg ||rhs||_2 (1e-10) */
    int max_refine;      /* refinement sweeps after the first solve (20)      */
    int max_cg;          /* CG iterations per inner solve (200)               */
    int target_relaxed;  /* 0: refine against C = 0 (Eq. kkt:condensed);
                            1: against C = D^{-1} (relaxed problem, Lifted
                            only)                                             */
    int subtree_cols;    /* subtrees of the supernodal tree with at most this
                            many columns (and at most 1024) are factorised
                            and solved by one CTA each (32); 0 disables       */
    int precision;       /* 0: factor in FP64 (default).  1: factor in FP32,
                            2: in double-float (pairs of FP32 numbers, ~48
                            significand bits, on the FP32 pipe), and refine
                            in FP64 against the FP64 system; if
                            the FP32 factor meets a non-positive pivot, or
                            the refinement stalls or hits max_refine, the
                            system is factorised again in FP64 and the solve
                            is redone (mixed-precision factorisation: an
                            extension; the paper's pipeline is FP64)          */
    int solver;          /* 0: supernodal Cholesky of the general pattern
                            (default).  1: block cyclic reduction of the
                            block-tridiagonal K of a stage-structured problem
                            (stage-major variables, blocks of `block`
                            variables; W within a stage, J rows within two
                            consecutive stages): the structure-exploiting,
                            parallel-in-time solver Sec. VII-B names as
                            future work.  FP64, single instance, block <= 80; the
                            analysis rejects other patterns (KKT_ERR_ARG);
                            kkt_factor_export is not available               */
    int block;           /* block size for solver 1 (2k+1 for the column)    */
    int staged_solve;    /* 1 (default): the level-scheduled triangular
                            solves stage each supernode's panel in shared
                            memory and start while the previous level runs
                            (programmatic dependent launch); 0: the plain
                            level kernels.  Levels whose panels do not fit
                            96 KB use the plain kernels either way.
                            2: dataflow triangular solves, one launch per
                            direction: CTAs take the subtree tasks and level
                            supernodes by ticket in a topological order of
                            the tree and wait (bounded) on per-item arrival
                            counters in L2 instead of one launch per level;
                            3: the same for the level supernodes only, the
                            subtree tasks in their own launches.  2 and 3
                            are used when the widest staged panel fits
                            100 KB, else 1 is                                */
} kkt_options;

/* Per-call report.  Fields not touched by a call keep their values. */
typedef struct {
    int refine_iters;    /* refinement sweeps after the first inner solve     */
    int cg_iters;        /* total CG iterations of the last solve (HyKKT)     */
    int failed_col;      /* first column (permuted order) with a non-positive
                            pivot in the last factor, -1 if none              */
    int status_detail;   /* precision of the factor in use: 0 FP64 (precision
                            0), 1 FP32, 2 FP64 after a fallback from FP32 or
                            double-float, 3 double-float; a solve that fell
                            back sets 2 as well                               */
    double bwd_err;      /* eta = ||b - K_orig v||_inf /
                                  (||K_orig||_inf ||v||_inf + ||b||_inf)      */
    double delta_x;      /* delta_x used by the last factor                    */
} kkt_info;

void kkt_default_options(kkt_options* opt);

/* Symbolic analysis (Sec. V-B: done once, the pattern of K is fixed across
 * IPM iterations).  n variables, m constraints.
 *   W_colptr[n+1], W_rowind[nnzW]: pattern of the LOWER triangle of the
 *       Hessian W, CSC, row indices >= column index (diagonal optional);
 *   J_rowptr[m+1], J_colind[nnzJ]: pattern of the Jacobian J (m x n), CSR;
 *       no column index repeated within a row.
 * Value arrays passed to kkt_factor follow exactly these entry orders.
 * On success *out receives a new context (free with kkt_destroy).
 * Errors: KKT_ERR_ARG on out-of-range or upper-triangular indices or a J row
 * that repeats a column,
 * KKT_ERR_OOM / KKT_ERR_CUDA on device failures. */
kkt_status kkt_analyse(int n, int m,
                       const int* W_colptr, const int* W_rowind,
                       const int* J_rowptr, const int* J_colind,
                       const kkt_options* opt, kkt_ctx** out);

/* Same analysis, host only: no device memory is touched, so it runs on a
 * machine without a GPU.  The context serves kkt_symbolic_sizes and
 * kkt_symbolic_export; kkt_factor on it returns KKT_ERR_STATE. */
kkt_status kkt_analyse_host(int n, int m,
                            const int* W_colptr, const int* W_rowind,
                            const int* J_rowptr, const int* J_colind,
                            const kkt_options* opt, kkt_ctx** out);

/* Sizes of the symbolic result of kkt_analyse (the one-time symbolic
 * factorisation that the paper keeps across refactorisations, Sec. V-B;
 * its SYM column of Table I): supernodes, nonzeros of L, stored panel
 * entries (nnz(L) plus explicit zeros of relaxed supernodes), total row
 * indices over supernodes, levels of the supernodal elimination tree, and
 * the factorisation flop count sum_j cc_j^2 of the exact structure.  With
 * solver = 1 (after a device analysis), levels and flops are those of the
 * block cyclic reduction (dense-block flops of every elimination and
 * update). */
kkt_status kkt_symbolic_sizes(const kkt_ctx* ctx, int* ns, int64_t* nnz_L,
                              int64_t* panel_entries, int64_t* row_entries,
                              int* levels, double* flops);

/* Copy out the symbolic analysis of Sec. V-B (fill-reducing ordering,
 * elimination tree, column counts, supernodes), host arrays, caller-allocated:
 * perm[n] (new -> old), parent[n] (etree of P K P^T, -1 for roots),
 * colcount[n], sn_ptr[ns+1], sn_rowptr[ns+1], sn_rows[row_entries]
 * (supernode row structures in permuted labels).  Any pointer may be NULL. */
kkt_status kkt_symbolic_export(const kkt_ctx* ctx, int* perm, int* parent,
                               int* colcount, int* sn_ptr, int* sn_rowptr,
                               int* sn_rows);

/* Numeric factorisation (refactorisation of Sec. V-B).
 *   d_Wval[nnzW]  W values in the kkt_analyse order;
 *   d_Jval[nnzJ]  J values in the kkt_analyse order;
 *   d_sigma[n]    Sigma_x (barrier diagonal of the variable bounds);
 *   d_D[m]        Lifted-KKT: the diagonal D (NULL means 1/delta);
 *                 HyKKT: must be NULL (D = gamma);
 *   delta_x       primal regularisation (inertia correction, Sec. III-B).
 * The library copies the values it needs (the residuals of later kkt_solve
 * calls use them), so the caller may reuse or free its buffers as soon as
 * the call returns.
 * Returns KKT_ERR_NOT_SPD with info->failed_col set when a pivot is not
 * positive (the caller raises delta_x and calls again). */
kkt_status kkt_factor(kkt_ctx* ctx, const double* d_Wval, const double* d_Jval,
                      const double* d_sigma, const double* d_D, double delta_x,
                      cudaStream_t stream, kkt_info* info);

/* Solve K_orig [dx; dy] = [r_x; r_y] with the factor of the last
 * kkt_factor (scheme per options), refining until eta <= tol_refine.
 *   d_rx[n], d_ry[m] in; d_dx[n], d_dy[m] out (all four non-NULL, else
 *   KKT_ERR_ARG);
 *   d_ds[m] (may be NULL): relaxed target only, ds = J dx - r_y.
 * Returns KKT_ERR_MAXIT / KKT_ERR_STALL when the tolerance is not reached
 * (the best iterate is still written) and KKT_ERR_STATE without a factor. */
kkt_status kkt_solve(kkt_ctx* ctx, const double* d_rx, const double* d_ry,
                     double* d_dx, double* d_dy, double* d_ds,
                     cudaStream_t stream, kkt_info* info);

/* ------------------------------------------------------------------------
 * Batches of independent systems (uneven sizes), solved together.  The
 * paper's method reuses one symbolic factor across IPM iterations (Sec.
 * V-B); a batch applies the same steps to the block-diagonal union of
 * `count` instances (e.g. many NMPC problems of different horizons), so that
 * every level of every instance's elimination tree is factorised and solved
 * in the same launches.  Vectors and value arrays of a batch are the
 * instances' own arrays concatenated in instance order (instance i owns
 * variables [x_off[i], x_off[i+1]) and constraints [y_off[i], y_off[i+1]);
 * its W and J values follow those of instance i-1).  kkt_factor, kkt_solve,
 * kkt_backsolve and kkt_factor_export accept a batch context unchanged; the
 * refinement and CG then run per instance (each with its own eta, stopping
 * rule and CG scalars), and kkt_info carries maxima (refine_iters, bwd_err),
 * the CG total and the first failing column.
 * ---------------------------------------------------------------------- */

/* Analysis of a batch: per instance the same arguments as kkt_analyse
 * (arrays of `count` host pointers), analysed concurrently on host threads.
 * The result equals kkt_analyse of the union's pattern.  The union must fit
 * 32-bit indices (n + m, nnz(W), nnz(J) < 2^31), else KKT_ERR_ARG. */
kkt_status kkt_analyse_batch(int count, const int* n, const int* m,
                             const int* const* W_colptr, const int* const* W_rowind,
                             const int* const* J_rowptr, const int* const* J_colind,
                             const kkt_options* opt, kkt_ctx** out);

/* Same, host only (see kkt_analyse_host). */
kkt_status kkt_analyse_batch_host(int count, const int* n, const int* m,
                                  const int* const* W_colptr, const int* const* W_rowind,
                                  const int* const* J_rowptr, const int* const* J_colind,
                                  const kkt_options* opt, kkt_ctx** out);

/* count (1 for a context from kkt_analyse), x_off[count+1], y_off[count+1];
 * any pointer may be NULL. */
kkt_status kkt_batch_layout(const kkt_ctx* ctx, int* count, int* x_off, int* y_off);

/* kkt_factor with one delta_x per instance (host array delta_x[count]).  An
 * instance whose pivot fails does not affect the others: the call returns
 * KKT_ERR_NOT_SPD, kkt_batch_results gives the failing instances, and
 * kkt_solve still solves the rest (unless every instance failed). */
kkt_status kkt_factor_batch(kkt_ctx* ctx, const double* d_Wval, const double* d_Jval,
                            const double* d_sigma, const double* d_D, const double* delta_x,
                            cudaStream_t stream, kkt_info* info);

/* One Newton step's linear algebra (Sec. III, the factorisation of Sec. V-B
 * and the refined Lifted-KKT or HyKKT solve of Sec. IV) as ONE CUDA graph
 * launch: kkt_factor_batch(d_Wval, d_Jval, d_sigma, d_D, delta_x) followed
 * by kkt_solve(d_rx, d_ry, d_dx, d_dy, NULL), with the refinement sweeps
 * (and HyKKT's CG iterations) as conditional WHILE nodes whose conditions
 * kernels set on the device, so that the host waits once, at the end.  The
 * stopping rules, kernels and per-instance results (kkt_batch_results,
 * info) are those of the two calls; kkt_solve and kkt_backsolve may follow
 * with the factor left behind.
 *   delta_x: host array of one value >= 0 per instance (one value for a
 *            kkt_analyse context), copied to pinned memory and from there
 *            to the device inside the graph;
 *   the device buffers as for kkt_factor_batch and kkt_solve (all but d_D
 *            non-NULL).
 * The graph is captured on the first call and replayed while the eight
 * device pointers stay the same; other pointers capture it again (a few
 * ms).  Supernodal FP64 factor only (options solver 0, precision 0; other
 * settings return KKT_ERR_ARG).  Returns KKT_ERR_NOT_SPD when some
 * instance's pivot failed (kkt_batch_results names them; the others are
 * solved), else KKT_OK, KKT_ERR_MAXIT or KKT_ERR_STALL as kkt_solve.
 * Synchronises the stream; the pinned buffers of the context are reused,
 * so calls on one context from several host threads must be serialised. */
kkt_status kkt_factor_solve(kkt_ctx* ctx, const double* d_Wval, const double* d_Jval,
                            const double* d_sigma, const double* d_D, const double* delta_x,
                            const double* d_rx, const double* d_ry, double* d_dx, double* d_dy,
                            cudaStream_t stream, kkt_info* info);

/* Autotuner of the supernode partition (the panel shapes the factor
 * kernels work on) for a batch, on this GPU: up to `sample` instances
 * (evenly spaced; <= 0 means 32) are analysed with each candidate setting of
 * relax_cols, relax_zeros, max_width and subtree_cols, and the numeric
 * factorisation of synthetic SPD values (K = I + J^T J) is timed with CUDA
 * events on `stream`; *best = *base (defaults if NULL) with the fastest
 * candidate's four fields, *best_ms (may be NULL) its median time.  The
 * paper has no counterpart (its factorisation is a vendor library's). */
kkt_status kkt_autotune_batch(int count, const int* n, const int* m,
                              const int* const* W_colptr, const int* const* W_rowind,
                              const int* const* J_rowptr, const int* const* J_colind,
                              const kkt_options* base, int sample, cudaStream_t stream,
                              kkt_options* best, double* best_ms);

/* Precision of the following factorisations: 0 (FP64) or the reduced
 * precision the context was analysed with (kkt_options.precision 1 or 2,
 * whose storage exists), else KKT_ERR_ARG.  For a driver that knows the
 * reduced precision will not refine (e.g. it fell back to FP64 at the
 * previous IPM iteration: late iterations only grow the spread of Sigma)
 * and would otherwise pay both factorisations; the paper keeps FP64
 * throughout (Sec. V-B), the reduced precision is an extension. */
kkt_status kkt_set_precision(kkt_ctx* ctx, int precision);

/* Per-instance switch of the factorisation of a batch: active[i] = 0 makes
 * the following factorisations leave instance i's panels as the assembly
 * leaves them (no factorisation work), so a solve of instance i is valid
 * only for a zero right-hand side (which gives zero); NULL switches every
 * instance on (the default).  Takes effect at the next kkt_factor,
 * kkt_factor_batch or kkt_factor_solve on the context; the array is copied,
 * but it must not change while a factorisation of this context is in
 * flight.  KKT_ERR_ARG for a non-NULL array on a single system.  (An
 * extension for batched serving, which the paper does not have: members of
 * a batch that take no step cost no factorisation.) */
kkt_status kkt_batch_set_active(kkt_ctx* ctx, const int* active);

/* Per-instance results of the last kkt_factor / kkt_solve (host arrays of
 * count entries, any may be NULL): status (KKT_OK, KKT_ERR_STALL,
 * KKT_ERR_MAXIT, KKT_ERR_NOT_SPD), refinement sweeps, CG iterations,
 * backward error eta (infinity for failed instances) and the first failing
 * column (permuted numbering of the union, -1 if none). */
kkt_status kkt_batch_results(const kkt_ctx* ctx, int* status, int* refine_iters,
                             int* cg_iters, double* bwd_err, int* failed_col);

/* Backsolve with the condensed matrix of the last successful kkt_factor
 * (the SOLVE column of Table I): d_x[n] = K^{-1} d_b[n], original ordering.
 * d_b and d_x may alias.  KKT_ERR_STATE without a factor. */
kkt_status kkt_backsolve(kkt_ctx* ctx, const double* d_b, double* d_x,
                         cudaStream_t stream);

/* Backsolve that allocates nothing (the paper has no counterpart: this is a
 * service for callers that may not allocate device memory, such as a
 * real-time control loop that must not touch the allocator after start-up,
 * or code that runs while another component owns every allocation).
 * Same result as kkt_backsolve: d_x[n] = K^{-1} d_b[n] with the factor of the
 * last successful kkt_factor.  Its only scratch (one permuted vector) is a
 * fixed device array inside the library of KKT_STATIC_SCRATCH_DOUBLES
 * doubles (16 MiB), which every GPU that loads the library holds until the
 * process exits.  Sizes n > KKT_STATIC_SCRATCH_DOUBLES return KKT_ERR_ARG.
 * The array is placed on the device, and its device address looked up once
 * per device, by kkt_analyse (with that device current), so this call itself
 * takes no device memory.  All calls share the one array: calls that overlap
 * on the GPU (other streams, other contexts of this library) race and give
 * wrong results.  Each call returns only after its stream has finished, so
 * calls from one host thread never overlap; calls from different host
 * threads must be serialised by the caller (e.g. one mutex around them).
 * No profiling events are recorded. */
#define KKT_STATIC_SCRATCH_DOUBLES (1 << 21)
kkt_status kkt_backsolve_noalloc(kkt_ctx* ctx, const double* d_b, double* d_x,
                                 cudaStream_t stream);

/* Test hook of bounds-check builds (the library compiled with
 * -DKKT_BOUNDS_CHECK=1, in which every index read from a precomputed map is
 * tested on the device before it is used, and a failed test makes
 * kkt_factor / kkt_solve / kkt_backsolve return KKT_ERR_INTERNAL without any
 * out-of-bounds access; not a step of the paper's method).  what = 1
 * overwrites one entry of the Schur-update relative-row map with a row one
 * past its target supernode's rows -- a wrong index that still lies inside
 * the factor storage -- so that a test can exercise the checks; what = 2
 * raises by one the arrival count the last item of the dataflow solves
 * waits for, so that its bounded wait runs out (the solve then returns
 * KKT_ERR_TIMEOUT); what = 0 restores both.  KKT_ERR_STATE in other
 * builds. */
kkt_status kkt_debug_corrupt_map(kkt_ctx* ctx, int what);

/* Diagnostic: copy the numeric factor L (permuted order) as CSC with the
 * panel structure: colptr[n+1], rowind[], val[] sized by the panel entries
 * below and on the diagonal (lower trapezoid of each supernode panel). */
kkt_status kkt_factor_export(kkt_ctx* ctx, int64_t* colptr, int* rowind,
                             double* val);

/* Message of the last error of ctx; with ctx == NULL, of the last call on
 * this thread that failed before a context existed (e.g. kkt_analyse). */
const char* kkt_last_error(const kkt_ctx* ctx);

/* Tracing (Table I/II of the paper split the time into symbolic analysis,
 * refactorisation and backsolve).  With profiling on, CUDA events recorded
 * on the caller's stream bracket the phases and their device times are
 * accumulated at the synchronisation that ends each call; the launch
 * counters are kept always. */
typedef struct {
    double assemble_ms;      /* assembly of the condensed matrix          */
    double factor_ms;        /* supernodal numeric factorisation         */
    double solve_ms;         /* triangular solves (forward + backward)   */
    double other_ms;         /* residuals, CG vector work, J/J^T products */
    int64_t launches;        /* kernels launched by this context          */
    int64_t factor_launches; /* of which numeric-factorisation kernels    */
    int64_t factor_calls;    /* kkt_factor calls                          */
    int64_t kinv_calls;      /* applications of K^{-1} (pairs of solves)  */
    int64_t fp32_factors;    /* reduced-precision factorizations (FP32 or
                                double-float, precision 1 or 2)           */
    int64_t fp64_fallbacks;  /* FP64 refactorizations after an FP32 factor
                                failed or did not refine to tol_refine    */
    int64_t graph_steps;     /* kkt_factor_solve calls (one graph launch
                                each)                                     */
} kkt_stats;

kkt_status kkt_set_profiling(kkt_ctx* ctx, int enable);
kkt_status kkt_get_stats(const kkt_ctx* ctx, kkt_stats* out);
kkt_status kkt_reset_stats(kkt_ctx* ctx);
void kkt_destroy(kkt_ctx* ctx);

/* ------------------------------------------------------------------------
 * Distillation-column model (Sec. VI-A), per-stage evaluation kernels.
 * params[16] (host): k, T, h, alpha, D, F, x_f, M, xbar, ubar, rho, xbar_0,
 * x_lo, x_hi, u_lo, u_hi.  Variables are stage-major
 * [x_1..x_k, y_1..y_k, u] per stage t = 0..T; constraints per stage are the
 * initial condition (t = 0) or implicit-Euler dynamics (t >= 1), then the
 * vapour-liquid equilibrium.
 * ---------------------------------------------------------------------- */

/* n = (2k+1)(T+1), m = 2k(T+1) and the pattern sizes. */
kkt_status kkt_tray_sizes(const double* params, int* n, int* m, int* nnzW,
                          int* nnzJ);

/* Host patterns in the order the evaluation kernels write values:
 * lower-CSC of W (every diagonal plus (u_t, x_it), (u_t, y_it)) and CSR of J
 * (columns ascending).  Arrays sized by kkt_tray_sizes. */
kkt_status kkt_tray_pattern(const double* params, int* W_colptr, int* W_rowind,
                            int* J_rowptr, int* J_colind);

/* Device evaluation at the primal point d_w[n] with multipliers d_lam[m]:
 *   d_f[1]        objective (NULL to skip)
 *   d_grad[n]     gradient of the objective (NULL to skip)
 *   d_c[m]        constraint values (NULL to skip)
 *   d_Jval[nnzJ]  Jacobian values (NULL to skip)
 *   d_Wval[nnzW]  Hessian of obj_weight * f + lam^T c, lower (NULL to skip;
 *                 d_lam may be NULL only when this is NULL)
 * Asynchronous on stream. */
kkt_status kkt_tray_eval(const double* params, const double* d_w,
                         const double* d_lam, double obj_weight, double* d_f,
                         double* d_grad, double* d_c, double* d_Jval,
                         double* d_Wval, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Minimal filter line-search interior-point driver (Sec. III: Newton steps
 * on F_mu(w) = 0, Eq. newtonstep, with a fraction-to-boundary rule; the
 * filter line search of Wachter & Biegler that MadNLP implements, in its
 * basic form: monotone barrier update, inertia correction by delta_x, no
 * second-order correction and no restoration phase).  Every step runs on the
 * device: derivative kernels of the column model, the KKT solve of this
 * library, and kernels for the step recovery, fraction to boundary, filter
 * measures and updates; only scalars come back to the host.
 *
 * Problem: min f(x) s.t. c(x) = 0, x_L <= x <= x_U (HyKKT, or Lifted-KKT
 * with relaxed = 0), or with relaxed = 1 the relaxed problem of
 * Eq. (problemrelaxation): c(x) - s = 0, -tau <= s <= tau, whose condensed
 * matrix is W + Sigma_x + J^T Sigma_s J (requires scheme KKT_LIFTED).
 * ---------------------------------------------------------------------- */
typedef struct kkt_ipm kkt_ipm;

typedef struct {
    double tol;        /* stop at scaled optimality error <= tol (1e-8)     */
    int max_iter;      /* iteration limit of kkt_ipm_solve (200)             */
    double mu_init;    /* initial barrier parameter (0.1)                   */
    int relaxed;       /* 1: Lifted-KKT relaxed problem (default: 1 for the
                          Lifted scheme, 0 for HyKKT)                       */
    double tau_relax;  /* relaxation tau (1e-8)                             */
} kkt_ipm_options;

typedef struct {
    int iter;          /* iterations taken so far                           */
    int ls_trials;     /* line-search trial points of the last step         */
    int refine_iters;  /* from the last KKT solve                           */
    int cg_iters;      /* from the last KKT solve                           */
    double mu, objective, inf_pr, inf_du, inf_compl, err0;
    double alpha_pr, alpha_du, delta_x, bwd_err;
    double t_eval_ms, t_kkt_ms, t_step_ms;   /* device time of the last step:
                          derivative evaluation, KKT factor + solve, total  */
    int launches;      /* kernels the driver itself launched in the last step
                          (the KKT context's own are counted in kkt_stats)  */
} kkt_ipm_info;

void kkt_ipm_default_options(kkt_ipm_options* opt);

/* Creates the driver for the column model with parameters tray_params[16]
 * (see kkt_tray_sizes); runs the symbolic analysis once (kopt may be NULL). */
kkt_status kkt_ipm_create(const double* tray_params, const kkt_options* kopt,
                          const kkt_ipm_options* iopt, kkt_ipm** out);

/* (Re)starts from d_x0[n] (NULL: compositions at xbar_0, controls at ubar),
 * pushed inside the bounds; multipliers y = 0, bound multipliers 1. */
kkt_status kkt_ipm_init(kkt_ipm* ipm, const double* d_x0, cudaStream_t stream);

/* One IPM iteration.  Returns KKT_OK after a step, KKT_CONVERGED when the
 * current point already satisfies the tolerance (no step taken),
 * KKT_ERR_STALL when the line search failed, KKT_ERR_NOT_SPD when inertia
 * correction gave up, or another error. */
kkt_status kkt_ipm_step(kkt_ipm* ipm, cudaStream_t stream, kkt_ipm_info* info);

/* Iterates kkt_ipm_step until convergence (returns KKT_CONVERGED), an error,
 * or max_iter iterations (returns KKT_ERR_MAXIT); info holds the last step. */
kkt_status kkt_ipm_solve(kkt_ipm* ipm, cudaStream_t stream, kkt_ipm_info* info);

/* Copies the current iterate (device arrays; any may be NULL): x[n], y[m],
 * z_L[n], z_U[n], s[m] (relaxed problem only). */
kkt_status kkt_ipm_get(const kkt_ipm* ipm, double* d_x, double* d_y, double* d_zl,
                       double* d_zu, double* d_s, cudaStream_t stream);

/* The KKT context the driver uses (for kkt_get_stats / profiling). */
kkt_ctx* kkt_ipm_kkt(kkt_ipm* ipm);

void kkt_ipm_destroy(kkt_ipm* ipm);

/* Receding-horizon use (Sec. V-B: the symbolic factor is kept across
 * solves).  Pins the stage-0 compositions to x0[k] (host; one value per
 * tray) in the initial-condition rows, instead of xbar_0 on every tray;
 * NULL restores xbar_0.  Takes effect at the next kkt_ipm_init. */
kkt_status kkt_ipm_set_initial_state(kkt_ipm* ipm, const double* x0, cudaStream_t stream);

/* kkt_ipm_init from a previous solution d_prev[n] shifted by one stage
 * (stage t takes stage t+1's values, the last stage keeps its own): the
 * warm start of the next receding-horizon solve. */
kkt_status kkt_ipm_init_shifted(kkt_ipm* ipm, const double* d_prev, cudaStream_t stream);

/* Warm start of the next receding-horizon solve from the driver's own last
 * iterate: primal variables, constraint multipliers and bound multipliers
 * (and, relaxed, slacks and their multipliers) shifted by one stage in
 * place, the primal pushed inside its bounds, barrier parameter mu, empty
 * filter; recenter = 1 resets the bound multipliers to mu / slack (the
 * products start on the central path).  KKT_ERR_STATE before any
 * kkt_ipm_init. */
kkt_status kkt_ipm_init_warm(kkt_ipm* ipm, double mu, int recenter, cudaStream_t stream);

/* Device memory held by the driver and its KKT context, in bytes. */
kkt_status kkt_ipm_device_bytes(const kkt_ipm* ipm, int64_t* bytes);

/* Device memory held by a KKT context, in bytes. */
kkt_status kkt_device_bytes(const kkt_ctx* ctx, int64_t* bytes);

/* ------------------------------------------------------------------------
 * Batched IPM: `count` column problems (one kkt_ipm each, "members") solved
 * in lock-step with ONE KKT system per iteration.  Every member keeps its
 * own iterate, barrier parameter, filter, inertia-correction ladder and line
 * search (the steps of kkt_ipm_step); the Newton step of Sec. III for all
 * members that still iterate is one factorisation and refined solve of the
 * block-diagonal union of their KKT systems (kkt_analyse_batch; with kopt
 * precision 0 one kkt_factor_solve graph launch, with precision 1 or 2 the
 * reduced-precision factor with FP64 refinement and fallback).  Each
 * phase of an iteration enqueues the kernels of every stepping member on
 * the one stream and synchronises once.  Members start and stop
 * independently (continuous batching, kkt_ipm_batch_start_member): one that
 * does not step is switched off in the union's factorisation
 * (kkt_batch_set_active) and has a zero right-hand side, so it costs no
 * factorisation work and its refinement stops at once.
 * ---------------------------------------------------------------------- */
typedef struct kkt_ipm_batch kkt_ipm_batch;

/* tray_params: count x 16 values (member i at tray_params + 16 i); kopt and
 * iopt apply to every member (either may be NULL). */
kkt_status kkt_ipm_batch_create(int count, const double* tray_params, const kkt_options* kopt,
                                const kkt_ipm_options* iopt, kkt_ipm_batch** out);

/* Member i (0 <= i < count), for kkt_ipm_init / kkt_ipm_init_shifted /
 * kkt_ipm_init_warm / kkt_ipm_set_initial_state / kkt_ipm_get.  Calling
 * kkt_ipm_step or kkt_ipm_solve on a member returns KKT_ERR_STATE. */
kkt_ipm* kkt_ipm_batch_member(kkt_ipm_batch* batch, int i);

/* Marks every member as iterating (each must have been initialised). */
kkt_status kkt_ipm_batch_start(kkt_ipm_batch* batch);

/* Continuous batching: member i, initialised since it last stopped
 * (kkt_ipm_init / kkt_ipm_init_shifted / kkt_ipm_init_warm), takes part in
 * the following kkt_ipm_batch_step calls while the other members go on.
 * KKT_ERR_STATE if it never was initialised or still iterates. */
kkt_status kkt_ipm_batch_start_member(kkt_ipm_batch* batch, int i);

/* Member i's state: status KKT_OK while it iterates, else its final status
 * (KKT_CONVERGED, KKT_ERR_MAXIT after max_iter steps, KKT_ERR_STALL, ...;
 * KKT_ERR_STATE before it first started); iters its iteration count. */
kkt_status kkt_ipm_batch_member_status(const kkt_ipm_batch* batch, int i, int* status, int* iters);

/* Device memory of the batch: the union's KKT context, the members' IPM
 * buffers and the union's value and vector arrays, in bytes. */
kkt_status kkt_ipm_batch_device_bytes(const kkt_ipm_batch* batch, int64_t* bytes);

/* One lock-step iteration of every member still iterating; info (may be
 * NULL) receives count reports, written for the members that took a step
 * or stopped in this call.  Returns KKT_CONVERGED when no member iterates
 * any more (per-member results: kkt_ipm_batch_solve's status array, or the
 * reports), KKT_OK otherwise, another code on a batch-wide error. */
kkt_status kkt_ipm_batch_step(kkt_ipm_batch* batch, cudaStream_t stream, kkt_ipm_info* info);

/* kkt_ipm_batch_start, then steps until no member iterates: status[i]
 * (KKT_CONVERGED, KKT_ERR_MAXIT after max_iter steps, KKT_ERR_STALL,
 * KKT_ERR_NOT_SPD, ...) and iters[i] per member (either may be NULL), info
 * as for kkt_ipm_batch_step (the last report of each member).  Returns
 * KKT_CONVERGED when every member converged, else the first member's
 * failure code. */
kkt_status kkt_ipm_batch_solve(kkt_ipm_batch* batch, cudaStream_t stream, int* status, int* iters,
                               kkt_ipm_info* info);

/* The batch's KKT context (stats, profiling) and its last error message. */
kkt_ctx* kkt_ipm_batch_kkt(kkt_ipm_batch* batch);
const char* kkt_ipm_batch_last_error(const kkt_ipm_batch* batch);

void kkt_ipm_batch_destroy(kkt_ipm_batch* batch);

/* ------------------------------------------------------------------------
 * NMPC serving (no counterpart in the paper, whose use case it serves: a
 * controller re-solves its horizon-T problem from each new state, reusing
 * the symbolic factorisation, Sec. V-B).  A server holds clients (one
 * column model each, fixed k and T) and runs their requests -- full IPM
 * solves -- on `slots` worker threads, each with its own CUDA stream, so
 * solves of different clients overlap on the device; a client's requests
 * run in submission order.  A client's context (symbolic analysis, factor
 * storage, IPM buffers, last solution) stays resident between requests
 * while it fits in hbm_budget_gb (least recently used idle contexts are
 * evicted to admit others); a request starts from the client's previous
 * solution shifted one stage (warm_start = 1), with the stage-0 state
 * given or, if omitted, taken from stage 1 of the previous solution.
 * ---------------------------------------------------------------------- */
typedef struct kkt_server kkt_server;

typedef struct {
    int slots;              /* concurrent solves (8)                              */
    double hbm_budget_gb;   /* device memory of resident contexts (40)            */
    int scheme;             /* KKT_LIFTED (default) or KKT_HYKKT                  */
    int precision;          /* kkt_options.precision (0)                          */
    double gamma;           /* HyKKT gamma (1e7)                                  */
    double tol;             /* IPM tolerance (1e-8)                               */
    int max_iter;           /* IPM iterations (200)                               */
    double mu_init;         /* initial barrier parameter (0.1)                    */
    int warm_start;         /* 1: start from the shifted previous iterate (1)     */
    double warm_mu;         /* barrier parameter of warm starts (1e-4)            */
    int warm_recenter;      /* 1: warm starts recentre the bound multipliers (1)  */
    int batch;              /* 0 (default): one solve per slot.  b > 0: batched
                               serving -- clients are grouped, in the order
                               they are added, into cohorts of up to b (a
                               cohort closes when full or at the first
                               request for one of its clients); a cohort is
                               one kkt_ipm_batch, so each IPM iteration of
                               all its running requests is one factorisation
                               and refined solve of the union of their KKT
                               systems (precision 1: FP32 factor, FP64
                               refinement); requests join and leave between
                               iterations; a slot runs one cohort at a time;
                               cohorts are admitted and evicted as a unit     */
} kkt_server_options;

typedef struct {
    int64_t id;
    int client, slot;
    int status;             /* KKT_CONVERGED, KKT_ERR_MAXIT or an error          */
    int iters;
    int cold;               /* 1: the client's context was created for it        */
    int warm;               /* 1: warm-started from the previous solution        */
    double objective, inf_pr, inf_du;
    double t_submit_ms, t_start_ms, t_done_ms;   /* since kkt_server_create      */
} kkt_request_result;

typedef struct {
    int64_t completed, failed, contexts_created, evictions;
    int64_t resident_bytes, peak_resident_bytes, queued;
    int resident_clients;
} kkt_server_stats;

void kkt_server_default_options(kkt_server_options* opt);

/* Starts the worker threads on CUDA device `device`. */
kkt_status kkt_server_create(const kkt_server_options* opt, int device, kkt_server** out);

/* Registers a client with its 16 model parameters (as kkt_tray_sizes). */
kkt_status kkt_server_add_client(kkt_server* srv, const double* params, int* client);

/* Queues a solve for `client`; x0[k] (host) is the measured state, NULL takes
 * it from the previous solution (or xbar_0 for the first request);
 * keep_solution = 1 keeps x for kkt_server_wait. */
kkt_status kkt_server_submit(kkt_server* srv, int client, const double* x0, int keep_solution,
                             int64_t* id);

/* Blocks until request `id` is done; copies its result and, if it was kept,
 * its solution x[n] into h_x (may be NULL). */
kkt_status kkt_server_wait(kkt_server* srv, int64_t id, kkt_request_result* out, double* h_x);

/* Blocks until every queued request is done. */
kkt_status kkt_server_drain(kkt_server* srv);

kkt_status kkt_server_get_stats(kkt_server* srv, kkt_server_stats* stats);

/* Finishes the running solves, stops the workers, frees every context. */
void kkt_server_destroy(kkt_server* srv);

/* ------------------------------------------------------------------------
 * Verification of the FP64 helper functions the kernels are built on (the
 * pivot reciprocal square root of the Cholesky, Sec. V-B, and the
 * reciprocals, bit-pattern comparisons and splits of the IPM's elementwise
 * kernels, Sec. III).  Evaluates on the device, elementwise,
 *   unary   y[i] = f(x[i])            for i < n
 *   binary  y[i] = f(x[i], x[n + i])  for i < n  (x holds 2n values)
 * with f one of KKT_FN_*.  x and y are device pointers; the call is
 * asynchronous on `stream` (cudaStream_t, NULL: the default stream).
 * Returns KKT_ERR_ARG for an unknown fn or n < 0.                          */
enum {
    KKT_FN_RSQRT = 0,    /* pivot 1/sqrt(x): FP32 seed + third-order step     */
    KKT_FN_RCP = 1,      /* 1/x: FP32 seed + third-order step (x > 0)         */
    KKT_FN_SPLIT_M = 2,  /* m of x = m 2^e, m in [0.5, 1), by the bit layout;
                            NaN unless x is positive and normal               */
    KKT_FN_SPLIT_E = 3,  /* e of the same split, as a double                  */
    KKT_FN_MAX_ABS = 4,  /* max(x0, |x1|) for x0 >= 0, a NaN x1 ignored      */
    KKT_FN_MAX_NN = 5,   /* max(x0, x1) of non-negative values                */
    KKT_FN_MIN_NN = 6,   /* min(x0, x1) of non-negative values                */
    KKT_FN_F32_ROUNDTRIP = 7  /* double(float(x)) by the bit layout (x in
                                 (1e-30, 1e30); truncates the mantissa)       */
};
kkt_status kkt_eval_fn(int fn, int n, const double* x, double* y, void* stream);

#ifdef __cplusplus
}
#endif
#endif
