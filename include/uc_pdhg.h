/*
 * uc_pdhg.h -- C ABI of the GB300 unit-commitment LP solver (restarted PDHG).
 *
 * The paper ("Rapid Concurrent GPU-CPU Solvers for Scalable Unit Commitment in
 * Large Power Grids") runs PDHG on the GPU on the LP relaxation of a
 * multi-period unit-commitment problem (Sec. II-C, Alg. 1 "Solver 1"), after a
 * presolve (Sec. II-D) and with an iteration limit of 100,000, an absolute
 * feasibility tolerance of 1e-5 and a convergence tolerance of 1e-4
 * (Sec. II-D).  This library implements that relaxation solve:
 *
 *   uc_build_lp     problem data -> raw DC-UC LP (host)
 *   uc_presolve     raw LP -> reduced, Ruiz/Pock-Chambolle scaled LP with
 *                   A and A^T, step size from ||A||_2 (host)
 *   uc_solve        restarted PDHG on the device (hand-written sm_103a kernels)
 *   uc_solve_batch  several LPs in one block-diagonal device solve
 *   uc_get_solution unscale + postsolve into p, u, v, theta, f, shed, LMPs
 *
 * Conventions for every call:
 *   - return value: UC_OK (0) or a negative UC_E* code; the message of the
 *     last failure on the calling thread is uc_last_error();
 *   - no C++ exception crosses this boundary;
 *   - handles (uc_lp, uc_presolved, uc_result) are owned by the library from
 *     creation until the matching uc_free_*; input arrays are copied, so the
 *     caller keeps ownership of everything it passes in;
 *   - output arrays are caller-allocated host memory of the stated size;
 *   - arrays are C-contiguous; "time-major" means index [t * K + k].
 */
#ifndef UC_PDHG_H
#define UC_PDHG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define UC_OK 0
#define UC_EINVAL (-1)       /* bad sizes or indices, non-positive reactance, self loop */
#define UC_ENOMEM (-2)       /* host or device allocation failed / budget exceeded */
#define UC_EINFEASIBLE (-3)  /* presolve, or a Farkas direction found by the Halpern solve, proved
                                the LP infeasible */
#define UC_EUNBOUNDED (-4)   /* presolve proved the LP unbounded */
#define UC_EITERLIMIT (-5)   /* max_iter reached before the tolerance (result valid) */
#define UC_ETIMEOUT (-6)     /* timeout_ms elapsed (result valid, last iterate) */
#define UC_ENUMERIC (-7)     /* NaN/Inf in the iterates */
#define UC_ECANCELLED (-8)   /* opts.cancel was set (result valid, last iterate) */
#define UC_ECUDA (-9)        /* a CUDA runtime call failed */

typedef struct uc_lp uc_lp;
typedef struct uc_presolved uc_presolved;
typedef struct uc_result uc_result;
typedef struct uc_session uc_session;

/* Multi-period DC unit-commitment data (model: DC relaxation of the UC
 * problem of Sec. II-A; the full GO Challenge 3 AC model is out of scope).
 * Buses 0..B-1, lines 0..L-1 (from != to), units 0..G-1, periods 0..T-1. */
typedef struct {
    int B, L, G, T;
    int ref_bus;                 /* angle reference, theta_ref = 0 */
    const int32_t *line_from;    /* [L] */
    const int32_t *line_to;      /* [L] */
    const double *x_pu;          /* [L] reactance (p.u., > 0) */
    const double *fmax;          /* [L] flow limit (MW, >= 0) */
    const int32_t *gen_bus;      /* [G] */
    const double *pmax;          /* [G] MW */
    const double *pmin;          /* [G] MW, 0 <= pmin <= pmax */
    const double *ramp;          /* [G] MW per period */
    const double *c_lin;         /* [G] $/MWh */
    const double *c_nl;          /* [G] $ per committed period */
    const double *c_su;          /* [G] $ per startup */
    const double *u0;            /* [G] commitment before period 0 (0 or 1) */
    const double *load;          /* [T*B] time-major MW, >= 0 */
    double voll;                 /* shed price $/MWh; <= 0: no shed columns (strict balance) */
} uc_problem;

typedef struct {
    int ruiz_iters;              /* Ruiz equilibration passes (default 10) */
    int pock_chambolle;          /* 1: one Pock-Chambolle pass, alpha = 1 (default 1) */
    int power_max_iter;          /* power-iteration products for ||A||_2 (default 500) */
    double power_tol;            /* relative change that stops it (default 1e-10) */
    int value_bits;              /* 64: FP64 matrix values on device; 32: FP32 (default 64) */
    int threads;                 /* host threads for presolve (0 = hardware concurrency) */
    int aggressive;              /* 1: also substitute doubleton equations a_f x_f + a_s x_s = q whose
                                    x_s appears in no other row (on the UC LP: the balance rows of
                                    leaf buses without units hold only the line flow and the shed
                                    column): x_s's bounds move onto x_f and its cost into x_f's, the
                                    row and x_s leave the LP, postsolve recovers both (the paper's
                                    tuned, more aggressive presolve, Sec. II-D).  0: off (default) */
    int power_device;            /* 1: run the power iteration for ||A_s||_2 on the current CUDA
                                    device (same steps and stopping rule, fixed-order device
                                    reductions; A_s and A_s^T are copied to device memory for the
                                    duration of the call); UC_ECUDA without a device.  0: host
                                    threads (default) */
    int eliminate_angles;        /* 1: substitute the free bus angles out before the other
                                    reductions.  Per period a breadth-first spanning tree of the grid
                                    is grown from the reference bus (each bus's lines in row order);
                                    the tree lines' flow rows and every angle column leave the LP,
                                    and each other line's flow row f_l - (theta_a - theta_b) / x_l = 0
                                    becomes f_l - (1/x_l) (sum of +-x_e f_e over the tree path from
                                    a to b) = 0 (Kirchhoff's voltage law on its fundamental cycle,
                                    each entry computed as -+s (1/x_l) / (1/x_e) from the stored
                                    1/x).  The LP is equivalent; postsolve puts the angles back down
                                    the tree and gives a tree line's flow row the dual that its flow
                                    column's reduced cost needs.  Row and column maps still point at
                                    the LP as built.  UC_EINVAL if a period's grid is not connected or
                                    has no single angle fixed at 0.  0: off (default) */
} uc_presolve_opts;

/* Device memory callback: return `bytes` bytes of device memory usable on
 * `stream` (aligned to 256 B), or NULL.  Used for every device allocation
 * when set; otherwise cudaMallocAsync/cudaFreeAsync on the solve's stream. */
typedef void *(*uc_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*uc_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);

typedef struct {
    double tol_rel_kkt;          /* relative KKT tolerance (default 1e-4, Sec. II-D) */
    double tol_abs_feas;         /* reported absolute feasibility threshold (default 1e-5) */
    int max_iter;                /* iteration limit (default 100000, Sec. II-D) */
    int n_eval;                  /* iterations between KKT / restart evaluations (default 64, even) */
    int use_graph;               /* 1: replay CUDA graphs of n_eval iterations (default 1) */
    int kernel_timing;           /* 1: time the primal and dual kernel of the middle iteration of every
                                    replay with events (graph path only) */
    double timeout_ms;           /* 0: none */
    const double *warm_x;        /* nullable [n] presolved-space primal start (scaled) */
    const double *warm_y;        /* nullable [m] presolved-space dual start (scaled) */
    double warm_omega;           /* > 0: initial primal weight (e.g. the final omega of the solve the
                                    warm start comes from); <= 0: omega0 of the presolve */
    uc_alloc_fn alloc;           /* nullable device allocator */
    uc_free_fn free;
    void *alloc_ctx;
    int spmv_kernel;             /* iteration kernels, one thread per row: 0 (default) rows in
                                    period-strided 16-row groups (in the device layout, 16 consecutive
                                    rows whose entry q is (col_q + s, val_q) in row s of the group, as
                                    for one constraint of one entity in consecutive periods) read the
                                    group's k <= 16 (column, value) slots instead of row pointers and
                                    CSR entries, the other rows their CSR row; 1: every row from CSR;
                                    2 staged: persistent CTAs that copy each 128-row chunk's matrix
                                    rows and vectors into shared memory ahead of use (Halpern only,
                                    rows of at most 640 entries, else UC_EINVAL).  The strided slots
                                    are not used by shared-matrix (lanes) sessions.  All variants give
                                    identical iterates. */
    int cta_rows;                /* threads per CTA of the iteration kernels: 0 (default 128), 128,
                                    256 or 512; results do not depend on it (tuning knob) */
    const int *rows_per_thread;  /* nullable [k]: rows each thread of LP i's CTAs handles, 1, 2 or
                                    4 (default 1); results do not depend on it (autotuned per size
                                    bucket, so LPs of one launch may differ) */
    int no_reorder;              /* 1: keep the LP's row/column order on the device.  Default: the
                                    layout of uc_presolved_device_order (entity-major, so a warp's
                                    gathers are contiguous, then sorted by length within 1024-row
                                    windows so warps see similar lengths); iterates are identical
                                    either way and results come back in the LP's order */
    int no_pdl;                  /* 1: launch iteration kernels without programmatic dependent
                                    launch (no overlap of consecutive kernels); default 0 */
    int algorithm;               /* 0 (default): restarted reflected Halpern PDHG; 1: PDLP iterate
                                    averaging with KKT restarts (both with constant step sizes) */
    int restart_metric;          /* Halpern restarts: 0 (default) weighted KKT of the map output,
                                    1 fixed-point residual of the last step, sqrt(omega |dx|^2 +
                                    |dy|^2 / omega); 2 that residual in the norm of the PDHG map's
                                    metric, sqrt(omega |dx|^2 + |dy|^2 / omega - 2 eta dy.A dx) */
    const volatile int *cancel;  /* nullable; a nonzero value (set from another thread) stops the
                                    solve at its next replay boundary with UC_ECANCELLED -- the
                                    "terminate the other solver" step of Alg. 1 */
    int stages;                  /* staged kernels: chunks in flight per CTA, 2..8 (0: default 2);
                                    results do not depend on it (tuning knob) */
    int lanes;                   /* 1: the session's 2 or 4 LPs share one scaled matrix (e.g. requests
                                    on one grid presolved with uc_presolve_reuse); it is stored once
                                    and the LPs' vectors are interleaved, so every row is read once
                                    for all of them (Halpern, row kernels; UC_EINVAL otherwise).
                                    Iterates are those of separate solves, bit for bit. */
    int adaptive_step;           /* 1: PDLP's adaptive step size (Applegate et al. 2021, Sec. 3.1) for
                                    algorithm 1: each iteration is an attempt with a trial step eta,
                                    accepted when eta <= ||dz||^2_omega / (2 |dy^T A dx|); next trial
                                    min((1 - (k+1)^-0.3) that bound, (1 + (k+1)^-0.6) eta), k = attempts
                                    so far; averages weighted by the accepted steps; attempts count as
                                    iterations (limit, evaluation period, restarts).  One LP per
                                    session, no lanes, row kernels; UC_EINVAL otherwise.  0: constant
                                    step (default) */
    double pw_kp, pw_ki, pw_kd;  /* primal-weight update at restarts, a PID controller on ln omega with
                                    error e = ln(omega dx / dy), dx and dy the primal and dual movement
                                    of the epoch: ln omega -= kp e + ki sum(e) + kd (e - e_prev).
                                    kp = 0.5, ki = kd = 0 is PDLP's rule.  Defaults: see
                                    uc_default_solve_opts */
    int polish;                  /* 1: primal feasibility polishing (uc_solve / uc_solve_batch, Halpern,
                                    no lanes): an LP whose result meets tol_rel_kkt but violates a row
                                    by more than tol_abs_feas (absolute, unscaled presolved LP; the
                                    paper's absolute feasibility tolerance, Sec. II-D) is iterated on
                                    with its objective cleared (c = 0), from the result's primal point,
                                    a zero dual and the final primal weight, until its largest row
                                    violation is at most tol_abs_feas.  The polished primal replaces
                                    the result's, the dual is kept, and the stats are those of the
                                    combined point.  0: off (default) */
    int polish_max_iter;         /* iteration limit of the polishing phase (0: 10000); if it is
                                    reached the result keeps its unpolished primal */
    double pw_guard;             /* residual-balance guard on the primal-weight update, kappa >= 1
                                    (0: off).  At a restart the controller's new omega is kept
                                    only if it moves toward balancing the relative residuals of the
                                    restart point: a decrease is dropped when rel_primal > kappa *
                                    rel_dual, an increase when rel_dual > kappa * rel_primal (a larger
                                    omega is a larger dual step, which works on primal
                                    infeasibility).  Halpern variant.  An LP without free columns
                                    (e.g. presolved with eliminate_angles) keeps its dual residual
                                    at rounding level, so the guard then blocks every decrease and
                                    should stay off.  UC_EINVAL for a negative, non-finite or (0, 1)
                                    value */
} uc_solve_opts;

typedef struct {
    int status;                  /* UC_OK, UC_EITERLIMIT, UC_ETIMEOUT, UC_ENUMERIC, UC_ECANCELLED,
                                    UC_EINFEASIBLE */
    int iters;                   /* PDHG iterations taken */
    int restarts;
    int evals;
    int returned_average;        /* 1 if the returned point is the iterate average */
    double rel_primal, rel_dual, rel_gap;  /* infinity-norm relative KKT parts (presolved LP) */
    double abs_primal;           /* max |primal violation| of the presolved LP (reported only) */
    double objective;            /* raw-LP objective of the returned point ($) */
    double dual_objective;       /* presolved dual objective + presolve constant */
    double omega;                /* final primal weight */
    double solve_ms;             /* device solve wall time (upload excluded) */
    double upload_ms;            /* host -> device copy and set-up */
    double primal_kernel_ms;     /* mean duration of the timed primal kernels (kernel_timing) */
    double dual_kernel_ms;       /* mean duration of the timed dual kernels (kernel_timing) */
    int timed_launches;          /* number of kernels each mean is over */
    int kernel_launches;         /* kernels launched by the session so far */
    int64_t h2d_bytes;           /* host -> device bytes of the session upload */
    int64_t d2h_bytes;           /* device -> host bytes of this result (+ status polls) */
    int rejected_steps;          /* adaptive step size: attempts that were rejected (else 0) */
    int polish_iters;            /* iterations of the polishing phase (0: not run) */
    int superbasic;              /* uc_crossover results: variables left strictly between their bounds
                                    (0: the point is a vertex) */
    double abs_primal_unpolished; /* abs_primal of the point before polishing */
} uc_stats;

void uc_default_presolve_opts(uc_presolve_opts *o);
void uc_default_solve_opts(uc_solve_opts *o);

/* Build the raw LP (model of Sec. II-A in DC form).  Columns per period t
 * (offset t*nc, nc = 3G+B+L(+B if voll>0)): p, u, v (G each), theta (B),
 * f (L), shed (B).  Rows: equality rows (bus balance, flow definition) for all
 * periods first, then ">=" rows (Pmax u - p, p - Pmin u, startup, ramp up,
 * ramp down).  Returns UC_EINVAL on bad data. */
int uc_build_lp(const uc_problem *prob, uc_lp **out);
int uc_lp_dims(const uc_lp *lp, int *n, int *m, int *m_eq, int64_t *nnz);
/* Copy the raw LP out (CSR, rows in order, columns ascending): rowptr [m+1],
 * colidx [nnz], val [nnz], q [m], c [n], l [n], u [n] (+-inf for free). */
int uc_lp_export(const uc_lp *lp, int32_t *rowptr, int32_t *colidx, double *val,
                 double *q, double *c, double *l, double *u);

/* Presolve (Sec. II-D, reduced form: fixed columns, singleton rows to bounds,
 * empty rows / columns; surviving rows and columns keep their order), then
 * scaling and the step size.  Host only, except the power iteration with
 * opts.power_device = 1.  UC_EINFEASIBLE / UC_EUNBOUNDED when presolve
 * proves it. */
int uc_presolve(const uc_lp *lp, const uc_presolve_opts *opts, uc_presolved **out);
/* Presolve `lp` reusing the scaling, scaled matrices and step size of `base`:
 * for an LP with the same grid and units as `base` (only loads differ), whose
 * raw matrix and presolve reductions are therefore identical.  The result is
 * what uc_presolve would give except that omega0 is recomputed from the new
 * q and c, while D_r, D_c, A_s and eta are the base's.  UC_EINVAL if the raw
 * matrix or the removed rows/columns differ.  Sessions accept it in
 * uc_session_update_lp for a slot that holds `base`. */
int uc_presolve_reuse(const uc_presolved *base, const uc_lp *lp, uc_presolved **out);
int uc_presolved_dims(const uc_presolved *ps, int *n, int *m, int *m_eq, int64_t *nnz);
/* Copy out the scaled reduced LP and its scaling: rowptr [m+1], colidx [nnz],
 * val [nnz] (FP64 scaled values), q, Dr [m], c, l, u, Dc [n], col_map [n] and
 * row_map [m] (raw indices), scalars [7] = {eta, omega0, power estimate of
 * ||A_s||_2, objective constant, ||q||_inf, ||c||_inf (both unscaled), the
 * bound eta is taken from}.  eta = 0.998 / bound, bound = max(estimate, U) with U
 * a certified upper bound on ||A_s||_2: 1 after the Pock-Chambolle pass (Schur
 * test), else sqrt(max row * max column absolute sum); the estimate alone is a
 * lower bound and could break PDHG's step condition tau sigma ||A||^2 < 1.  Any
 * pointer may be NULL to skip that array. */
int uc_presolved_export(const uc_presolved *ps, int32_t *rowptr, int32_t *colidx, double *val,
                        double *q, double *c, double *l, double *u, double *Dr, double *Dc,
                        int32_t *col_map, int32_t *row_map, double *scalars);

/* The layout a device session gives the presolved LP (host only, no device
 * needed): prow [m] and pcol [n] receive, for each device position in order, the
 * presolved row / column stored there.  With reorder != 0 (the solver's
 * default) rows and columns are sorted by the (kind, unit / bus / line, period)
 * label of the raw row or column they come from, equality rows first, so that
 * consecutive rows are one constraint of one entity in consecutive periods and
 * a warp's gathers read consecutive entries; then, within windows of 1024
 * positions, by decreasing number of entries (stable).  reorder = 0 gives the
 * identity.  UC_EINVAL on null pointers; the caller owns both arrays. */
int uc_presolved_device_order(const uc_presolved *ps, int reorder, int32_t *prow, int32_t *pcol);
/* Period-strided groups of the device layout of A (transpose = 0) or A^T (1),
 * host only.  Rows are taken in groups of 16 consecutive device rows; a group is
 * strided when its rows have one entry count k and, for each entry q, row s of
 * the group has device column col_q + s and value val_q.  counts [5] receives
 * groups, strided groups, entries, entries in strided groups and slots.  When
 * k, off, col and val are non-NULL they receive, per group, k (or -1) [groups],
 * the first slot [groups + 1], and per slot the first row's device column and
 * the shared value [slots]; call once with NULL arrays to size them. */
int uc_presolved_strided_groups(const uc_presolved *ps, int transpose, int64_t *counts, int32_t *k,
                                int32_t *off, int32_t *col, double *val);

/* Restarted, diagonally scaled PDHG on the device (Sec. II-C "PDHG (GPU)"),
 * stopping at relative KKT <= tol_rel_kkt (infinity norm, unscaled presolved
 * LP) or at max_iter.  `stream` is a cudaStream_t (NULL: legacy default).
 * The solve is synchronous: it returns when the device work has finished.
 * Returns the solve status; *out is set (and must be freed) whenever the
 * status is UC_OK, UC_EITERLIMIT, UC_ETIMEOUT, UC_ECANCELLED, UC_ENUMERIC or
 * UC_EINFEASIBLE (a Farkas direction was found; see uc_get_iterate). */
int uc_solve(const uc_presolved *ps, const uc_solve_opts *opts, void *stream, uc_result **out);

/* Solve k presolved LPs at once: their matrices are packed block-diagonally
 * (or, with opts->lanes, stored once for 2 or 4 LPs that share it) and every
 * iteration launches one primal and one dual kernel for all of them; each LP
 * keeps its own step sizes, restarts and stopping test and freezes when it
 * converges.  outs[i] receives LP i's result.  Returns UC_OK if every LP
 * reached the tolerance, else the first non-OK status. */
int uc_solve_batch(const uc_presolved *const *ps, int k, const uc_solve_opts *opts, void *stream,
                   uc_result **outs);

/* Device-resident sessions.  A session uploads k presolved LPs once (matrices
 * block-diagonal, or one shared matrix with interleaved vectors when
 * opts->lanes is set; per-LP vectors, start points, CUDA graph of n_eval
 * iterations) and then solves them any number of times; it is what uc_solve
 * and uc_solve_batch use internally, and what a server uses to keep
 * instances resident, warm-start re-solves and refill finished slots while
 * the other LPs keep iterating (continuous batching).  A session is used by
 * one host thread at a time; its device work runs on `stream`.
 *
 *   uc_session_create     upload; no LP runs until it is reset
 *   uc_session_reset      LP i (all if i < 0) back to its start point; the
 *                         initial KKT anchor is computed on the device
 *   uc_session_run        replay until every reset LP has stopped, or after
 *                         max_replays replays (<= 0: enough for max_iter);
 *                         *n_running = LPs still iterating; returns UC_OK,
 *                         UC_ECANCELLED or UC_ETIMEOUT (host-side stops)
 *   uc_session_status     1 idle, 2 iterating, else the LP's final status
 *   uc_session_result     copy LP i's state out as a uc_result (LP becomes idle)
 *   uc_session_set_start  warm start of LP i (scaled presolved space, [n], [m];
 *                         NULL = zeros) and its initial primal weight (omega > 0;
 *                         <= 0 keeps the presolve's omega0), used by the next reset
 *   uc_session_update_lp  replace slot i by an LP with the same scaled matrix
 *                         (e.g. the same grid and units with another load):
 *                         new q, c, l, u and scalars; the start point becomes
 *                         clip(0, l, u), y = 0.  UC_EINVAL if the matrix differs.
 *   uc_session_device_bytes  bytes of device memory the session holds */
int uc_session_create(const uc_presolved *const *ps, int k, const uc_solve_opts *opts, void *stream,
                      uc_session **out);
int uc_session_reset(uc_session *s, int i);
int uc_session_run(uc_session *s, int max_replays, int *n_running);
int uc_session_status(const uc_session *s, int i);
int uc_session_result(uc_session *s, int i, uc_result **out);
int uc_session_set_start(uc_session *s, int i, const double *x, const double *y, double omega);
int uc_session_update_lp(uc_session *s, int i, const uc_presolved *ps);
size_t uc_session_device_bytes(const uc_session *s);
void uc_session_free(uc_session *s);

/* Unscale and postsolve the returned point and split it: p, u, v [T*G];
 * theta, shed, lmp [T*B] (lmp = balance-row duals, $/MWh); f [T*L].  Any
 * array may be NULL.  stats may be NULL. */
int uc_get_solution(const uc_result *res, double *p, double *u, double *v, double *theta,
                    double *f, double *shed, double *lmp, uc_stats *stats);
/* Raw-LP primal [raw n] and dual [raw m] of the returned point. */
/* Crossover: from the returned point of a finished solve to a vertex (basic
 * solution) of the presolved LP -- the stage that follows PDHG in the paper's
 * GPU arm (Sec. II-C, Alg. 1 "Solver 1"; Sec. III-C).  Host only.  The point is
 * clipped to its bounds, phase 1 of a bounded revised simplex (dense basis
 * inverse, nonbasic variables allowed strictly inside their bounds) removes
 * the row residuals, phase 2 optimises, and a primal push moves every variable
 * left inside its bounds to a bound or into the basis.  *out is a new result
 * (free with uc_free_result) whose returned point is the vertex and whose dual
 * is the simplex multipliers; its stats carry the pivots in `iters`, the KKT
 * figures of the vertex and `superbasic` = 0 for a vertex.  max_pivots <= 0:
 * 50 (n + m).  UC_EINVAL for LPs with more than 20000 rows (the basis inverse
 * is dense) or a result without a returned point; UC_EITERLIMIT at the pivot
 * limit; UC_EINFEASIBLE when phase 1 ends with a residual; the caller keeps
 * `res`. */
int uc_crossover(const uc_result *res, int64_t max_pivots, uc_result **out);

/* The host simplex of uc_crossover from the cold start (each column at its
 * bound nearest 0, an artificial per row): an optimal vertex of the presolved
 * LP on the CPU, the CPU arm of uc_solve_concurrent.  cancel (nullable): a
 * nonzero value stops it at its next pivot with UC_ECANCELLED.  Same limits
 * and status codes as uc_crossover; stats.solve_ms is its wall time. */
int uc_simplex_solve(const uc_presolved *ps, int64_t max_pivots, const volatile int *cancel, uc_result **out);

/* Alg. 1 of the paper (Sec. II-C): the device PDHG (uc_solve with *opts, on
 * the calling thread) and the host simplex (uc_simplex_solve, on a second
 * thread) run at once on the same LP; the first to end optimal stops the other
 * through its cancel flag, and its result is returned (*winner: 0 device,
 * 1 host).  An arm that ends without an optimal result does not stop the
 * other; the host arm refuses LPs of more than 20000 rows, so on those the
 * device arm runs alone.  opts->cancel is replaced by the race's own flag. */
int uc_solve_concurrent(const uc_presolved *ps, const uc_solve_opts *opts, void *stream, uc_result **out,
                        int *winner);

/* A result holding a caller's point (x [n], y [m], scaled presolved LP, the
 * LP's own order; host memory, copied) with its KKT figures, e.g. to run
 * uc_crossover or uc_get_solution on a point from elsewhere.  Host only. */
int uc_result_from_point(const uc_presolved *ps, const double *x, const double *y, uc_result **out);

int uc_get_raw_solution(const uc_result *res, double *x, double *y);
/* Presolved-space, SCALED iterates: which = 0 current iterate, 1 the average
 * since the last restart (averaging variant) or the restart anchor (Halpern
 * variant), 2 returned point (Halpern: the last PDHG map output), 3 (status
 * UC_EINFEASIBLE only) the Farkas direction that proved the LP infeasible:
 * y_hat - y_in of the last step, x zeros; x [n], y [m].  Unscaled, the
 * direction is D_r y: y_I >= 0, -A^T D_r y lies in the cone the bounds allow
 * and its dual objective is positive, each up to a relative 1e-8. */
int uc_get_iterate(const uc_result *res, int which, double *x, double *y);

/* Device view of a presolved, scaled LP as uc_presolved_export returns it,
 * copied by the caller into device memory (every pointer is device memory):
 * A (m x n) and A^T (n x m) in CSR with FP64 values, the scaled c, l, u
 * (+-inf allowed) and column scales D_c [n], the scaled q and row scales
 * D_r [m]; rows [0, m_eq) are equalities, the rest ">="; q_inf and c_inf are
 * the unscaled infinity norms (scalars[4], scalars[5] of the export). */
typedef struct {
    int n, m, m_eq;
    const int32_t *A_rowptr, *A_colidx;
    const double *A_val;
    const int32_t *AT_rowptr, *AT_colidx;
    const double *AT_val;
    const double *c, *l, *u, *Dc;
    const double *q, *Dr;
    double q_inf, c_inf;
} uc_device_lp;

/* Relative KKT of a scaled presolved point (x [n], y [m], device memory) --
 * the same quantities the solver's own evaluation reports, NaN included --
 * computed WITHOUT ANY DEVICE ALLOCATION.  The paper has no counterpart: this
 * entry exists for callers that cannot allocate device memory, e.g. a process
 * whose device memory is all reserved ahead of time by its own pool allocator
 * (a fresh driver allocation would fail or fragment that pool), or a
 * latency-bound loop that must not enter the allocator (cudaMalloc and
 * cudaFree may synchronise the device).
 * Results go to `out`, 8 doubles of caller-owned device memory:
 * {rel_primal, rel_dual, rel_gap, KKT_omega (with the given omega > 0),
 *  primal objective, dual objective (both of the scaled presolved LP, no
 *  presolve constant), max |unscaled primal residual|, 0}.
 * Work is queued on `stream` (a cudaStream_t; NULL = legacy default) and the
 * call returns without waiting for it.
 * Scratch: a fixed array of 8192 x 8 doubles (512 KiB) in the library's
 * device image, held by every GPU that loads the library until exit.  LPs
 * with ceil(m/1024) + ceil(n/1024) > 8192 (about 8.4 million rows + columns)
 * are rejected with UC_EINVAL.  All calls share that array, so calls whose
 * device work overlaps (several streams or host threads at once) race and
 * must be serialised by the caller; no part of it needs to start at zero.
 * Set-up: every call looks up the array's device address for the current
 * device (cudaGetSymbolAddress, which allocates nothing), so a context that was
 * reset and re-created never gets a stale address, and makes sure the entry's
 * two kernels are loaded (cudaFuncGetAttributes).  Under CUDA's lazy module
 * loading the driver may take device memory for their code on the first call
 * on each device (and on the first call after a cudaDeviceReset); make that
 * first call before starting any stream capture.  No cudaMalloc, cudaFree or
 * other allocating call is made. */
int uc_kkt_noalloc(const uc_device_lp *lp, const double *x, const double *y, double omega, double *out,
                   void *stream);

void uc_free_lp(uc_lp *lp);
void uc_free_presolved(uc_presolved *ps);
void uc_free_result(uc_result *res);
const char *uc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* UC_PDHG_H */
