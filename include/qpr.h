/*
 * qpr.h -- C ABI of the GB300 quantum PageRank solver.
 *
 * The solver integrates the quantum-stochastic-walk Lindblad equation
 * (Eq. 1 / Eq. S7 of "TensorFlow Solver for Quantum PageRank in Large-Scale
 * Networks")
 *
 *   d rho/dt = -(1-omega) i [H, rho]
 *              + omega sum_ij ( L_ij rho L_ij^dag - 1/2 {L_ij^dag L_ij, rho} ),
 *   L_ij = sqrt(G_ij) |i><j|,
 *
 * directly on the N x N complex density matrix with classical RK4
 * (Supplementary Note 2, fourth-order scheme), never forming the N^2 x N^2
 * superoperator of Eq. 2. H and G come from a weighted directed edge list
 * (Supplementary Note 1): A_ij = w for a link j -> i, H_ij = -max(A_ij, A_ji)
 * (Eq. S6), G = alpha S + (1 - alpha) F with S the column-normalised
 * adjacency and F_ij = 1/(N-1) off the diagonal (Eq. S2, Eq. S4).
 *
 * Conventions shared by every entry point:
 *   - A density matrix is N x N complex128, row-major, (re, im) interleaved
 *     (the layout of a C99 `double complex` array or a torch.complex128
 *     tensor). A rho argument may point to device memory or to host memory
 *     (pageable or pinned); the library detects which and copies as needed.
 *   - Every input density matrix is first made exactly Hermitian,
 *     (rho + rho^dag)/2, and divided by its real trace; every output density
 *     matrix has unit real trace.
 *   - All work runs on the context's CUDA stream (qpr_options.cuda_stream, or
 *     a stream the context creates). The calls return when their results are
 *     complete and visible to the host.
 *   - Entry points never abort and never trap. They return a status; the
 *     message of the last failure is qpr_last_error(ctx). After a CUDA error
 *     the context is poisoned: every later call returns QPR_E_CUDA.
 *   - Memory passed in is owned by the caller; the context owns its own
 *     device buffers until qpr_destroy.
 */
#ifndef QPR_H
#define QPR_H

#include <stdint.h>

#if defined(__GNUC__)
#define QPR_API __attribute__((visibility("default")))
#else
#define QPR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qpr_ctx qpr_ctx;

typedef enum {
    QPR_OK = 0,
    QPR_E_ARG = 1,           /* invalid argument (null pointer, dt <= 0, alpha/omega outside [0,1], ...) */
    QPR_E_GRAPH = 2,         /* invalid edge list (index outside [0,n), negative or non-finite weight) */
    QPR_E_CUDA = 3,          /* CUDA runtime error; the context is poisoned */
    QPR_E_OOM = 4,           /* device or host allocation failed */
    QPR_E_UNSTABLE = 5,      /* dt outside the RK4 stability estimate (qpr_evolve only) */
    QPR_E_NOT_CONVERGED = 6, /* max_steps reached before the residual fell below tol */
    QPR_E_TIMEOUT = 7,       /* a device-side wait gave up (the context is not poisoned) */
    QPR_E_NONFINITE = 8      /* a NaN or Inf appeared in the state or the residual */
} qpr_status;

/* Arithmetic of the RK4 stages.
 * QPR_FP64: every stage in FP64 (the plain form).
 * QPR_MIXED: RK4 in delta form against an exact FP64 reference. Every
 *   ref_refresh steps the state is renormalised, R = y / tr(y), and F = f(R)
 *   is evaluated exactly in FP64, which also gives the exact residual ||F||_F.
 *   In between, each stage evaluates only f(Y_s - R) (f is linear) in FP32
 *   (or split BF16 on tensor cores for the dense backend), and the RK
 *   accumulation of the delta y - R is carried in float-float (two FP32
 *   planes, about 48 bits); y = R + delta is formed in FP64 at each refresh.
 *   A residual that passes the FP32-accurate
 *   per-step estimate is confirmed by an exact FP64 refresh before the solve
 *   stops, so the returned state satisfies the FP64 stop rule. */
enum { QPR_FP64 = 0, QPR_MIXED = 1 };
/* Diagonal of H. Eq. S6 prints H_ii = -outDeg(i); the symmetrised-adjacency
 * form with a zero diagonal is the default because the printed diagonal
 * makes RK4 at dt = 0.01 unstable on heavy-tailed weighted graphs. */
enum { QPR_HDIAG_ZERO = 0, QPR_HDIAG_NEG_OUTDEG = 1 };
/* Column of S for a node without out-links: F's column, 1/(N-1) off the
 * diagonal (default), or the uniform column 1/N. */
enum { QPR_DANGLING_F = 0, QPR_DANGLING_UNIFORM = 1 };
/* How the O(N^2)-per-row product H rho of each RK4 stage is formed.
 * DENSE: tensor-core GEMM of the dense N x N H against [Re rho | Im rho]
 * (4 N^3 flops per stage). SPARSE: CSR H times rho in FP64 (4 nnz(H) N
 * flops per stage, bandwidth bound). AUTO picks SPARSE when H has fewer than
 * N^2 / 8 nonzeros. Both produce the same FP64 right-hand side up to
 * summation order. */
enum { QPR_BACKEND_AUTO = 0, QPR_BACKEND_DENSE = 1, QPR_BACKEND_SPARSE = 2 };
/* Form of the FP32 stage of QPR_MIXED with the sparse backend.
 * COLUMNS: per stage a column-block product X = H (Y_s - R), each CTA
 *   staging 16 complex columns of the delta in shared memory with TMA, then
 *   a tile-pair epilogue: 2 launches per stage (the product grid's leading
 *   CTAs form the gain G p on the SMs the product leaves free); where the
 *   staged operands fit one CTA's shared memory (N padded to 32 <= 1536).
 * COLUMNS_PERSISTENT: the same arithmetic in one cooperative launch per
 *   block of ref_refresh steps, grid barriers between the phases (needs
 *   cooperative launch support).
 * TILES: one launch per stage; each 32 x 32 tile pair gathers, from L2, the
 *   row slices of the delta that its rows' nonzeros select.
 * COLUMNS_GATHER: the column-block product for any N without staging the
 *   block: each CTA (row split r, block J of 32 columns) stages only its CSR
 *   entries and reads every nonzero's 32 values of block J through L1 and
 *   L2 (one 128-byte line per plane); the splits of a block run side by
 *   side, so the block is read from DRAM about once.
 * AUTO (default): COLUMNS where it applies, else COLUMNS_GATHER, else TILES.
 * COLUMNS and COLUMNS_PERSISTENT give bitwise the same results (each row's
 * products summed in entry order); COLUMNS_GATHER and TILES differ from them
 * only in FP32 summation order. (Value 4 is not used.) */
enum {
    QPR_SPARSE_FORM_AUTO = 0,
    QPR_SPARSE_FORM_COLUMNS = 1,
    QPR_SPARSE_FORM_TILES = 2,
    QPR_SPARSE_FORM_COLUMNS_PERSISTENT = 3,
    QPR_SPARSE_FORM_COLUMNS_GATHER = 5
};

typedef struct {
    int32_t precision;   /* QPR_FP64 (default) or QPR_MIXED */
    int32_t h_diag;      /* QPR_HDIAG_ZERO (default) or QPR_HDIAG_NEG_OUTDEG */
    int32_t dangling;    /* QPR_DANGLING_F (default) or QPR_DANGLING_UNIFORM */
    int32_t graph_steps; /* RK4 steps per captured CUDA graph launch (default 32; 0 = no graphs) */
    void *cuda_stream;   /* cudaStream_t the caller's inputs are ordered on (NULL = legacy default stream) */
    int32_t device;      /* CUDA device ordinal (default -1: the current device) */
    int32_t backend;     /* QPR_BACKEND_AUTO (default), QPR_BACKEND_DENSE or QPR_BACKEND_SPARSE */
    int32_t ref_refresh; /* QPR_MIXED: steps between exact FP64 reference refreshes (default 32) */
    int32_t sparse_form; /* QPR_MIXED, sparse backend: QPR_SPARSE_FORM_* (default AUTO) */
    int32_t test_fault;  /* testing only (default 0). 1: every grid barrier of the COLUMNS_PERSISTENT
                            form waits for one arrival more than its grid makes, so each wait
                            gives up after its time limit (about a second) and the call returns
                            QPR_E_TIMEOUT; the context stays usable. Other forms ignore it. */
    int32_t row_splits;  /* COLUMNS, COLUMNS_GATHER: row splits of the product, at least this many
                            (default 0: chosen by the plan; at most 16, 64 for the gather form) */
    int32_t adaptive_refresh; /* QPR_MIXED steady-state solves: 1 (default) lengthens the window between
                            refreshes as the residual falls, up to 8 x ref_refresh steps, while
                            (steps since the refresh)^2 x residual <= ref_refresh^2 x the first
                            residual; 0: a refresh every ref_refresh steps. Trajectories always
                            refresh every ref_refresh steps. */
    int32_t reserved[1];
} qpr_options;

typedef struct {
    int64_t steps;       /* RK4 steps taken (the step index n at which the residual passed) */
    int64_t substeps_m;  /* dt was split into m equal substeps for stability */
    double t;            /* integrated time, steps * dt / m */
    double residual;     /* ||f(rho_n)||_F of the returned state (FP64) */
    double trace_before; /* Re tr of the unnormalised state before the last division */
    double seconds;      /* wall time of the call */
    int64_t kernel_launches; /* kernels this call launched (early-exit launches included) */
    int32_t converged;   /* 1 if residual < tol */
    int32_t reserved[3];
} qpr_stats;

/* Fill *opt with the defaults listed above. */
QPR_API qpr_status qpr_default_options(qpr_options *opt);

/* Build a solver context from a weighted directed edge list.
 * n       number of nodes (>= 2; F needs N - 1 > 0, Eq. S2).
 * m       number of edges (>= 0); edge e is the link src[e] -> dst[e] with
 *         weight w[e] (w == NULL: unit weights). Host arrays.
 * alpha   damping of the Google matrix, in [0, 1] (Eq. S4's q).
 * omega   quantum/classical mixing, in [0, 1] (Eq. 1).
 * Duplicate links sum their weights; self-loops and zero weights are dropped.
 * Errors: QPR_E_ARG (n < 2, alpha/omega outside [0,1], null pointers),
 * QPR_E_GRAPH (index outside [0,n), weight negative or not finite),
 * QPR_E_OOM, QPR_E_CUDA. On error *out is NULL. */
QPR_API qpr_status qpr_create(qpr_ctx **out, int64_t n, int64_t m, const int64_t *src, const int64_t *dst,
                      const double *w, double alpha, double omega, const qpr_options *opt);

/* Free the context and its device buffers. NULL is ignored. */
QPR_API void qpr_destroy(qpr_ctx *ctx);

/* Message of the last failure on this context ("" if none). ctx may be NULL
 * (the message of the last failed qpr_create on this thread). */
QPR_API const char *qpr_last_error(const qpr_ctx *ctx);
QPR_API const char *qpr_status_string(qpr_status s);

/* Number of nodes and the estimated spectral spread lambda_max - lambda_min
 * of H used by the RK4 step-size check. qpr_backend: the backend in use
 * (QPR_BACKEND_DENSE or QPR_BACKEND_SPARSE). qpr_sparse_form: the form of
 * the FP32 sparse stage in use (QPR_SPARSE_FORM_COLUMNS,
 * _COLUMNS_PERSISTENT, _COLUMNS_GATHER or _TILES; 0 when the context is not
 * QPR_MIXED with the sparse backend). */
QPR_API int64_t qpr_n(const qpr_ctx *ctx);
QPR_API int32_t qpr_backend(const qpr_ctx *ctx);
QPR_API int32_t qpr_sparse_form(const qpr_ctx *ctx);
/* Geometry of the column-block product in use, into out[4]: row splits,
 * complex columns per column block (16 for COLUMNS and COLUMNS_PERSISTENT,
 * 32 for COLUMNS_GATHER), CTAs of one product launch (column blocks x row
 * splits) and the product kernel's dynamic shared memory in bytes. All 0
 * for the tile-pair form.
 * Errors: QPR_E_ARG (ctx or out NULL). */
QPR_API qpr_status qpr_sparse_plan(const qpr_ctx *ctx, int32_t *out);
QPR_API double qpr_h_spread(const qpr_ctx *ctx);

/* Largest dt for which the context considers one RK4 step stable: it needs
 * dt * ((1 - omega) * spread(H) + 2 omega) <= 2.5, a half-disk inside RK4's
 * stability region. */
QPR_API double qpr_max_stable_dt(const qpr_ctx *ctx);

/* out = f(rho), one evaluation of the Lindblad right-hand side (Eq. S7) on
 * the Hermitian part of rho, without trace normalisation. rho and out: N x N
 * complex128, host or device; they may not alias. */
QPR_API qpr_status qpr_rhs(qpr_ctx *ctx, const void *rho, void *out);

/* *resid_out = ||f(rho)||_F over all N^2 entries, in FP64, for the
 * Hermitian part of rho, without trace normalisation. */
QPR_API qpr_status qpr_residual(qpr_ctx *ctx, const void *rho, double *resid_out);

/* Fixed-step RK4: rho <- the state after `steps` steps of length dt, each
 * step followed by division by the real trace. rho is read and overwritten
 * in place (host or device). QPR_E_UNSTABLE if dt exceeds
 * qpr_max_stable_dt(ctx). steps == 0 returns the normalised input. */
QPR_API qpr_status qpr_evolve(qpr_ctx *ctx, void *rho, double dt, int64_t steps);

/* RK4 from the initial state in rho (for example I/N) until the first step
 * index n with ||f(rho_n)||_F < tol, or
 * until max_steps steps were taken. rho_n (unit trace) is written back to
 * rho. If dt exceeds the stability estimate, each step is split into the
 * smallest number m of equal substeps that passes; stats->substeps_m
 * reports m and steps counts substeps.
 * Returns QPR_OK when converged, QPR_E_NOT_CONVERGED when max_steps was
 * reached (rho then holds the last state), QPR_E_NONFINITE on NaN/Inf.
 * out may be NULL. */
QPR_API qpr_status qpr_steady_state(qpr_ctx *ctx, void *rho, double dt, double tol, int64_t max_steps,
                            qpr_stats *out);

/* Per-kernel timing of the RK4 step, for roofline measurements (the paper
 * has no counterpart). Runs `steps` RK4 steps (steps >= 1) from rho (rho
 * itself is not modified) on the context's stream without CUDA graphs and
 * without programmatic dependent launch: every kernel runs alone, between
 * two CUDA events, so each time below is one kernel's own duration (plus
 * the launch and event granularity, about a microsecond), not the
 * overlapped time of the solve's graph launches (there the SpMM grid and the
 * epilogue overlap their prologues with the previous kernel).
 * Means over all launches of the kind, in milliseconds. */
typedef struct {
    double product_ms;   /* the H rho product: the column-block SpMM (COLUMNS, COLUMNS_PERSISTENT) or
                            gather SpMM (COLUMNS_GATHER), whose leading CTAs also form the gain; the fused
                            stage kernel of the other forms (product and epilogue in one launch) */
    double epilogue_ms;  /* the epilogue kernel of the two-kernel column-block forms; 0 otherwise */
    double gain_ms;      /* the gain kernel G p (0 where the product or stage kernel forms the gain) */
    double refresh_ms;   /* QPR_MIXED: one exact FP64 reference refresh, all its kernels; 0 otherwise */
    double step_ms;      /* the kernels of one RK4 step run one at a time (the sum of the above) */
    int32_t launches_per_step;
    int32_t reserved[3];
} qpr_profile;

QPR_API qpr_status qpr_profile_step(qpr_ctx *ctx, const void *rho, double dt, int64_t steps, qpr_profile *out);

/* The same kernels inside a chain of launches with programmatic dependent
 * launch, as the solve runs them (for roofline measurements; the paper has
 * no counterpart). From rho (not modified) it runs one exact refresh and
 * stage 1, then launches the stage-2 SpMM grid `reps` times back to back
 * (each launch reads the same stage input and writes the same X and gain)
 * and the stage-2 epilogue `reps` times (each reads X and the stage input
 * and writes the same next stage input), each launch allowed to start its
 * prologue while the previous one finishes, with CUDA events around each
 * chain on the context's stream. out_ms[0] = mean time per SpMM launch,
 * out_ms[1] = per epilogue launch (milliseconds; 2 doubles, host). QPR_MIXED
 * with a column-block form (COLUMNS, COLUMNS_PERSISTENT's kernels,
 * COLUMNS_GATHER) only, else QPR_E_ARG; reps in [1, 4096]. */
QPR_API qpr_status qpr_profile_chain(qpr_ctx *ctx, const void *rho, double dt, int32_t reps, double *out_ms);

/* p[i] = Re rho_ii (the probability at node i); p: N doubles, host or
 * device. rank (nullable): N int64 node indices in descending order of p,
 * ties to the lower index (the ranking of the main text's airline study). */
QPR_API qpr_status qpr_populations(qpr_ctx *ctx, const void *rho, double *p, int64_t *rank);

/* ---- adaptive RKF45 (the paper's own integrator) ----
 * The RKF45 scheme of Supplementary Note 2: per attempt of step h the six
 * stages of Eq. S10, the fourth-order solution y_{k+1} (Eq. S11) and the
 * fifth-order solution z_{k+1} (Eq. S12), with the printed 845/4101 and
 * 2197/4101 read as 845/4104 and 2197/4104 (the values for which each stage
 * row sums to its node and the weights of Eq. S11 sum to one), and the step
 * factor s = (Tol h / (2 |z_{k+1} - y_{k+1}|))^(1/4) of Eq. S13. Readings
 * where the note is silent: |.| is the largest modulus over the N^2 entries;
 * an attempt is accepted when |z - y| <= Tol h, and y_{k+1} (or z_{k+1},
 * order 5) becomes the state; after every attempt h <- min(s h, h_max) with s
 * clipped to [1/10, 4]; a trajectory's last step ends exactly at t_end.
 * Both fourth- and fifth-order propagated solutions are slightly anti-damping
 * near the imaginary axis (|P4(iy)| up to 1.03, |P5(iy)| up to 1.004 for y
 * below about 2.3), which the coherences' damping omega h must offset: with
 * order 4 steady-state solves stall near a residual of 1e-4 for omega <= 0.6
 * on the heavy-tailed graphs, with order 5 only below omega ~ 0.3; fixed-step
 * RK4 (qpr_steady_state) has no such limit.
 * Computed in the mixed delta form of QPR_MIXED on the column-block sparse
 * stage (COLUMNS, COLUMNS_PERSISTENT or COLUMNS_GATHER; else QPR_E_ARG): f is
 * linear, so an attempt is the polynomial P4(hL) (y) and the discrepancy
 * (P5 - P4)(hL) y, formed from the six powers (hL)^k y in FP32 with the
 * state in float-float against the exact FP64 reference; the step-size
 * controller runs on the device; the state is renormalised at every exact
 * refresh (each block of ref_refresh attempts). The paper has no
 * tolerance; Tol and h_max are the caller's. */
typedef struct {
    double h0;       /* first step (<= 0: 0.01; clipped to h_max) */
    double step_tol; /* Tol of Eq. S13 (<= 0: 1e-6) */
    double h_max;    /* largest step (<= 0: qpr_max_stable_dt(ctx), the RK4 stability estimate, which also
                        keeps RKF45's fourth-order solution stable on these problems) */
    double t_end;    /* > 0: integrate the trajectory to this time; <= 0: solve for the steady state */
    int32_t order;   /* the solution an accepted attempt keeps: 4 (or 0, default) y_{k+1} of Eq. S11, which
                        the note names the approximation; 5 z_{k+1} of Eq. S12, the alternative it offers */
    int32_t reserved[3];
} qpr_rkf45_options;

typedef struct {
    int64_t accepted;        /* accepted steps (the state's step index) */
    int64_t rejected;        /* rejected attempts */
    double t;                /* integrated time */
    double h_next;           /* the step the next attempt would take */
    double residual;         /* ||f(rho)||_F of the returned state (FP64, exact) */
    double last_discrepancy; /* |z - y| of the last attempt */
    double seconds;          /* wall time of the call */
    int64_t kernel_launches;
    int32_t converged;       /* 1: steady state below tol, or t_end reached */
    int32_t reserved[3];
} qpr_rkf45_stats;

/* RKF45 from the state in rho (host or device, overwritten with the result,
 * unit trace). Steady state (opt->t_end <= 0): until the first accepted state
 * with ||f||_F < tol, confirmed in FP64, or max_steps accepted steps.
 * Trajectory (t_end > 0): to time t_end (tol ignored), at most max_steps
 * accepted steps. Attempts are bounded by 16 max_steps + 64 ref_refresh.
 * Returns QPR_OK, QPR_E_NOT_CONVERGED, QPR_E_NONFINITE, QPR_E_ARG,
 * QPR_E_TIMEOUT, QPR_E_CUDA, QPR_E_OOM (the first call allocates the form's
 * extra buffers). opt and out may be NULL. */
QPR_API qpr_status qpr_rkf45(qpr_ctx *ctx, void *rho, const qpr_rkf45_options *opt, double tol, int64_t max_steps,
                             qpr_rkf45_stats *out);

/* ---- classical PageRank and hub classes ----
 * The main text compares the quantum PageRank ranking of the airline network
 * with the classical PageRank and sorts nodes into hubs (its airline-ranking
 * paragraph: main hubs above c/N, secondary hubs between 1/N and c/N, with
 * c = 10).
 *
 * qpr_pagerank: the classical PageRank pi of the context's graph, the
 * stationary vector of G = alpha S + (1 - alpha) F (Eq. S4, Eq. S2): G pi =
 * pi, sum pi = 1 (also the populations of the omega = 1 steady state). Power
 * iteration in FP64 on the device from the uniform vector, each iterate
 * divided by its sum, until the L1 change of one iteration is below tol
 * (checked every 8 iterations) or max_iter iterations. pi: N doubles, host or
 * device; iters (nullable): the iterations run. Returns QPR_OK,
 * QPR_E_NOT_CONVERGED (pi then holds the last iterate), QPR_E_NONFINITE,
 * QPR_E_ARG (tol <= 0, max_iter < 1, pi NULL), QPR_E_CUDA.
 *
 * qpr_hub_classes: classes[i] = 2 for a main hub (p_i > c/N), 1 for a
 * secondary hub (1/N < p_i <= c/N; the text leaves the side of the
 * equalities open), 0 otherwise, for any probability vector p of the
 * context's N nodes (the populations from qpr_populations, or pi). p: N
 * doubles, host or device; classes (nullable): N int32, host or device;
 * counts (nullable, host): the number of nodes in classes 0, 1, 2. c >= 1.
 * Returns QPR_OK, QPR_E_ARG, QPR_E_CUDA. */
QPR_API qpr_status qpr_pagerank(qpr_ctx *ctx, double tol, int64_t max_iter, double *pi, int64_t *iters);
QPR_API qpr_status qpr_hub_classes(qpr_ctx *ctx, const double *p, double c, int32_t *classes, int64_t *counts);

/* ---- many problems in one batched run ----
 * One problem of a batch: a weighted edge list (as in qpr_create), its own
 * omega, and its density matrix rho (N x N complex128, host or device),
 * read as rho0 and overwritten with the steady state. */
typedef struct {
    int64_t n;
    int64_t m;
    const int64_t *src;
    const int64_t *dst;
    const double *w; /* NULL: unit weights */
    double omega;
    void *rho;
} qpr_problem;

/* Steady states of `count` independent problems (graphs of any sizes and
 * omegas, shared alpha, dt, tol and options), integrated together by the
 * mixed-precision RK4 form on the sparse backend (QPR_MIXED; options
 * h_diag, dangling, ref_refresh, adaptive_refresh, device and cuda_stream
 * apply). Each block of ref_refresh steps (with the exact refreshes that
 * are due) is one captured CUDA graph over work lists of every problem still
 * running: the column-block SpMM units in size classes of the padded edge
 * (one launch each, with the class's own shared memory), the tile pairs of
 * the epilogues. A problem whose exact FP64 residual passes tol (or that
 * reaches max_steps) is retired on the device at once (its kernels return
 * immediately) and leaves the lists when they are rebuilt. Every problem's
 * result is bitwise the one qpr_steady_state returns for it alone with
 * QPR_MIXED, QPR_BACKEND_SPARSE and the same stage form (COLUMNS where the
 * whole column block fits, N padded to 32 <= 1536; TILES above).
 * stats (nullable) receives one entry per problem
 * (seconds and kernel_launches are those of the whole call). Returns
 * QPR_OK when every problem converged, QPR_E_NOT_CONVERGED when some
 * reached max_steps, QPR_E_NONFINITE, QPR_E_ARG / QPR_E_GRAPH (message of
 * qpr_last_error(NULL) names the problem), QPR_E_OOM, QPR_E_CUDA,
 * QPR_E_TIMEOUT. Synchronous. */
QPR_API qpr_status qpr_batch_steady_state(int64_t count, const qpr_problem *problems, double alpha, double dt,
                                          double tol, int64_t max_steps, const qpr_options *opt, qpr_stats *stats);

/* ---- autotuner ----
 * Chooses, for one problem and one precision, the configuration of the
 * stage by timing short real runs (qpr_evolve from I/N, 4 warm-up steps,
 * then max(32, 2 ref_refresh) timed steps) of every candidate on the device.
 * The paper has no counterpart. QPR_MIXED: the backend (sparse, or the
 * split-BF16 tcgen05 dense stage), for the sparse backend the stage form
 * (COLUMNS with row splits 1-4 and the plan's own choice, COLUMNS_GATHER
 * with the plan's splits, half and twice as many, TILES; candidates whose
 * plan repeats an earlier one are skipped), then ref_refresh in
 * {16, 32, 64} for the winner. QPR_FP64: the backend (CSR gathers or DMMA).
 * With cache_path (nullable) the choice is read from / appended to a text
 * file keyed by GPU name, precision, floor(log2 N) and
 * floor(log2(nnz(H)/N + 1)); a cached answer sets from_cache. `base`
 * supplies the other options (NULL: defaults); a context created with base
 * plus backend, sparse_form, row_splits and ref_refresh from the result runs
 * the chosen configuration. */
typedef struct {
    int32_t backend;
    int32_t ref_refresh;
    double ms_per_step;  /* measured wall time of one step of the chosen configuration */
    int32_t from_cache;
    int32_t sparse_form; /* QPR_MIXED sparse: the chosen QPR_SPARSE_FORM_* (AUTO otherwise) */
    int32_t row_splits;  /* the chosen row splits (0: the plan's own choice) */
    int32_t reserved[1];
} qpr_tune_result;

QPR_API qpr_status qpr_autotune(int64_t n, int64_t m, const int64_t *src, const int64_t *dst, const double *w,
                                double alpha, double omega, double dt, const qpr_options *base,
                                const char *cache_path, qpr_tune_result *out);

/* ---- learned warm start ----
 * A 4-layer message-passing network (width 64, BF16 weights, FP32
 * accumulation) that predicts the steady-state populations from the graph;
 * rho0 = diag(p_hat) then starts qpr_steady_state near its fixed point,
 * while rho0 = I/N stays the fallback. The paper has no learned component;
 * the network serves only as an initial guess, and the stop rule of the
 * solver decides the answer. Definition of features, layers and loss:
 * features [1, omega, log1p(in-strength), log1p(out-strength),
 * log1p(in-degree), log1p(out-degree), log(N pi_i), dangles] with pi the
 * classical PageRank (the omega = 1 steady state); layers
 * z = h Ws + (P h) Wn + b, h = relu(z) with P the row-normalised A + A^T;
 * p_hat = softmax(h_4 wo + bo); loss -sum_i p_i log p_hat_i.
 * Parameters: qpr_gnn_param_count() floats in the order Ws1 [8][64],
 * Wn1 [8][64], b1 [64], then Ws, Wn [64][64] and b [64] of layers 2-4, then
 * wo [64], bo [1]. */
typedef struct qpr_gnn qpr_gnn;

/* One training sample: a graph (as in qpr_create), its omega and the target
 * populations p (host, n doubles, summing to 1). */
typedef struct {
    int64_t n;
    int64_t m;
    const int64_t *src;
    const int64_t *dst;
    const double *w;
    double omega;
    const double *p;
} qpr_gnn_sample;

QPR_API int64_t qpr_gnn_param_count(void);
/* Glorot-uniform weights from `seed`, zero biases; device < 0: current. */
QPR_API qpr_status qpr_gnn_create(qpr_gnn **out, uint64_t seed, int32_t device);
QPR_API void qpr_gnn_destroy(qpr_gnn *g);
/* Copy the FP32 master parameters out of / into the network (host arrays of
 * qpr_gnn_param_count() floats); setting resets the Adam state. */
QPR_API qpr_status qpr_gnn_get_params(qpr_gnn *g, float *host_params);
QPR_API qpr_status qpr_gnn_set_params(qpr_gnn *g, const float *host_params);
/* p_hat (n doubles, host or device) for a graph and omega. */
QPR_API qpr_status qpr_gnn_predict(qpr_gnn *g, int64_t n, int64_t m, const int64_t *src, const int64_t *dst,
                                   const double *w, double alpha, double omega, double *p_hat);
/* Loss of one sample and its gradient with respect to the parameters
 * (host outputs; grad: qpr_gnn_param_count() floats, nullable). */
QPR_API qpr_status qpr_gnn_loss_grad(qpr_gnn *g, const qpr_gnn_sample *sample, double alpha, double *loss,
                                     float *grad);
/* Adam (beta 0.9 / 0.999, eps 1e-8) on the mean gradient of minibatches of
 * `batch` samples, `epochs` passes in an order shuffled from `seed`;
 * epoch_loss (nullable, `epochs` doubles) receives the mean loss of each
 * pass. */
QPR_API qpr_status qpr_gnn_train(qpr_gnn *g, int64_t count, const qpr_gnn_sample *samples, double alpha,
                                 int32_t epochs, int32_t batch, double lr, uint64_t seed, double *epoch_loss);

/* ---- right-hand side without any allocation ----
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc: hosts that hand out all device memory from
 * their own pool and forbid libraries from allocating, services held to a
 * fixed device-memory budget, and code that must not allocate after
 * start-up. It computes out = f(rho) exactly as qpr_rhs does (sparse CSR
 * stage kernel), but every input and output is the caller's and the scratch
 * lives in a file-scope __device__ array sized for N <= QPR_NOALLOC_MAX_N
 * (about 2.1 MB, resident on every device that loads the library until the
 * process exits). It calls no cudaMalloc, cudaFree or other allocating
 * routine.
 *
 * n            nodes, 2 <= n <= QPR_NOALLOC_MAX_N (else QPR_E_ARG).
 * h_ptr/h_col/h_val   CSR of H (Eq. S6) on the device: n + 1 row pointers,
 *              column indices, values, rows in any column order.
 * s_ptr/s_col/s_val   CSR of S on the device, the column-normalised
 *              adjacency A_ij / outDeg(j), holding only columns j with
 *              outDeg(j) > 0; dangling_flags (n bytes, device) marks the
 *              columns without out-links, which take F's column
 *              (QPR_DANGLING_F) or the uniform column (QPR_DANGLING_UNIFORM).
 * alpha, omega in [0, 1].
 * rho, out     N x N complex128 row-major on the device; must not alias.
 * cuda_stream  stream the work is queued on (NULL: legacy default stream).
 * The call only queues work and returns; out is ready when the stream
 * reaches that point. Errors: QPR_E_ARG (n outside [2, QPR_NOALLOC_MAX_N], a
 * NULL pointer, alpha/omega/dangling_mode out of range), QPR_E_CUDA.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture. All calls on a device share the scratch array
 * and each leaves its contents behind; calls whose GPU work overlaps (other
 * streams, other threads) race on it and must be serialised by the caller. */
#define QPR_NOALLOC_MAX_N 256
QPR_API qpr_status qpr_rhs_noalloc(int64_t n, const int32_t *h_ptr, const int32_t *h_col, const double *h_val,
                                   const int32_t *s_ptr, const int32_t *s_col, const double *s_val,
                                   const uint8_t *dangling_flags, double alpha, double omega,
                                   int32_t dangling_mode, const void *rho, void *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* QPR_H */
