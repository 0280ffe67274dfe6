/*
 * pdr.h -- C ABI of libpdr, a GB300 (sm_103a) implementation of Potential
 * Difference Reduction (PDR) for the multicommodity-flow feasibility problem.
 *
 * Paper: P. Liu, "A Localized Method for Multicommodity Flow Problem",
 * arXiv 2108.07549.  Section numbers, equations and algorithms below refer
 * to it.
 *
 * Problem (eq. (1)): a directed graph G(V, E) with n vertices and m edges,
 * capacities u_e >= 0, and K commodities (s_k, t_k, d_k) with s_k != t_k and
 * d_k > 0.  A flow f_e,k >= 0 is feasible when sum_k f_e,k <= u_e on every
 * edge and every commodity is conserved with supply d_k at s_k and demand
 * d_k at t_k.
 *
 * Method (Section 4, Alg. 1 with the edge solver of Alg. 2): starting from
 * f = 0, every sweep computes the excess Delta_ik (eq. (3), (3h)), the
 * heights h_ik = Delta_ik / delta_i (eq. (2)), the congestion
 * psi_e = max(0, sum_k f_e,k - u_e) (eq. (41)) and the objective
 * z = 1/2 sum psi^2 + 1/2 sum delta_i h^2; it stops when a stop rule fires,
 * and otherwise replaces every edge's flows by the exact minimiser of its
 * quadratic subproblem (eq. (10)).
 *
 * Conventions shared by every entry point:
 *  - Edge e is CSR position e: its tail is the vertex i with
 *    row_ptr[i] <= e < row_ptr[i+1], its head is col[e].
 *  - Flow arrays are edge-major and commodity-contiguous: f[e*K + k].
 *    Height arrays are vertex-major: h[i*K + k].
 *  - Host pointers are read or written only during the call; the caller
 *    keeps ownership of every array it passes.  A context owns all device
 *    memory it allocates and frees it in pdr_destroy.
 *  - Device work is enqueued on the CUDA stream given to pdr_create (NULL =
 *    the legacy default stream); calls that return host data synchronise
 *    that stream before returning.
 *  - Every function returns a pdr_status.  The library never aborts, traps
 *    or prints; the message of the last failure on a context is returned by
 *    pdr_last_error.  A context is not thread-safe: calls on one context
 *    must not overlap.
 */
#ifndef PDR_H
#define PDR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pdr_ctx pdr_ctx; /* opaque solver context */

typedef enum {
    PDR_OK = 0,
    PDR_ERR_INVALID_ARG = 1, /* an argument violates the stated domain */
    PDR_ERR_OOM = 2,         /* device or host allocation failed */
    PDR_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    PDR_ERR_NUMERIC = 4,     /* a non-finite objective appeared */
    PDR_ERR_NOT_SOLVED = 5,  /* reserved */
    PDR_ERR_UNSUPPORTED = 6, /* option or size outside what this build supports */
    PDR_ERR_TIMEOUT = 7      /* a device-side wait ran out of its time limit; the kernel left, the
                                solve stopped, and the context stays usable */
} pdr_status;

typedef enum {
    PDR_VERDICT_UNKNOWN = 0,   /* neither test below is met yet */
    PDR_VERDICT_FEASIBLE = 1,  /* eq. (1) residuals are within the tolerance */
    PDR_VERDICT_INFEASIBLE = 2 /* a Farkas certificate proves eq. (1) empty */
} pdr_verdict;

typedef enum {
    PDR_PREC_FP32 = 0,         /* flows, heights and the edge QP in FP32 */
    PDR_PREC_FP64 = 1,         /* everything in FP64 */
    PDR_PREC_FP32_FP64TAIL = 2 /* FP32 until its stop rules fire, then FP64 */
} pdr_precision;

typedef enum {
    PDR_ALGO_ESO = 0, /* Alg. 1 with the exact edge solver of Alg. 2 (PDR-ESO) */
    PDR_ALGO_AGD = 1, /* Alg. 3: projected gradient step with adaptive learning rate (PDR-AGD) */
    PDR_ALGO_GDM = 2, /* Alg. 4: Alg. 3 with momentum (PDR-GDM) */
    PDR_ALGO_CK = 3   /* Alg. 1 with the capacity kept (Program (6), Section "Further Discussion on
                         Optimality Condition"): every edge projects Alg. 2's c_k = f_k + (h_ik - h_jk)/2
                         onto {f >= 0, sum_k f_k <= u_e}, i.e. f'_k = max(0, c_k - g) with g = 0 if
                         sum_k max(0, c_k) <= u_e, else sum_k f'_k = u_e.  The paper gives the program's
                         optimality conditions but no algorithm; this is Alg. 1's local step with the
                         capacity term kept as a constraint (a projected gradient step of size 1/2).
                         The flows never exceed the capacities; the objective is 1/2 sum delta h^2. */
} pdr_algo;

typedef enum {
    PDR_STOP_MAX_SWEEPS = 0, /* t reached max_sweeps */
    PDR_STOP_OBJECTIVE = 1,  /* |z^(t) - z^(t-1)| < eps_obj (Alg. 1) */
    PDR_STOP_RESIDUAL = 2,   /* cap_rel <= resid_tol and cons_rel <= resid_tol */
    PDR_STOP_RELATIVE = 3,   /* |z^(t) - z^(t-1)| <= eps_rel * z^(t) */
    PDR_STOP_NUMERIC = 4,    /* z is not finite */
    PDR_STOP_STALL = 5,      /* FP32 phase of PDR_PREC_FP32_FP64TAIL: z^(t) >= z^(t-1) */
    PDR_STOP_PLATEAU = 6     /* FP32 phase of PDR_PREC_FP32_FP64TAIL: over a window of 1024 sweeps
                                the smallest max(cap_rel, cons_rel), already below 1000 x resid_tol
                                (1e-3 when resid_tol <= 0), fell by less than 1e-4 of the previous
                                window's (the FP32 rounding floor) */
} pdr_stop_reason;

typedef struct {
    int32_t precision;  /* pdr_precision (default PDR_PREC_FP32) */
    int32_t use_graph;  /* sweep-loop engine.  1: the loop runs on the device as one CUDA graph with
                           a conditional while node (default).  0: the same kernels are launched
                           from a host loop that reads the stop flag between chunks of sweeps.
                           2: one persistent cooperative kernel runs the excess pass and the edge
                           QPs of every sweep, separated by grid barriers, for 1024 sweeps per
                           launch (PDR_ALGO_ESO with a lane-group edge variant, K <= 1024 in FP32
                           or 512 in FP64; otherwise 1 is used); a barrier that waits more than
                           about a second ends the solve with PDR_ERR_TIMEOUT.
                           3: one thread-block cluster (1-8 blocks) runs the whole solve --
                           excess pass, objective and stop test, edge QPs, separated by
                           cluster barriers -- for 2048 sweeps per launch, as the batched
                           form does for its small instances (PDR_ALGO_ESO or PDR_ALGO_CK,
                           m x K <= 2^18 and a lane-group edge variant of at most 4 vectors
                           per lane; otherwise 1 is used).  An instance that one block solves
                           and whose arrays fit in 100 KB of shared memory (flows, heights,
                           roots, partials, state and the read-only arrays of a sweep) is
                           solved there, copied in and out once per launch.  FP64 sweeps
                           (PDR_PREC_FP64 and the FP64 tail) run on engine 1: one block has
                           one SM's FP64 rate.  Same flows and sweeps as 1. */
    double eps_obj;     /* Alg. 1 stop rule, absolute; <= 0 disables (default 1e-6, Section 7) */
    double resid_tol;   /* residual stop and feasibility tolerance; <= 0 disables the stop (default 1e-6) */
    double eps_rel;     /* relative objective-change stop; <= 0 disables (default 0) */
    int64_t max_sweeps; /* upper bound on QP updates per solve (default 1,000,000) */
    int32_t trace_len;  /* number of z^(t) values kept for pdr_trace (default 0) */
    int32_t algo;       /* pdr_algo (default PDR_ALGO_ESO) */
    /* Alg. 3 / Alg. 4 parameters (Section 7).  A value <= 0 (gamma < 0)
     * selects the paper's default for the chosen algorithm: AGD beta_init
     * 0.25, beta_max 0.5; GDM beta_init 0.1, beta_max 0.2, gamma 0.9; both
     * beta_min 1/K, alpha_inc 2, alpha_dec 0.5.  Ignored by PDR_ALGO_ESO. */
    double beta_init, beta_min, beta_max, alpha_inc, alpha_dec, gamma;
    /* Kernel variant of the edge update (a tuning choice; every variant
     * computes the same step).  -1 (default): the library's choice for K.
     * 0..pdr_num_edge_variants()-1: that entry of the variant table (the
     * numbering pdr_batch_tuning reports); its row capacity
     * (pdr_edge_variant_capacity) must hold K in every precision the solve
     * uses, else PDR_ERR_INVALID_ARG. */
    int32_t edge_variant;
    /* Kernel form of the excess pass (eq. (2), (3); a tuning choice, every form
     * gives bit-identical heights).  -1 (default): the library's choice
     * (form 2 where it can be resident, else 0).
     * 0: one thread per (vertex, 4 values) gathers the incident flow rows.
     * 1..5: per block, one warp brings the incident row segments of a
     * contiguous range of vertices into shared memory with bulk copies
     * (cp.async.bulk) through a ring of stages, and the other warps add them:
     * 1 = 4 stages of 8 segments of 2 KB (four adding warps), 2 = 2 stages
     * of 8 (2 KB), 3 = 4 stages of 4 (2 KB), 4 = 2 stages of 8 segments of
     * 512 B (one adding warp), 5 = 4 stages of 8 (512 B).  A form that
     * cannot be resident on the device gives PDR_ERR_INVALID_ARG. */
    int32_t excess_variant;
} pdr_options;

typedef struct {
    int64_t sweeps;      /* QP updates applied by the last solve (both phases) */
    int64_t sweeps_fp64; /* of which in FP64 */
    double z;            /* objective of the returned flows (FP64 reduction) */
    double dz;           /* z^(t) - z^(t-1) at the stop */
    double cap_abs;      /* max_e max(0, sum_k f_e,k - u_e) */
    double cap_rel;      /* max_e of the same / max(u_e, mean positive u) */
    double cons_abs;     /* max_{i,k} |Delta_ik| (conservation residual) */
    double cons_rel;     /* max_{i,k} |Delta_ik| / d_k */
    double f_min;        /* min_{e,k} f_e,k */
    double margin;       /* Farkas margin; > 0 proves infeasibility */
    double margin_scale; /* sum of the margin's absolute terms */
    double ms_total;     /* wall time of the solve in milliseconds */
    int32_t verdict;     /* pdr_verdict */
    int32_t stop_reason; /* pdr_stop_reason */
    int32_t stop_reason_fp32; /* PDR_PREC_FP32_FP64TAIL: the pdr_stop_reason that ended the FP32
                                 phase (it decides whether the FP64 tail ran); -1 otherwise */
    int32_t pad;
} pdr_result;

/* Fills *opt with the defaults listed in pdr_options.  Returns PDR_OK, or
 * PDR_ERR_INVALID_ARG if opt is NULL. */
pdr_status pdr_default_options(pdr_options *opt);

/* Creates a solver for one instance of eq. (1) and builds its adjacency on
 * the device (Table "Notation": delta+(i), delta-(i), delta_i = out-degree +
 * in-degree).
 *   n        number of vertices, n >= 1
 *   m        number of edges, 0 <= m < 2^31
 *   row_ptr  host int64 [n+1]: row_ptr[0] = 0, non-decreasing, row_ptr[n] = m
 *   col      host int32 [m]: head of each edge, 0 <= col[e] < n, no self-loops
 *   u        host double [m]: capacities, finite and >= 0
 *   K        number of commodities, 1 <= K
 *   s, t     host int32 [K]: origin and destination, in range, s_k != t_k
 *   d        host double [K]: demands, finite and > 0
 *   opt      options, or NULL for the defaults
 *   stream   a cudaStream_t (NULL = legacy default stream)
 *   out      receives the context (NULL on failure)
 * Copies every input; flows start at 0.  Parallel edges are allowed.
 * Errors: PDR_ERR_INVALID_ARG (domain violation, message names the first
 * offending index), PDR_ERR_OOM, PDR_ERR_CUDA. */
pdr_status pdr_create(int32_t n, int64_t m, const int64_t *row_ptr, const int32_t *col, const double *u,
                      int32_t K, const int32_t *s, const int32_t *t, const double *d, const pdr_options *opt,
                      void *stream, pdr_ctx **out);

/* Replaces the options of ctx (the instance is kept).  NULL restores the
 * defaults.  Errors: PDR_ERR_INVALID_ARG. */
pdr_status pdr_set_options(pdr_ctx *ctx, const pdr_options *opt);

/* Runs Alg. 1 (or Alg. 3 / Alg. 4, by opt.algo) from the current state until
 * a stop rule fires (the sweep loop runs on the device as one CUDA graph),
 * then evaluates the eq. (1) residuals and the certificate in FP64 (as
 * pdr_residuals).  Leaves f^(t), the flows whose objective triggered the
 * stop, as the current flows (with the learning rates and velocities of the
 * same iteration for Alg. 3 / Alg. 4).  out may be NULL.
 * Errors: PDR_ERR_CUDA, PDR_ERR_NUMERIC. */
pdr_status pdr_solve(pdr_ctx *ctx, pdr_result *out);

/* Runs exactly `count` sweeps of the chosen algorithm (excess/heights,
 * congestion, objective, flow update) with every stop rule disabled; the
 * iteration counter t continues from the last solve or sweep (it drives the
 * learning-rate schedule of Alg. 3 / Alg. 4).  Used to compare single sweeps
 * with a reference.  Errors: PDR_ERR_INVALID_ARG (count < 0), PDR_ERR_CUDA. */
pdr_status pdr_sweeps(pdr_ctx *ctx, int64_t count);

/* Sets every flow to 0, every velocity to 0 and every learning rate to
 * beta_init, and the iteration counter to 0 (the start of Alg. 1, 3 and 4). */
pdr_status pdr_reset(pdr_ctx *ctx);

/* Copies host flows f[m*K] (double, edge-major) into the context, rounding
 * to the working precision; velocities restart at 0, learning rates at
 * beta_init and the iteration counter at 0.  Errors: PDR_ERR_INVALID_ARG
 * (NULL; negative or non-finite entries are not checked, the caller
 * supplies f >= 0). */
pdr_status pdr_set_flows(pdr_ctx *ctx, const double *f);

/* Copies the current flows to f[m*K] (double, edge-major), caller-owned.
 * f may be pageable host memory, or any memory the GPU can write (pinned
 * host memory from cudaMallocHost / cudaHostRegister, device or managed
 * memory): there a kernel packs and widens the rows into f directly.
 * Synchronises the context's stream.  Errors: PDR_ERR_INVALID_ARG (f NULL
 * with m > 0), PDR_ERR_CUDA. */
pdr_status pdr_flows(pdr_ctx *ctx, double *f);

/* Checkpoint and resume of a solve (the loop state of Alg. 1, 3 and 4).
 * The checkpoint is a host byte buffer, opaque, for one library version.  It
 * holds the current flows in the working precision and the warm starts of
 * the edge QPs.  For Alg. 3/4 it also holds the learning rates, and for
 * Alg. 4 the velocities.  It further holds the iteration counter t, the
 * previous objective z^(t-1) and the objective trace so far.
 *
 * pdr_state_size writes the buffer size the next pdr_get_state needs.
 * pdr_get_state fills buf with `bytes` >= that size; the caller owns buf.
 * Both synchronise the context's stream.
 *
 * pdr_set_state restores a checkpoint into a context.  The context must
 * come from the same instance sizes (n, m, K) and algorithm.  Its precision
 * option must admit the checkpoint's working precision: FP32 checkpoints
 * need FP32 or FP32 with FP64 tail; FP64 checkpoints need FP64 or FP32
 * with FP64 tail.  The next pdr_solve then continues the interrupted solve
 * instead of starting at t = 0: it uses the same sweep counter, stop rules
 * and trace slots.  The flows of every later sweep are bit-identical to the
 * uninterrupted solve's.  The objective partials are recomputed from the
 * restored flows, so z agrees to rounding.  A checkpoint taken after a
 * stopped solve resumes at the sweep that stopped; with a larger
 * max_sweeps, it goes on from there.  pdr_sweeps also continues the
 * counter.  pdr_reset and pdr_set_flows cancel a pending resume.
 *
 * Errors:
 * - PDR_ERR_INVALID_ARG: NULL arguments; a buffer too small, truncated or
 *   of another version; a checkpoint of other sizes, another algorithm or
 *   an inadmissible precision.
 * - PDR_ERR_CUDA. */
pdr_status pdr_state_size(pdr_ctx *ctx, int64_t *bytes);
pdr_status pdr_get_state(pdr_ctx *ctx, void *buf, int64_t bytes);
pdr_status pdr_set_state(pdr_ctx *ctx, const void *buf, int64_t bytes);

/* Test hook for the time limit of the device-side waits.
 * - Waits: the bulk-copy excess forms (pdr_options.excess_variant 1..5)
 *   waits on shared-memory barriers.
 * - Default limit: 2^32 SM clock cycles, about 2 s.
 * - cycles: sets that limit; 1000 <= cycles <= 2^32.
 * - hold_end = 1: the form's producer never posts the end marker of its
 *   ring.  Every block's consumers then wait out the limit, with no copy in
 *   flight, and the call that ran the sweep returns PDR_ERR_TIMEOUT.
 * - hold_end = 0: normal operation.
 * Errors: PDR_ERR_INVALID_ARG. */
pdr_status pdr_debug_wait(pdr_ctx *ctx, int64_t cycles, int32_t hold_end);

/* Test hook for the time limit of the persistent engine's grid barrier
 * (pdr_options.use_graph = 2).  No counterpart in the paper.
 * - Each wait at the barrier gives up after limit_ns nanoseconds of the
 *   GPU's global timer (default 2e9, 2 s; 1e5 <= limit_ns <= 2e9), raises a
 *   flag that ends every other block's wait, and every block leaves the
 *   kernel; the solve returns PDR_ERR_TIMEOUT and the context stays usable.
 * - withhold = 1: block 0 leaves the kernel at its first barrier without
 *   arriving (it has no copy in flight), so the other blocks' waits run out.
 * - withhold = 0: normal operation.
 * Errors: PDR_ERR_INVALID_ARG. */
pdr_status pdr_debug_barrier(pdr_ctx *ctx, int64_t limit_ns, int32_t withhold);

/* Test hook for host-side failure injection: the nth device allocation the
 * library makes from now on (in pdr_create, pdr_set_options, pdr_batch_create,
 * ...) fails as if the device were out of memory, and the call that made it
 * returns PDR_ERR_OOM after releasing what it had allocated.  nth = 0 turns
 * the injection off; it also ends after the failure.  Process-wide.
 * Errors: PDR_ERR_INVALID_ARG (nth < 0). */
pdr_status pdr_debug_fail_alloc(int64_t nth);

/* Selected rows of the current state: out[q*K + k] = f_{edges[q],k}
 * (which = 0) or the Alg. 4 velocity v_{edges[q],k} (which = 1), for
 * q < count (double).  For checking large instances edge by edge without
 * copying every row.  Errors: PDR_ERR_INVALID_ARG (NULL, an edge id outside
 * [0, m), or which = 1 on a context that does not run Alg. 4). */
pdr_status pdr_flow_rows(pdr_ctx *ctx, int32_t which, const int64_t *edges, int64_t count, double *out);

/* State of Alg. 3 / Alg. 4 of the current iteration: learning rates beta[m]
 * and (Alg. 4) velocities v[m*K] (edge-major) into host arrays; either may
 * be NULL.  Errors: PDR_ERR_INVALID_ARG if the context runs Alg. 1. */
pdr_status pdr_gd_state(pdr_ctx *ctx, double *beta, double *v);

/* Replaces the Alg. 3 / Alg. 4 state: beta[m] (> 0) and, for Alg. 4, v[m*K]
 * (NULL = zeros).  The flows are kept.  Errors: PDR_ERR_INVALID_ARG. */
pdr_status pdr_set_gd_state(pdr_ctx *ctx, const double *beta, const double *v);


/* Heights h_ik (eq. (2)) of the current flows, computed in the working
 * precision by the sweep's excess kernel, into host h[n*K] (double). */
pdr_status pdr_heights(pdr_ctx *ctx, double *h);

/* Congestion psi_e (eq. (41)) of the current flows into host psi[m]. */
pdr_status pdr_congestion(pdr_ctx *ctx, double *psi);

/* Objective z of Alg. 1 at the current flows (FP64 reduction of the working
 * precision heights and congestion) into *z. */
pdr_status pdr_objective(pdr_ctx *ctx, double *z);

/* The in-adjacency built on the device: in_ptr[n+1] (int64), in_eid[m]
 * (int32, edge ids entering each vertex in ascending order) and deg[n]
 * (int32, delta_i).  Any output may be NULL. */
pdr_status pdr_adjacency(pdr_ctx *ctx, int64_t *in_ptr, int32_t *in_eid, int32_t *deg);

/* eq. (1) residuals, Farkas certificate and verdict of the current flows,
 * all computed on the device in FP64 from the stored flows.  The
 * certificate uses potentials h and lengths l_e = max(0, max_k (h_ik - h_jk));
 * margin = sum_k d_k (h_{s_k,k} - h_{t_k,k}) - sum_e u_e l_e > 0 proves
 * eq. (1) infeasible (Farkas' lemma; Theorems 1 and 2 of Section 3).
 * Verdict: INFEASIBLE if margin > 1e-9 * margin_scale or a commodity
 * endpoint has degree 0; FEASIBLE if cap_rel <= resid_tol and
 * cons_rel <= resid_tol; UNKNOWN otherwise.  Fills every field of *out
 * except sweeps, sweeps_fp64, dz, ms_total and stop_reason, which keep the
 * values of the last solve. */
pdr_status pdr_residuals(pdr_ctx *ctx, pdr_result *out);

/* Copies up to `len` values of the objective trace z^(0), z^(1), ... of the
 * last solve (kept when trace_len > 0) into host z; *count receives the
 * number of values written. */
pdr_status pdr_trace(pdr_ctx *ctx, double *z, int64_t len, int64_t *count);

/* Instance sizes: n, m, K, and the padded row length Kp used on the device. */
pdr_status pdr_sizes(const pdr_ctx *ctx, int32_t *n, int64_t *m, int32_t *K, int32_t *Kp);

/* Times `launches` back-to-back launches of one sweep kernel on the current
 * state, each bracketed by CUDA events on the context's stream, and returns
 * the mean duration in milliseconds.  which = 0: edge QP (Alg. 2);
 * which = 1: excess/height (eq. (3), (2)).  If flush_bytes > 0 a buffer of
 * that size is overwritten before every launch so each starts with a cold
 * L2.  Each QP launch repeats the solve's next sweep.  It reads the current
 * flows and the roots that warm-start that sweep, and writes the other
 * buffers.  The device state is put back afterwards, so the current flows,
 * warm starts and iteration counter do not change.  Errors:
 * PDR_ERR_INVALID_ARG, PDR_ERR_CUDA, PDR_ERR_OOM. */
pdr_status pdr_time_kernel(pdr_ctx *ctx, int32_t which, int32_t launches, int64_t flush_bytes, double *ms);

/* pdr_sweeps(ctx, count) with CUDA events on the context's stream around
 * each launch of the excess kernel and of the update kernel (the edge QP
 * of Alg. 2 or the capacity-kept step, or the gradient step of Alg. 3/4).
 * The kernels are launched from the host, one after the other.  Writes the
 * mean duration of each kernel over the `count` sweeps, in milliseconds:
 * the kernels' average cost along a real run of the solve, with its warm
 * starts and its L2 state.  The flows advance as with pdr_sweeps.  Errors:
 * PDR_ERR_INVALID_ARG (NULL, count < 1), PDR_ERR_CUDA. */
pdr_status pdr_time_sweeps(pdr_ctx *ctx, int64_t count, double *ms_excess, double *ms_update);

/* Number of entries in the edge-kernel variant table (pdr_options.edge_variant). */
int32_t pdr_num_edge_variants(void);

/* Row capacity of variant v: the largest K it holds in `precision`
 * (PDR_PREC_FP32 or PDR_PREC_FP64).  *pipelined (may be NULL) receives 1 for
 * the persistent pipelined warp forms of Alg. 2 and 2 for the staged block
 * forms (one block per SM that keeps the next edge's rows in flight as bulk
 * copies into shared memory), 0 for the plain forms; Alg. 3/4 run the plain
 * form of a pipelined or staged variant.  Returns -1 if v or precision is out
 * of range (nothing written). */
int32_t pdr_edge_variant_capacity(int32_t v, int32_t precision, int32_t *pipelined);

/* In-adjacency and degrees of a graph that already lives in device memory,
 * computed without allocating any memory.  The paper has no counterpart:
 * this is a deployment entry point, not a step of the method.
 *
 * Who needs it: a caller whose device memory is owned by another allocator
 * (a framework's caching pool that has claimed the GPU, or a service that
 * reserves all memory at start-up and must not allocate afterwards) cannot
 * call cudaMalloc, so it cannot use pdr_create.  This function takes the
 * caller's device arrays and uses a fixed scratch area compiled into the
 * library instead of allocating one.
 *   n        number of vertices, 1 <= n <= 262,144 (the scratch limit;
 *            larger n returns PDR_ERR_INVALID_ARG and does no GPU work)
 *   m        number of edges, 0 <= m < 2^31
 *   row_ptr  device int64 [n+1], col device int32 [m]: the out-adjacency
 *            (edge id = CSR position); checked on the device, a malformed
 *            CSR returns PDR_ERR_INVALID_ARG with nothing written
 *   in_ptr   device int64 [n+1] (out): offsets of the in-adjacency
 *   in_eid   device int32 [m] (out): edge ids entering each vertex, ascending
 *   deg      device int32 [n] (out): out-degree + in-degree
 *   stream   cudaStream_t to run on (NULL = legacy default stream)
 * The outputs equal those of pdr_adjacency on a context built from the same
 * graph.  The call synchronises the stream before returning.
 * Scratch: 4 MiB of device memory per GPU that loads the library, held until
 * the process exits, shared by every call: calls whose GPU work overlaps
 * (other host threads, or other streams of the same device) race on it and
 * must be serialised by the caller.  Every call looks up the scratch's
 * device address on the current device before it launches anything (nothing
 * is cached across calls, so a cudaDeviceReset between calls is harmless);
 * make the first call on a device before any stream capture begins.  On
 * failure pdr_last_error(NULL) returns the message.  Errors:
 * PDR_ERR_INVALID_ARG, PDR_ERR_CUDA. */
pdr_status pdr_adjacency_static(int32_t n, int64_t m, const int64_t *row_ptr, const int32_t *col, int64_t *in_ptr,
                                int32_t *in_eid, int32_t *deg, void *stream);

/* Replaces the capacities u[m] and/or the demands d[K] (NULL keeps them);
 * same domain as pdr_create.  The flows are kept.  u and d may be host
 * memory, or both device (or managed) memory: then they are checked and
 * converted on the device (no host copy; the call synchronises the
 * context's stream to read the check), with the same results.  An array
 * outside the domain changes nothing.  Errors: PDR_ERR_INVALID_ARG (domain,
 * or one host and one device array), PDR_ERR_CUDA. */
pdr_status pdr_set_data(pdr_ctx *ctx, const double *u, const double *d);

/* Differentiated form.  L(u, d) = z(f^(T)), the objective of Alg. 1 after T
 * sweeps from f = 0 (no stop rule), and, if grad_u / grad_d are not NULL, its
 * gradient with respect to the capacities (grad_u[m]) and demands
 * (grad_d[K]) by reverse mode through the T sweeps (the derivatives of
 * eq. (3), (2), eq. "cpgrad" and of Alg. 2's active-set solution, or of the
 * capacity-kept projection for PDR_ALGO_CK; at a kink of max(0, .) or of an
 * active set, the derivative of the active set the forward took).  Flows
 * are checkpointed every ckpt_every sweeps and each segment's sweeps are
 * recomputed on the way back, so the workspace is about (T/ckpt_every +
 * ckpt_every) flow arrays plus ckpt_every height arrays.  ckpt_every = 1
 * keeps every sweep's flows, heights and roots from the forward pass
 * instead (T + 1 flow arrays and T height arrays) and recomputes nothing;
 * the results are the same bit for bit.
 * The context keeps that workspace after a call with gradients and reuses
 * every buffer that is large enough, so later calls with the same T and
 * ckpt_every allocate nothing; pdr_destroy frees it (and a failed call
 * does).  Runs in the context's
 * working precision (FP32 or FP64; gradients accumulate in FP64) and leaves
 * f^(T) as the current flows.  grad_u and grad_d may be host or device
 * memory (the copy follows unified addressing); L is a host double.
 * Errors: PDR_ERR_INVALID_ARG (T < 0, ckpt_every < 1, or a context that
 * runs Alg. 3 or Alg. 4), PDR_ERR_OOM, PDR_ERR_CUDA. */
pdr_status pdr_backward(pdr_ctx *ctx, int64_t T, int32_t ckpt_every, double *L, double *grad_u, double *grad_d);

/* ------------------------------------------------------------------------ */
/* Batched form: many independent instances, one graph launch per solve      */
/* ------------------------------------------------------------------------ */

typedef struct pdr_batch pdr_batch; /* opaque; owns one context per instance */

/* One instance of eq. (1), with the same meaning and rules as the
 * arguments of pdr_create. */
typedef struct {
    int32_t n;
    int32_t K;
    int64_t m;
    const int64_t *row_ptr;
    const int32_t *col;
    const double *u;
    const int32_t *s;
    const int32_t *t;
    const double *d;
} pdr_instance;

/* Creates a batch of `count` independent instances (Alg. 1 applied to each,
 * with the options opt shared by all).  Every instance gets its own context
 * on `stream`; an autotuner then times the edge-kernel variants that fit each
 * instance's row length (lanes per edge, vectors per lane, block size) on
 * that instance and keeps the fastest; opt->edge_variant >= 0 fixes the
 * variant for every instance instead.  Errors: PDR_ERR_INVALID_ARG (count <
 * 1, NULL, or an instance rejected by pdr_create: the message names it),
 * PDR_ERR_OOM, PDR_ERR_CUDA, PDR_ERR_UNSUPPORTED. */
pdr_status pdr_batch_create(int32_t count, const pdr_instance *inst, const pdr_options *opt, void *stream,
                            pdr_batch **out);

/* Solves every instance from its current state.  Small instances (m x K <=
 * 2^18 on a lane-group variant of at most 4 vectors per lane, Alg. 1 or
 * Program (6)) run their FP32 sweeps on one thread-block cluster each, in
 * shared launches of the cluster kernel (engine 3 of pdr_options.use_graph,
 * with its shared-memory form for the instances that fit).  The others, and
 * every FP64 sweep (one block has only one SM's FP64 rate), run in one CUDA
 * graph launch: a conditional while loop whose body holds one chain of
 * sweeps per instance; the chains are independent, so the instances run
 * concurrently.  Each instance stops by its own stop
 * rules (a stopped instance's kernels return at once); the loop ends when
 * the last one stops.  The flows equal, bit for bit, single-instance solves
 * with the same edge variant.  With
 * PDR_PREC_FP32_FP64TAIL a second launch then runs FP64 sweeps for the
 * instances whose FP32 phase stopped on the objective rules (as pdr_solve
 * does for one instance).  Then each instance's residuals and verdict are
 * evaluated as by pdr_residuals.
 * results may be NULL, else it receives `count` results in input order.
 * Errors: PDR_ERR_CUDA, PDR_ERR_NUMERIC (some instance's objective became
 * non-finite). */
pdr_status pdr_batch_solve(pdr_batch *batch, pdr_result *results);

/* Resets every instance (as pdr_reset). */
pdr_status pdr_batch_reset(pdr_batch *batch);

/* The context of instance `index`, owned by the batch (do not destroy it):
 * use it with pdr_flows, pdr_residuals, pdr_adjacency and the other read-out
 * calls.  Errors: PDR_ERR_INVALID_ARG. */
pdr_status pdr_batch_context(pdr_batch *batch, int32_t index, pdr_ctx **ctx);

/* The edge-kernel variant the autotuner chose for each instance
 * (cfg[count], an index into the library's variant table) and its mean
 * launch time in microseconds (us[count]); either may be NULL. */
pdr_status pdr_batch_tuning(const pdr_batch *batch, int32_t *cfg, double *us);

/* Frees the batch and every context it owns.  NULL is ignored. */
void pdr_batch_destroy(pdr_batch *batch);

/* Message of the last failure on ctx (or, if ctx is NULL, of the last failed
 * pdr_create or pdr_adjacency_static on this thread).  Never NULL; valid
 * until the next call. */
const char *pdr_last_error(const pdr_ctx *ctx);

/* Frees every resource of ctx.  NULL is ignored. */
void pdr_destroy(pdr_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* PDR_H */
