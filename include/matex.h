/*
 * matex.h — C ABI of the GB300 batched R-MATEX integrator.
 *
 * The library integrates the RC power-grid ODE of Eq. 1,
 *     C x'(t) = -G x(t) + B u(t),     C = diag(c),  G symmetric positive definite,
 * with piecewise-linear current loads u(t), by the rational (shift-and-invert)
 * Krylov matrix-exponential method R-MATEX (Sec. 3.3.2, Alg. 1 with
 * X1 = C + gamma G, X2 = C; Eq. 9 for H_m; the empirical residual of
 * Sec. 3.3.3).  The loads are split into "bump" groups (Sec. 3.1); each group
 * is simulated on its own local transition spots (Alg. 2) and the group
 * responses are summed by superposition.  Every group is one column of a
 * batched launch on one GPU.
 *
 * Conventions for every call:
 *   - All floating point is IEEE FP64 (double).  Indices are int32 unless
 *     noted; CSR row pointers are int64.
 *   - "host" pointers are read during the call only and copied; the caller
 *     keeps ownership.  "device" pointers are CUDA global-memory pointers on
 *     the device that was current at matex_setup; the caller owns them.
 *   - Work is issued on the CUDA stream given to matex_setup (NULL = legacy
 *     default stream).  Calls that return results synchronise that stream
 *     before returning.
 *   - No call throws or aborts.  Each returns a matex_status; on failure
 *     matex_last_error() describes it.  A failed call leaves the context
 *     usable unless the status is MATEX_ERR_CUDA (a sticky device error).
 *   - One context must not be used from two host threads at once.
 *
 * Node order: every node-indexed array in this interface uses the caller's
 * (original) numbering.  The library reorders internally.
 */
#ifndef MATEX_H_
#define MATEX_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct matex_ctx matex_ctx;

typedef enum matex_status {
  MATEX_OK = 0,
  MATEX_ERR_ARG = 1,      /* invalid argument (sizes, indices, NULL, non-increasing PWL times) */
  MATEX_ERR_NOT_SPD = 2,  /* G or C + gamma G has a non-positive pivot */
  MATEX_ERR_CUDA = 3,     /* a CUDA runtime call failed */
  MATEX_ERR_TIMEOUT = 4,  /* a bounded device wait gave up */
  MATEX_ERR_NOCONV = 5,   /* strict mode: some segment reached m_max without meeting tol
                             (results are still written) */
  MATEX_ERR_OOM = 6,      /* device or host allocation failed */
  MATEX_ERR_STATE = 7     /* call not valid in the context's current state */
} matex_status;

/* Options of matex_setup.  Start from matex_default_opts(). */
typedef struct matex_opts {
  int32_t col_block;       /* column block of the triangular solves: 0 = tuned per tree level,
                              else 1, 2, 4 or 8 for every level */
  int32_t group_select;    /* -1: all groups; g >= 0: simulate only group g */
  int32_t include_dc;      /* 1: add the pads' constant DC state x_dc = G^{-1} dc_inject */
  int32_t n_rows;          /* 0: output every node; else the number of rows in `rows` */
  const int32_t* rows;     /* host, n_rows original node indices to output (copied) */
  const int32_t* replay_m; /* host or NULL: Krylov dimension to use per (group, segment),
                              groups in order, segments in time order (copied); NULL = adaptive */
  int64_t n_replay;        /* number of entries in replay_m (must equal the segment total) */
  int32_t max_width;       /* cap on supernode width (0 = 1024) */
  int32_t strict;          /* 1: return MATEX_ERR_NOCONV when m_max is reached unconverged */
  int32_t solve_mode;      /* 0: one persistent launch per triangular-solve pair, tasks ordered
                              by dependency counters; 1: one launch per tree level; 2 (default):
                              chosen per column count by the setup-time autotuner */
  int32_t tape;            /* what every run keeps on the device so that matex_grad can follow
                              it: 0 nothing; 1 the full tape, each segment's Krylov basis,
                              solve outputs and Hessenberg (memory ~ segments x m x n);
                              2 checkpoints, each group's state x and carried input solution
                              z at the start of every tape_window-th segment round (memory ~
                              segments x n / tape_window); matex_grad then recomputes each
                              window's segments from its checkpoint, tape_block groups at a
                              time, with the run's Krylov dimensions, and reverses them */
  int32_t krylov;          /* Krylov space of the circuit solver (Alg. 1): 0 (default) rational,
                              X1 = C + gamma G (R-MATEX, Sec. 3.3.2); 1 inverted, X1 = G
                              (I-MATEX, Sec. 3.3.1); 2 standard, w = A v = -C^{-1} G v (MEXP,
                              Sec. 2.3; needs m far above 20 on stiff grids).  The residual's
                              h_{m+1,m} is scaled by 1, 1/gamma, gamma so that tol (V) serves all
                              three.  tape = 1 requires 0 */
  int32_t graph;           /* 1 (default): after a plain run, record the run's launches as a
                              CUDA graph and replay it in later runs while the device's
                              active-column counts match the recorded ones (checked on the
                              device; on a mismatch the run is redone plainly and re-recorded);
                              0: every run is issued launch by launch */
  double tail_eps;         /* 0 (default): exact.  eps > 0 (V): a group's term of an output
                              (Eq. 6 with -P) is shortened once it stays small for the rest of
                              its segment: past the last output where ||y||_2 > eps/2 its V y
                              part is left out (|V y|_inf <= ||y||_2 for an orthonormal V), and
                              the whole term when also max|z - w| + L max|z'| <= eps/2.  Each
                              output entry then differs from the exact run by at most
                              eps x (number of groups), plus rounding.  Changes the work done,
                              so such runs are timed apart from exact ones.  tape = 1 requires
                              0.  Negative or non-finite: MATEX_ERR_ARG */
  int32_t tape_window;     /* tape = 2: segment rounds per checkpoint window; 0 (default): the
                              setup chooses it, with tape_block, from the free device memory
                              (the largest block that fits, then the window with the least
                              memory) */
  int32_t tape_block;      /* tape = 2: groups recomputed together (columns of the recompute
                              and reverse launches); 0 (default): chosen at setup */
  int32_t recombine;       /* V y of the recombination (Eq. 6 at the outputs): 0 (default) on
                              the tensor cores where it pays (exact runs, rounds of 16 to
                              kdim_cap basis vectors), as an error-free decomposition of the
                              FP64 operands into 6-bit bf16 slices whose products the FP32
                              accumulators hold exactly (error of the order of an FP64 dot
                              product); 1: FP64 FMAs only */
  int32_t decompose;       /* 0 (default): the groups as given (Sec. 3.1's bump groups);
                              1: every group's input is split further into single ramps: on
                              [0, T] a source is its value at t = 0 plus, at each of its
                              breakpoints tau in [0, T), a ramp ds max(0, t - tau) (ds: change
                              of slope at tau), and every (group, tau) becomes a column of its
                              own (a group's non-zero starting values one more).  A ramp
                              starts from zero state, so its Krylov basis needs no earlier
                              segment and all ramps are independent; the responses sum to the
                              same outputs.  Order of the columns (matex_get_m): by group,
                              its constant part first, then its ramps by tau.  Requires
                              group_select -1 and tape 0; new currents need a new context */
  int32_t resident;        /* segment rounds on small grids: 0 (default) chosen at setup, 1 off,
                              2 on.  A resident round runs each column's whole segment (input
                              solutions, Arnoldi with its residual test, output coefficients,
                              next state) in one CTA, both triangular substitutions level by
                              level in its shared memory; only the recombination is a launch of
                              its own.  Possible when n <= 8192 (and 16 n + 34 KB fit one CTA's
                              shared memory), krylov 0 or 1, tape 0 and tail_eps 0; 2 returns
                              MATEX_ERR_ARG otherwise.  With 0 the setup times one such solve
                              pair against the batched path's single-column pair and takes the
                              resident rounds when they are at most twice as long (they also
                              replace the ~12 other launches of every Arnoldi step).  The
                              input solutions of every segment (sources only) are solved ahead
                              of the rounds in one launch when they fit a quarter of the free
                              memory; 3: as 2, but each round kernel solves its own (the path
                              taken when they do not fit; the same results bit for bit) */
  int32_t tc_solve;        /* supernodes at least tc_min_width wide in the level solves: 0
                              (default) chosen at setup per column count, 1 off, 2 on.  Their
                              two dense products per supernode (P_s b_s forward, P_s^T [..]
                              backward) run on the bf16 tensor cores as an error-free split of
                              the FP64 operands into nine 6-bit digits (error of the order of an
                              FP64 dot product), the rest of each level on the FP64 kernels.
                              With 0 the setup times the solve pair both ways at each column
                              count it tunes and keeps the tensor cores where they are faster.
                              Level launches only (not the persistent solve) */
  int32_t tc_min_width;    /* 0 (default): 64; else at least 32 */
  int32_t single_column;   /* solves of one right-hand side: 0 (default) chosen at setup, 1 off,
                              2 on.  The single-column level kernels run one launch per tree level
                              and direction like the level launches, with everything that does
                              not depend on the right-hand side (work descriptors, panel entries,
                              gather rows) loaded before the previous level completes and one
                              group of lanes per output row or column (no partial sums through
                              memory).  With 0 the setup times the single-column solve pair both
                              ways and keeps the faster (the new kernels when at least 5 %
                              faster) */
} matex_opts;

/* Counters and timings of the last matex_run (or of setup for the setup_* fields). */
typedef struct matex_stats {
  double setup_order_ms;   /* nested-dissection ordering + symbolic analysis (host) */
  double setup_factor_ms;  /* numeric L D L^T of C + gamma G and of G (host) */
  double setup_upload_ms;  /* host -> device upload of factors and tables */
  double run_ms;           /* wall time of the last matex_run (host clock, synchronised) */
  int64_t nnz_L;           /* strictly lower nonzeros of one factor */
  int32_t n_supernodes;
  int32_t n_levels;        /* depth of the supernodal elimination tree */
  int32_t n_segments;      /* total (group, segment) pairs */
  int32_t krylov_segments; /* segments that built a basis (non-quiescent) */
  int32_t sum_m;           /* sum of Krylov dimensions over segments */
  int32_t max_m;
  int32_t nonconv;         /* segments that stopped at m_max above tol */
  int32_t breakdowns;      /* segments that ended in a happy breakdown */
  int32_t sweeps_M;        /* batched solves with C + gamma G */
  int32_t sweeps_G;        /* batched solves with G */
  int64_t solve_columns;   /* right-hand sides solved, over all sweeps */
  int32_t kernel_launches; /* kernels launched by the last matex_run */
  int32_t rounds;          /* segment rounds (max segments over the selected groups) */
  int32_t graph_replay;    /* 1: the last run replayed the captured CUDA graph */
  double graph_capture_ms; /* host time of the last graph capture + instantiation */
  int64_t nnz_L_exact;     /* strictly lower nonzeros of L for the ordering, without the
                              explicit zeros of relaxed amalgamation that nnz_L counts */
  int32_t tape_window;     /* tape = 2: rounds per checkpoint window and groups per recompute */
  int32_t tape_block;      /*   block as set up (0 otherwise) */
  int64_t tape_bytes;      /* device bytes of the adjoint's tape (tape 1) or of its checkpoints,
                              window tape and reverse work buffers (tape 2) */
  int32_t tc_rounds;       /* segment rounds of the last run whose V y ran on the tensor cores */
  int32_t resident;        /* 1: the segment rounds run as resident rounds (opts.resident) */
  int32_t tc_solve_supernodes;  /* supernodes whose solve products can run on the tensor cores
                                   (0: none or tc_solve off) */
  int32_t tc_solve_min_cols;    /* smallest column count at which they do (0: never) */
  int32_t single_column;        /* 1: single-column solves run the single-column level kernels */
} matex_stats;

void matex_default_opts(matex_opts* opts);

/*
 * Build a context: check the inputs, order and factor C + gamma G and G once
 * (the serial part of Alg. 2), build each group's local transition spots
 * (Sec. 3.1: the breakpoints of its sources inside (0, T) plus 0 and T),
 * assign every output time t_o = o*dt_out (o = 0..N, N = round(t_end/dt_out),
 * simulation end T = N*dt_out) to the segment (l_j, l_{j+1}] containing it,
 * and upload everything to the current device.
 *
 *   n                 number of nodes (> 0)
 *   c                 host[n], node capacitances (F), all > 0
 *   g_rowptr, g_col,  host CSR of G (both triangles, symmetric, SPD), int64 row
 *   g_val             pointers [n+1], int32 columns, values in S
 *   dc_inject         host[n] or NULL, constant injected currents (A), e.g. pads'
 *                     Norton currents Vdd/R_pad; forms x_dc = G^{-1} dc_inject
 *   n_src, src_node   host[n_src], node of each piecewise-linear source (>= 0)
 *   pwl_off           host[n_src+1], offsets into pwl_t / pwl_v (>= 1 point each)
 *   pwl_t, pwl_v      host, breakpoint times (s, strictly increasing per source)
 *                     and injected currents (A; loads are negative).  Before the
 *                     first and after the last breakpoint the value is held.
 *   src_group         host[n_src], group of each source in [0, n_groups)
 *   gamma             shift of the rational Krylov space, (C + gamma G)^{-1} C (s)
 *   tol               residual tolerance of Sec. 3.3.3 (V, absolute)
 *   m_max             largest Krylov dimension, 1..20
 *   t_end, dt_out     simulated time span and output spacing (s)
 *   opts              NULL for defaults
 *   stream            cudaStream_t, or NULL
 * On success *out receives a context to be released with matex_destroy.
 */
matex_status matex_setup(matex_ctx** out, int64_t n, const double* c, const int64_t* g_rowptr,
                         const int32_t* g_col, const double* g_val, const double* dc_inject,
                         int32_t n_src, const int32_t* src_node, const int32_t* pwl_off,
                         const double* pwl_t, const double* pwl_v, const int32_t* src_group,
                         int32_t n_groups, double gamma, double tol, int32_t m_max, double t_end,
                         double dt_out, const matex_opts* opts, void* stream);

/*
 * Run the batched R-MATEX transient (Alg. 2 per group, Alg. 1 per segment,
 * superposition over groups) and write the node voltages:
 *   x_out  device, [N+1][n_rows] row-major (n_rows = n when no row list was
 *          given): x_out[o*n_rows + r] = x(t_o) at the r-th output node.
 *   stats  host or NULL.
 * Synchronises the stream.  Returns MATEX_ERR_NOCONV only in strict mode.
 */
matex_status matex_run(matex_ctx* ctx, double* x_out, matex_stats* stats);

/*
 * End-to-end variant with host buffers: copies the source currents pwl_v
 * (host, same layout and length as at setup, or NULL to keep the current
 * ones) to the device, runs, and copies the result to x_out_host (host,
 * [N+1][n_rows]).  Page-locked host memory makes the copies asynchronous.
 */
matex_status matex_run_host(matex_ctx* ctx, const double* pwl_v_host, double* x_out_host,
                            matex_stats* stats);

/*
 * Several independent contexts (e.g. grids of different sizes, each set up on
 * its own) run as one CUDA graph launch: each context's recorded run is a
 * branch of one graph, the branches have no edges between them, so the GPU
 * runs the grids concurrently.  Built with matex_batch_create (contexts
 * without a recorded run are run once plainly and recorded; each needs
 * opts.graph = 1), run with matex_batch_run:
 *   x_outs     host array [count] of device output pointers, one per context
 *              (layout as matex_run)
 *   stats      host [count] or NULL
 *   grid_ms    host [count] or NULL: per context, the time from the start of
 *              the batch launch to the end of that context's branch (CUDA
 *              events inside the graph)
 * A context whose device counts diverged from its recording is redone plainly,
 * re-recorded, and the batch graph rebuilt; results are then the plain run's.
 * The batch does not own the contexts; destroy it before any of them.
 */
typedef struct matex_batch matex_batch;
matex_status matex_batch_create(matex_batch** out, matex_ctx* const* ctxs, int32_t count);
matex_status matex_batch_run(matex_batch* batch, double* const* x_outs, matex_stats* stats,
                             float* grid_ms);
const char* matex_batch_last_error(const matex_batch* batch);
void matex_batch_destroy(matex_batch* batch);

/*
 * Scheduling mode of later runs: 0 (default) runs every group as a column of
 * one batched sweep per segment round; 1 runs the same kernels one group at a
 * time (one column per launch, groups in order), the unbatched comparison.
 * Both give the same result up to rounding.
 */
matex_status matex_set_batching(matex_ctx* ctx, int32_t one_group_at_a_time);

/*
 * Vector-Jacobian product of the last run's outputs (no counterpart in the
 * paper; the discrete adjoint of Alg. 2 / Alg. 1 as run): given
 *   xbar   device, [N+1][n_rows], dL/dx_out for the run's output rows,
 * writes
 *   dc     device [n], dL/dc_i (original node order), and
 *   damp   device [n_src], dL/da_s, where a_s scales source s's currents as given
 *          at matex_setup (u_s = a_s * u_s,setup): evaluated at the currents the
 *          run used, so after matex_set_sources(a_s * u_s,setup) it is dL/da_s at
 *          that a (a_s = 0 included).  Like dc it is the derivative of the run as
 *          computed: a group whose sources are all at zero builds no Krylov
 *          basis (a zero start vector), so its gradient then has no part from
 *          the exponential term.
 * The Krylov dimensions are those of the last run (as if replayed).  Requires
 * a context set up with opts.tape = 1 or 2 and a preceding matex_run.  With
 * tape = 2 the segments are recomputed from the run's checkpoints first (the
 * recomputed Krylov process follows the run's dimensions; MATEX_ERR_STATE if
 * a recomputed segment retires its column at another step).  Reuses the
 * forward's factors (both matrices are symmetric).  Synchronises the stream.
 */
matex_status matex_grad(matex_ctx* ctx, const double* xbar, double* dc, double* damp);

/*
 * Replace the node capacitances (host [n], original order, all > 0): C + gamma G
 * is refactorised on the host with the existing symbolic structure and its
 * panels re-uploaded (G is unchanged).
 */
matex_status matex_set_caps(matex_ctx* ctx, const double* c);

/*
 * Replace the source currents (host, layout of pwl_v at setup).  The
 * breakpoint times stay those of setup.  Setup skips the segments on which a
 * group has injected nothing since t = 0 (their response is exactly zero);
 * values that would make such a segment, or a group's current at t = 0,
 * non-zero return MATEX_ERR_ARG and change nothing (set up a new context).
 * Scaling the setup currents never does.
 */
matex_status matex_set_sources(matex_ctx* ctx, const double* pwl_v_host);

/*
 * Solve with one of the two factors for ncols right-hand sides:
 *   which = 0: x = (C + gamma G)^{-1} b      which = 1: x = G^{-1} b
 *   b, x   device, [ncols][n] (each column a contiguous n-vector, original order);
 *          may alias.
 */
matex_status matex_solve(matex_ctx* ctx, int32_t which, int32_t ncols, const double* b, double* x);

/*
 * The same solves through the resident rounds' substitution: one CTA per
 * right-hand side runs both triangular sweeps level by level in its shared
 * memory (one launch for all ncols, no atomics: results reproducible bit for
 * bit).  which, ncols, b, x as for matex_solve (device, [ncols][n], original
 * order; may alias).  MATEX_ERR_STATE when the context was set up without
 * it (n > 8192 or the CTA's shared memory too small, krylov 2, tape,
 * tail_eps > 0 or resident = 1).
 */
matex_status matex_solve_resident(matex_ctx* ctx, int32_t which, int32_t ncols, const double* b,
                                  double* x);

/*
 * Device time of the bare batched solve pair (forward and backward
 * substitution of Alg. 1's operator apply, Sec. 3.3.2) on the context's own
 * column buffer, without the moves matex_solve adds around it (no
 * counterpart in the paper; the measurement behind the solve's roofline):
 * which as for matex_solve, or 2 and 3 for the same factors through the
 * resident substitution (one CTA per column; MATEX_ERR_STATE without it);
 * 1 <= ncols <= the buffer width (the largest
 * segment round, rounded up to 8, at least 8); one warm-up, then reps timed
 * solves with CUDA events on the context's stream, in the launch mode the
 * context uses for ncols.  *best_ms receives the fastest, *mean_ms (may be
 * NULL) the mean.  The buffer's values are whatever the last call left.
 * Synchronises the stream.
 */
matex_status matex_time_solve(matex_ctx* ctx, int32_t which, int32_t ncols, int32_t reps,
                              float* best_ms, float* mean_ms);

/*
 * Same solve as matex_solve, for callers that are not allowed to allocate
 * device memory (no counterpart in the paper).  Code running inside another
 * library's allocator or memory-pool callback, or in a process whose device
 * memory is owned by a pool it must not grow, cannot call cudaMalloc; it can
 * still solve with a context built earlier.  This call allocates nothing and
 * uses none of the context's work buffers: its right-hand-side buffers and
 * dependency counters live in one static 16 MiB device array inside the
 * library, held on every device where a context was set up until the process
 * exits.
 *   which, ncols, b, x  as for matex_solve (device pointers, [ncols][n]).
 * Limits: n <= 917,504 nodes and at most 174,761 supernodes in the factor;
 * larger factors get MATEX_ERR_ARG with the limit in matex_last_error().
 * Right-hand sides are processed in chunks that fit the array (fewer columns
 * per chunk for larger n).  Each chunk runs the launch mode the context uses
 * for that column count (per tree level, or one persistent launch).
 * matex_setup does the set-up this call needs on its device: it looks up the
 * array's device address (cudaGetSymbolAddress, which also loads the module
 * that holds the array) and loads every solve kernel, so the first call
 * triggers no lazy module loading either.  Every call shares the one array,
 * and its contents after a call are those of the last chunk: calls that
 * overlap on the GPU (other streams, other host threads, other contexts on
 * the same device) race with each other and must be serialised by the
 * caller.  Synchronises the context's stream.
 */
matex_status matex_solve_noalloc(matex_ctx* ctx, int32_t which, int32_t ncols, const double* b,
                                 double* x);

/*
 * Batched small dense exponentials as used for e^{h H_m} (Eq. 9):
 *   A      device, [batch][m][m] row-major;  h device [batch];  E device [batch][m][m]
 *   E[b] = expm(h[b] * A[b]),  1 <= m <= 20.
 */
matex_status matex_expm(matex_ctx* ctx, int32_t batch, int32_t m, const double* A, const double* h,
                        double* E);

/* Krylov dimension used per (group, segment) by the last run, in the replay_m
 * layout; *count receives the total (write at most cap entries to m_host). */
matex_status matex_get_m(matex_ctx* ctx, int32_t* m_host, int64_t cap, int64_t* count);

/* Sizes: N+1 output times, rows per output, total segments. */
matex_status matex_get_sizes(matex_ctx* ctx, int32_t* n_times, int32_t* n_rows, int64_t* n_segments);

/*
 * Per-kernel-class profile of the runs made while profiling is on.  Each
 * timed unit is bracketed by CUDA events on the context's stream:
 *   class 0 triangular-solve sweeps (all tree levels of one batched solve)
 *   class 1 node-major <-> vector-major moves around the solves
 *   class 2 Gram-Schmidt (dot products, reductions, updates, normalisation)
 *   class 3 small dense work (start norms, residual tests, e^{hH} coefficients)
 *   class 4 recombination + superposition of the group responses
 *   class 5 segment inputs, state hand-off, output permutation and the rest
 * For each class: ms[c] total event time, units[c] timed units, launches[c]
 * kernels, flops[c] and bytes[c] the algorithmic FP64 flops and DRAM bytes
 * of the work done (the minimum the method needs; see the kernels' comments).
 */
#define MATEX_PROF_CLASSES 6
typedef struct matex_profile {
  double ms[MATEX_PROF_CLASSES];
  int64_t units[MATEX_PROF_CLASSES];
  int64_t launches[MATEX_PROF_CLASSES];
  double flops[MATEX_PROF_CLASSES];
  double bytes[MATEX_PROF_CLASSES];
} matex_profile;

/*
 * Failure-injection hook for tests of the bounded waits: while on, every
 * persistent solve gets one dependency that never completes (the last root
 * supernode waits for a child that does not exist).  Its wait gives up after
 * about one second, the kernel returns, and the call reports
 * MATEX_ERR_TIMEOUT; the context stays usable once the hook is off.
 */
matex_status matex_debug_inject_wait(matex_ctx* ctx, int32_t on);

/* on = 1 starts (and zeroes) profiling, on = 0 stops it. */
matex_status matex_set_profiling(matex_ctx* ctx, int32_t on);
matex_status matex_get_profile(matex_ctx* ctx, matex_profile* out);

/*
 * Result of the setup-time autotuner (solve_mode 2): for each measured column
 * count ncols[i] the launch mode chosen (0 persistent, 1 per level) and the
 * best times of both (ms[2i], ms[2i+1]; -1 when read from the cache file named
 * by the environment variable MATEX_AUTOTUNE_CACHE).  Writes at most cap entries;
 * *count receives the number measured.
 */
matex_status matex_get_autotune(matex_ctx* ctx, int32_t* ncols, int32_t* mode, float* ms,
                               int32_t cap, int32_t* count);

/*
 * Column blocks of the level-by-level solve launches (no counterpart in the
 * paper): for each of the *nlev levels of the supernodal tree (leaves first)
 * the number of right-hand sides a thread block of the forward (kb_fwd) and
 * backward (kb_bwd) substitution carries.  With solve_mode 2 and col_block 0
 * the setup-time tuner times 1, 2, 4 and 8 per level and direction at the
 * context's full column count and keeps the fastest; ms (host [2*cap] or
 * NULL) receives the chosen blocks' times (forward, backward per level; -1
 * when not tuned or read from the cache).  Writes at most cap levels.
 */
matex_status matex_get_level_blocks(matex_ctx* ctx, int32_t* kb_fwd, int32_t* kb_bwd, float* ms,
                                    int32_t cap, int32_t* nlev);

/* Setup statistics (ordering, factor sizes, timings). */
matex_status matex_get_setup_stats(matex_ctx* ctx, matex_stats* stats);

/*
 * Host-only check of the setup path, no GPU needed: nested-dissection
 * ordering, supernodal symbolic analysis and L D L^T of diag(dshift) + alpha A
 * (A host CSR as for G; dshift host[n] or NULL), then a CPU forward/backward
 * substitution with exactly the factor panels the GPU kernels read, for
 * ncols right-hand sides b (host [ncols][n], original order) into x (host,
 * same layout).  info (host [5], may be NULL) receives
 * {nnz_L, n_supernodes, n_levels, max_width_seen, nnz_L_exact}.
 */
matex_status matex_host_factor_solve(int64_t n, const int64_t* rowptr, const int32_t* col,
                                     const double* val, const double* dshift, double alpha,
                                     int32_t max_width, int32_t ncols, const double* b, double* x,
                                     int64_t* info);

/*
 * Host-only check of the work plan of the single-column level kernels (the
 * operator apply of Alg. 1 and the input solves of Eq. 5/6 with one
 * right-hand side), built for G given as host CSR as for
 * matex_host_factor_solve (max_width <= 0: the setup's default): the same
 * ordering, symbolic analysis and plan as matex_setup, then every warp's
 * lanes mapped to their rows the way the kernels do it.  info (host [6], may
 * be NULL) receives {levels, forward warps, backward warps, panel rows,
 * supernode columns, mapping errors}.  MATEX_ERR_STATE when a lane lands
 * outside its level, group size or supernode, or a row or column is not
 * taken exactly once.  No GPU needed.
 */
matex_status matex_host_single_column_plan(int64_t n, const int64_t* rowptr, const int32_t* col,
                                           const double* val, int32_t max_width, int64_t* info);

/*
 * Fixed-step trapezoidal integration of Eq. 1 (Eq. 2), the method the paper
 * compares R-MATEX against, on the same batched triangular solves:
 *   (C + h/2 G) x_{n+1} = (C - h/2 G) x_n + h/2 (b_n + b_{n+1}),
 *   b(t) = B u(t) (+ dc_inject when opts.include_dc), all sources at once,
 * from the DC state x_0 = G^{-1} b(0), with h = dt_out / substeps (substeps
 * >= 1).  Writes the states at the output times t_o = o*dt_out into x_out
 * (device, [N+1][n_rows], as matex_run) and, if ms_out (host) is not NULL,
 * the device time of the integration (CUDA events; excludes the one-time host
 * factorisation of C + h/2 G, redone when h changes).  The first call for a
 * given substeps records the step loop as a CUDA graph; later calls replay
 * it.  Uses the current source currents.  Synchronises the stream.
 */
matex_status matex_tr_run(matex_ctx* ctx, int32_t substeps, double* x_out, double* ms_out);

/*
 * Measured FP64 throughput of the current device (no counterpart in the
 * paper; the denominator of the ALU roofline the kernels are reported
 * against): one kernel of independent fused multiply-add chains over every
 * SM, timed with CUDA events; *tflops receives the best of `reps` launches
 * (2 flops per FMA), *ms (host, may be NULL) its duration.  Synchronises the
 * device; allocates 8 bytes of device memory for the call.
 */
matex_status matex_measure_fp64_peak(int32_t reps, double* tflops, double* ms);

const char* matex_last_error(const matex_ctx* ctx);
const char* matex_status_string(matex_status s);
void matex_destroy(matex_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MATEX_H_ */
