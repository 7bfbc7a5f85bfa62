/*
 * lamg.h -- C-ABI of the GB300 (sm_103a) Lean Algebraic Multigrid library.
 *
 * Solves the compatible graph-Laplacian system of Livne & Brandt, "Lean
 * Algebraic Multigrid (LAMG): Fast Graph Laplacian Linear Solver", arXiv
 * 1108.1310, Sec. 1, Eq. (1.3):
 *
 *     A x = b,   1^T x = 0,
 *
 * A the Laplacian of a connected graph with positive weights (Eq. (1.2)),
 * b zero-sum.  lamg_setup builds the multilevel hierarchy of Sec. 4.1
 * (test-vector relaxation, affinities Eq. (3.5), energy ratios Eq. (3.12),
 * caliber-1 aggregation Sec. 3.4, Galerkin operators Eq. (2.5)); lamg_solve
 * runs the cycles of Sec. 4.2 (Gauss-Seidel Eq. (2.3), restriction and
 * prolongation Eqs. (2.5)-(2.6), flat energy correction Eq. (3.9) or iterate
 * recombination Eq. (3.13), dense coarsest solve, mean subtraction).
 *
 * Conventions for every entry point:
 *  - Graph input: the off-diagonal pattern of A as a CSR holding both
 *    directions of every edge, columns strictly increasing within each row,
 *    no self loops, w_uv == w_vu bit for bit, w > 0 and finite.  a_uu is
 *    implied (sum of the row's weights).  Fewer than 2^31 stored entries.
 *  - "device" pointers must be device-accessible memory of the current CUDA
 *    device; "host" pointers ordinary host memory.  The caller owns all
 *    arrays it passes.  lamg_setup copies what it needs; the caller may free
 *    its inputs when lamg_setup returns.  The handle owns the hierarchy and
 *    its workspaces until lamg_free.
 *  - All device work is ordered on the given stream (0 = legacy default).
 *    Calls that return statistics or convergence decisions synchronise the
 *    stream before returning; their device outputs are then complete.
 *  - Every function returns a lamg_status and never aborts; the text of the
 *    last error of the calling thread is available from lamg_last_error().
 *  - A handle may be used by one thread at a time.
 */
#ifndef LAMG_H
#define LAMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lamg_ctx *lamg_handle;
typedef void *lamg_stream;   /* a cudaStream_t */

typedef enum {
    LAMG_OK = 0,
    LAMG_ERR_ARG = 1,              /* malformed argument or CSR                      */
    LAMG_ERR_NOT_SYMMETRIC = 2,    /* w_uv != w_vu or a missing reverse entry        */
    LAMG_ERR_BAD_WEIGHT = 3,       /* w <= 0, NaN or Inf                              */
    LAMG_ERR_DISCONNECTED = 4,     /* the graph has more than one component           */
    LAMG_ERR_RHS_NOT_ZERO_SUM = 5, /* |1^T b| > 1e-10 ||b||_1 (Sec. 1 needs b zero-sum) */
    LAMG_ERR_OOM = 6,              /* device allocation failed                        */
    LAMG_ERR_CUDA = 7,             /* a CUDA call failed (message in lamg_last_error) */
    LAMG_ERR_NOT_CONVERGED = 8,    /* max_cycles reached above tol; x is the iterate  */
    LAMG_ERR_TIMEOUT = 9           /* a bounded device wait ran out                   */
} lamg_status;

typedef enum { LAMG_FP64 = 0, LAMG_FP32_IR = 1 } lamg_precision;

/* Parameters of Sec. 4; lamg_default_options fills the paper's values and the
 * build's readings of the points the paper leaves open. */
typedef struct {
    int32_t  struct_size;      /* sizeof(lamg_options), set by lamg_default_options;
                                  lamg_setup rejects any other value with LAMG_ERR_ARG,
                                  so a caller built against another layout of this
                                  struct fails instead of passing misread fields       */
    double   gamma;            /* cycle index (Sec. 4.1): 1.5                          */
    int32_t  k_finest;         /* TVs at the finest level (Sec. 4.1): 4                 */
    int32_t  k_max;            /* TVs grow up to this at coarse levels: 10 (max 16)     */
    int32_t  k_step;           /* TV growth per level: 1                                */
    int32_t  nu_tv;            /* GS sweeps per TV (Sec. 4.1): 3                        */
    int32_t  nu1, nu2;         /* pre/post relaxations (Eq. (4.1)): 1, 2                */
    int32_t  n_coarsest;       /* stop coarsening below this many nodes: 150           */
    double   q_max;            /* energy-ratio acceptance (Sec. 3.4.5): 2.5             */
    double   hub_factor;       /* hub test (Sec. 3.4.1 footnote): 8                     */
    double   weak_tol;         /* weak-edge threshold: 1e-8                             */
    double   alpha_stall;      /* a level whose best coarsening ratio exceeds this is final: 0.95 */
    double   relax_fast_ratio; /* TV energy ratio per sweep at or below which GS counts as
                                  fast and the level is final; <= 0 disables (default 0) */
    int32_t  max_rounds;       /* aggregation stages per level: 8                       */
    int32_t  max_levels;       /* depth limit: 100                                      */
    int32_t  dense_max;        /* largest coarsest level solved by the dense inverse: 1024 */
    int32_t  coarse_sweeps;    /* GS sweeps when the coarsest level is larger: 5       */
    double   mu_flat;          /* flat energy correction (Eq. (3.10), Q = 2): 4/3      */
    uint64_t seed;             /* seed of the counter-based generator: 1               */
    int32_t  adaptive;         /* 1: iterate recombination (Eq. (3.13)); 0: flat mu    */
    int32_t  max_cycles;       /* solve limit: 200                                     */
    int32_t  ir_inner;         /* FP32 cycles per FP64 refinement step: 2               */
    int32_t  validate;         /* 1: check the input graph (symmetry, weights, connectivity) */
    int32_t  keep_setup_data;  /* 1: keep TVs, affinities, energy ratios for inspection */
    int32_t  project_rhs;      /* 0: a b that is not zero-sum (per graph, per column) is
                                  rejected with LAMG_ERR_RHS_NOT_ZERO_SUM; 1: the solve
                                  uses b minus its mean instead (per graph, per column),
                                  the compatible part of b (Sec. 1), and leaves the
                                  caller's b unchanged                                    */
    double   mu_adaptive;      /* restriction factor of the adaptive cycle (recombination,
                                  Eq. (3.13)): 1 (default) or a mild flat correction
                                  on top of recombination; see the oracle's figures.
                                  Must lie in (0, 4), else LAMG_ERR_ARG                 */
    double   gamma_coarse_max; /* cap of the cycle index gamma^l at the coarse levels
                                  (|E^l| <= .1 |E|), Eq. (4.1): 2 as printed.  1 makes
                                  the coarse part of the cycle a V-cycle.  Must lie in
                                  [1, 2], else LAMG_ERR_ARG                             */
    int32_t  elim;             /* 1: low-degree elimination levels before each aggregation
                                  (Sec. 3.2): an independent set F of degree-1..4 nodes,
                                  taken by one sweep in decreasing hashed priority, is
                                  replaced by the Schur complement on the rest; the level
                                  above it then has gamma = 1 and no relaxation, and the
                                  cycle back-substitutes F exactly.  Default 0.           */
    double   elim_min_frac;    /* an elimination round is kept only if it removes at least
                                  this fraction of the level's nodes: 0.1                 */
    int32_t  lgmg_nx;          /* > 0: Lean Geometric Multigrid (Sec. 6) on an
                                  lgmg_nx x lgmg_nx periodic 5-point grid numbered row by
                                  row (n = lgmg_nx^2, else LAMG_ERR_ARG): 2x2 aggregates
                                  and red-black colours at every level, gamma at every
                                  level; the paper's setting solves with adaptive = 0 and
                                  mu_flat = 2.  Coarsening stops below n_coarsest nodes or
                                  at an odd side or a side below 6.  Default 0           */
    int32_t  agg_rule;         /* aggregation stages (Sec. 3.4.2):
                                  2 (default): the paper's scan, visiting the undecided
                                  nodes in decreasing priority splitmix64(key_l + u)
                                  (ties to the lower index), at most two stages; the
                                  GPU runs it in parallel rounds that reproduce the
                                  sequential scan exactly;
                                  1: the same scan in node-index order, the paper's
                                  sequential form (deeper rounds on grids);
                                  0: the parallel handshake of mutual best neighbours  */
    int32_t  recomb_finest;    /* 1 (default): the adaptive cycle also recombines the
                                  iterates of the finest level (Eq. (3.13)), so that
                                  its coarse correction is energy-corrected too;
                                  0: recombination below the finest level only       */
    int32_t  relax_rule;       /* 0 (default): multicolour Gauss-Seidel on the JP
                                  colouring; 1: lexicographic Gauss-Seidel (Eq. (2.3))
                                  exactly, swept as the level sets of the lower-
                                  triangular dependency graph (colour[u] = 1 + the
                                  largest colour of a lower-index neighbour), for the
                                  TV sweeps and the cycle alike                      */
    int32_t  sb_work32;        /* a level whose entries + rows are at most this runs all
                                  its ops on one block of the cycle engine (block
                                  barriers instead of grid barriers), FP32 cycles;
                                  0 (default): 16384.  A performance knob only: the
                                  results do not depend on it beyond rounding        */
    int32_t  sb_work64;        /* the same for FP64 cycles; 0 (default): 16384        */
    int32_t  tail_work32;      /* a colour with at most this many entries joins a run
                                  of small colours swept by one block, FP32; 0
                                  (default): 2048                                     */
    int32_t  tail_work64;      /* the same for FP64; 0 (default): 512                  */
    int32_t  colour_rule;      /* priority of the Jones-Plassmann colouring, which
                                  equals the greedy colouring in that order:
                                  0 (default): degree, then splitmix64(key_l + u),
                                  then the lower index; 1: degree, then the lower
                                  index (red-black on a grid numbered by position) */
    int32_t  negative_weights; /* 1: accept graphs with negative edge weights (Sec. 5,
                                  grids with negative weights): every weight nonzero
                                  and finite, every row's sum of weights positive
                                  (else LAMG_ERR_BAD_WEIGHT); the Laplacian should be
                                  positive semi-definite.  The energy-ratio test uses
                                  |w_uv| in the nodal energies.  0 (default): weights
                                  must be positive                                   */
} lamg_options;

typedef struct {
    int32_t levels;            /* hierarchy depth L                                     */
    int32_t cycles;            /* cycles run by the last solve (FP32 cycles under IR)   */
    int32_t outer_steps;       /* FP64 refinement steps (IR) or cycles (FP64)          */
    int32_t status;            /* status of the last solve                             */
    double  rel_res;           /* ||b - A x||_2 / ||b||_2 at exit (FP64)                */
    double  acf;               /* (r_p / r_0)^(1/p), Sec. 5.1                           */
    double  t_setup_s;         /* wall time of lamg_setup                              */
    double  t_solve_s;         /* wall time of the last solve                          */
    int64_t nnz_total;         /* stored off-diagonal entries over all levels          */
    int64_t bytes_per_cycle;   /* algorithmic bytes of one FP64 cycle (model)          */
    int64_t bytes_per_cycle32; /* same for one FP32 cycle                              */
} lamg_stats;

void        lamg_default_options(lamg_options *opt);
const char *lamg_last_error(void);

/* lamg_setup -- build the hierarchy (Sec. 4.1).
 *  n        number of nodes, 1 <= n < 2^31
 *  row_ptr  device, int64[n+1], row_ptr[0] = 0
 *  col      device, int32[row_ptr[n]]
 *  w        device, FP64 (w_is_fp32 = 0) or FP32 (w_is_fp32 = 1) [row_ptr[n]]
 *  opt      host, may be NULL for defaults
 *  out      host; receives the handle (NULL on error)
 * Errors: LAMG_ERR_ARG / NOT_SYMMETRIC / BAD_WEIGHT / DISCONNECTED when
 * opt->validate is set, LAMG_ERR_OOM, LAMG_ERR_CUDA. */
lamg_status lamg_setup(int64_t n, const int64_t *row_ptr, const int32_t *col, const void *w,
                       int32_t w_is_fp32, const lamg_options *opt, lamg_stream stream,
                       lamg_handle *out);

/* lamg_setup_graphs -- one hierarchy for a block-diagonal union of
 * num_graphs independent graphs (the batched many-graphs form; the paper
 * treats one connected graph, Sec. 1, and says to split a disconnected one
 * into its components).  Graph g owns the level-1 nodes
 * [graph_ptr[g], graph_ptr[g+1]) of the CSR, which holds all graphs.
 *  graph_ptr  HOST int64[num_graphs + 1], graph_ptr[0] = 0,
 *             graph_ptr[num_graphs] = n, strictly increasing; copied.
 * The setup rules of Sec. 4.1 run unchanged on the union (they are local to
 * nodes and edges; the stopping tests use the union's totals).  Per graph:
 * the zero-sum test on b, the level-1 mean projection and the stopping test
 * ||r_g|| <= tol ||b_g|| of lamg_solve; the dense coarsest solve uses
 * A + sum_K 1_K 1_K^T / n_K over the coarsest level's components K.  A graph
 * coarsened to one isolated node is left unchanged by relaxation.
 * Errors as lamg_setup, plus: an edge joining two graphs, or graph_ptr
 * malformed: LAMG_ERR_ARG; a graph not connected: LAMG_ERR_DISCONNECTED
 * (with opt->validate).  lamg_solve, lamg_solve_host, lamg_cycle and
 * lamg_adjoint work per graph on such a handle (st->rel_res is the largest
 * per-graph relative residual); lamg_solve_batched needs num_graphs = 1. */
lamg_status lamg_setup_graphs(int32_t num_graphs, const int64_t *graph_ptr, int64_t n,
                              const int64_t *row_ptr, const int32_t *col, const void *w,
                              int32_t w_is_fp32, const lamg_options *opt, lamg_stream stream,
                              lamg_handle *out);

/* lamg_graph_residuals -- per-graph ||b_g - A x_g|| / ||b_g|| of the last
 * lamg_solve (or lamg_solve_host / lamg_adjoint) on a handle from
 * lamg_setup_graphs.  rel_res_host: host double[num_graphs].  LAMG_ERR_ARG for
 * a single-graph handle or before any solve. */
lamg_status lamg_graph_residuals(lamg_handle h, double *rel_res_host);

/* lamg_solve -- cycles of Sec. 4.2 until ||b - A x||_2 <= tol ||b||_2.
 *  b  device FP64[n], zero-sum (LAMG_ERR_RHS_NOT_ZERO_SUM otherwise, unless
 *     the options set project_rhs: then b minus its mean is solved for, and
 *     ||b - mean|| is the norm of the stopping test)
 *  x  device FP64[n]; in: initial guess, out: the zero-mean iterate
 *  precision  LAMG_FP64: FP64 cycles.  LAMG_FP32_IR: FP32 cycles inside FP64
 *             iterative refinement (outer residual, mean projection and the
 *             coarsest solve in FP64).
 *  st  host, may be NULL.
 * Returns LAMG_ERR_NOT_CONVERGED (x valid) when max_cycles is reached. */
lamg_status lamg_solve(lamg_handle h, const double *b, double *x, double tol,
                       lamg_precision precision, lamg_stream stream, lamg_stats *st);

/* lamg_solve_host -- lamg_solve with host arrays; the host<->device copies
 * run on the stream inside the call (end-to-end form). */
lamg_status lamg_solve_host(lamg_handle h, const double *b_host, double *x_host, double tol,
                            lamg_precision precision, lamg_stream stream, lamg_stats *st);

/* lamg_solve_batched -- nrhs right-hand sides on one hierarchy.  The setup
 * is reused (Sec. 1: once the hierarchy exists, further right-hand sides
 * cost only cycles), and up to 128 columns at a time run through one cycle
 * program whose kernels gather 4 interleaved columns per neighbour (SpMM).
 *  B, X  device FP64, row-interleaved: entry (u, j) at [u * ld + j], ld >= nrhs.
 *        X in: initial guesses, out: zero-mean iterates.
 *  Every column of B must be zero-sum (LAMG_ERR_RHS_NOT_ZERO_SUM names the
 *  first one that is not), unless the options set project_rhs: then each
 *  column's mean is subtracted on the device copy.  Each column has its own recombination
 *  coefficients, mean projection and stopping test; the call returns when all
 *  columns have reached tol (LAMG_ERR_NOT_CONVERGED, X valid, otherwise).
 *  st: host array of nrhs stats (cycles/outer_steps: when that column
 *  converged; rel_res: at exit), may be NULL. */
lamg_status lamg_solve_batched(lamg_handle h, int32_t nrhs, const double *B, double *X,
                               int64_t ld, double tol, lamg_precision precision,
                               lamg_stream stream, lamg_stats *st);

/* lamg_autotune_batched -- picks the column chunk of lamg_solve_batched
 * (columns per engine run: 16, 32, 64 or 128) for this handle by timing one
 * refinement step of nrhs columns at each chunk (CUDA events on `stream`),
 * and keeps the fastest in the handle.  chosen_cols (host, may be NULL)
 * receives it; ms_host (host double[4], may be NULL) the four step times.
 * Needs a single-graph handle (LAMG_ERR_ARG otherwise).  Synchronises. */
lamg_status lamg_autotune_batched(lamg_handle h, int32_t nrhs, lamg_precision precision,
                                  lamg_stream stream, int32_t *chosen_cols, double *ms_host);

/* lamg_set_batch_cols -- sets the column chunk directly (a value cached from
 * an earlier lamg_autotune_batched): 0 (the default, 128) or a power of two
 * in [4, 128]; LAMG_ERR_ARG otherwise. */
lamg_status lamg_set_batch_cols(lamg_handle h, int32_t cols);

/* lamg_adjoint -- gradient of a scalar loss L(x) of the solution x = A^+ b.
 *  Given g = dL/dx (device FP64[n]) it solves A lambda = g - mean(g) with the
 *  same hierarchy (A is symmetric), so dL/db = lambda, and, for the m edges
 *  (eu[e], ev[e]) (device int32[m]), dL/dw_e = -(lambda_u - lambda_v)(x_u - x_v),
 *  from dA/dw_uv = (e_u - e_v)(e_u - e_v)^T (Eq. (1.2)).
 *  x       device FP64[n], the solution of the forward solve
 *  lambda  device FP64[n], out
 *  dw      device, FP64 (dw_is_fp32 = 0) or FP32 [m], out; NULL skips it */
lamg_status lamg_adjoint(lamg_handle h, const double *x, const double *g, double *lambda,
                         const int32_t *eu, const int32_t *ev, int64_t m, void *dw,
                         int32_t dw_is_fp32, double tol, lamg_precision precision,
                         lamg_stream stream, lamg_stats *st);

/* lamg_free -- release the handle and everything it owns (NULL is a no-op). */
void lamg_free(lamg_handle h);

/* ---- introspection (tests and benchmarks) ---- */

/* Per-level summary.  info[0..15]: n, nnz, ncolours, K, nc, rounds, sel_round,
 * coarsest, stop_reason, alpha (FP64 bits), gamma_l (FP64 bits), tv_ratio (FP64
 * bits), jp_rounds, dense (1 if the coarsest is solved by the dense inverse),
 * elim (1 if the next level is this level's Schur complement), nF (eliminated
 * nodes). */
lamg_status lamg_level_info(lamg_handle h, int32_t level, int64_t *info_host);

/* Copy one per-level array to host memory.  Fields (natural node order):
 *  0 row_ptr int64[n+1]   1 col int32[nnz]   2 w FP64[nnz]   3 colour int32[n]
 *  4 agg int32[n]         5 state int32[n]   6 hub uint8[n]
 *  7 tv FP64[n*K]         8 affinity FP64[nnz]  9 q FP64[nnz]   10 score FP64[nnz]
 *  11 cidx int32[n]: on a level followed by elimination, the coarse index of each
 *     node, -1 for the eliminated nodes
 * Fields 7-9 need keep_setup_data.  Returns LAMG_ERR_ARG for a field that the
 * level does not have. */
lamg_status lamg_level_copy(lamg_handle h, int32_t level, int32_t field, void *host_dst,
                            int64_t bytes);

/* Run exactly one cycle plus the mean subtraction on device x (FP64 cycles). */
lamg_status lamg_cycle(lamg_handle h, const double *b, double *x, int32_t adaptive,
                       lamg_stream stream);

/* ---- allocation-free cycle (a library addition: the paper has no counterpart) ----
 *
 * Does what lamg_cycle does -- one cycle plus the mean subtraction on device
 * x, FP64 arithmetic, same results -- but allocates no device or host memory.
 * It is for callers that cannot allocate inside their loop: a Krylov solver
 * applying one cycle per iteration as a preconditioner under a fixed memory
 * budget, or a serving loop where an allocation could stall on the device or
 * fail once the memory is committed elsewhere.
 *
 *  - The handle must already own its solve buffers and the one-cycle program
 *    for this `adaptive` value: call lamg_cycle once with the same `adaptive`
 *    first (lamg_solve creates the buffers but not that program).  An
 *    unprepared handle gets LAMG_ERR_ARG and nothing runs.
 *  - The run's scratch (one row of 8 partial sums per engine block, the grid
 *    barrier's two words and an error word) is a fixed 33,024-byte array in
 *    the library's device image, one per device, with room for at most 512
 *    engine blocks; a device whose engine grid is larger (SM count x resident
 *    blocks per SM) is rejected with LAMG_ERR_ARG.  The first call on a device
 *    looks the array's address up, with that device current; make this first
 *    call before any stream capture begins.  Every call clears the barrier and
 *    error words before its launch.
 *  - The array is shared by every handle on the device: calls whose GPU work
 *    overlaps (issued on different streams or from different threads) race on
 *    it and on the handle, and give wrong results.  Serialise them.
 *  - Synchronises `stream` before returning; LAMG_ERR_TIMEOUT as for lamg_cycle.
 */
lamg_status lamg_cycle_noalloc(lamg_handle h, const double *b, double *x, int32_t adaptive,
                               lamg_stream stream);

/* lamg_barrier_selftest -- diagnostic of the failure path of the cycle
 * engine's grid barrier (no paper counterpart).  Launches the barrier alone on
 * the engine's grid.  hold_one_block = 0: every block arrives; returns
 * LAMG_OK.  hold_one_block = 1: one block never arrives, the others give up
 * after the bounded wait (one to two seconds), set the error word and return;
 * the call returns LAMG_ERR_TIMEOUT and the context stays usable.  Nothing
 * faults or hangs.  Synchronises `stream`. */
lamg_status lamg_barrier_selftest(int32_t hold_one_block, lamg_stream stream);

/* Profiling of the cycle engine: average device time in milliseconds (CUDA
 * events on the solve's stream) and count of the engine launches -- one per
 * FP64 cycle, or per FP32-in-FP64 refinement step -- made while profiling is
 * on, and the model bytes of one launch (the cycles it runs plus the FP64
 * residual, update and projection).  enable = 1 resets the counters and
 * starts recording; 0 stops. */
lamg_status lamg_profile(lamg_handle h, int32_t enable, double *avg_ms, int64_t *count,
                         int64_t *bytes_per_launch);

/* The cycle engine's op timer, an introspection aid with no counterpart in the
 * paper.  mode 1: start timing on this handle (allocates one 128 KB table on the
 * device, zeroed); block 0 then reads its clock around every op of every later
 * engine launch of h, which adds a little time to each op.  mode 0: copy the
 * rows of the table with a non-zero count into the caller's host arrays (at
 * most cap rows; *n_rows gets the number of such rows, which may exceed cap),
 * then zero the table; timing continues.  mode -1: stop and free the table.
 * A row is (level, op type, single_block, count, total ns): op types are the
 * engine's op codes 0..31 in the order OP_SWEEP, OP_SWEEP_RUN, OP_RESID,
 * OP_RESTRICT, OP_ZERO, OP_COARSE, OP_PROLONG, OP_RECOMB_DOTS,
 * OP_RECOMB_APPLY, OP_MEAN_PART, OP_MEAN_APPLY, OP_IR_PREP, OP_IR_UPDATE,
 * OP_MEAN64_PART, OP_MEAN64_APPLY, OP_RES64, OP_NORM64_FIN, OP_SWEEP_SMEM,
 * OP_GMEAN_PART, OP_GMEAN_APPLY, OP_GMEAN64_PART, OP_GMEAN64_APPLY, OP_GNORM64,
 * OP_TAIL_PRE, OP_TAIL_RUN, OP_ELIM_RESTRICT, OP_ELIM_PROLONG, OP_ELIM_BACK;
 * single_block 1 marks ops that block 0 ran alone.  The arrays may be NULL when
 * cap is 0.  Errors: LAMG_ERR_ARG for a NULL handle or a bad mode. */
lamg_status lamg_op_times(lamg_handle h, int32_t mode, int32_t cap, int32_t *level, int32_t *op,
                          int32_t *single_block, int64_t *count, double *total_ns, int32_t *n_rows);

/* Number of this library's kernel launches since it was loaded (a
 * cooperative engine launch counts once). */
lamg_status lamg_launch_count(int64_t *count_host);

#ifdef __cplusplus
}
#endif
#endif
