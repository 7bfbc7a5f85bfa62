/*
 * lamg_oracle.h -- plain serial FP64 CPU reference of the Lean Algebraic
 * Multigrid (LAMG) path of Livne & Brandt, "Lean Algebraic Multigrid (LAMG):
 * Fast Graph Laplacian Linear Solver" (arXiv 1108.1310).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists so that the tests, the
 * package's smoke check and the benchmark's CPU-baseline leg can check and
 * time the CUDA library against an obviously correct implementation.  The
 * product path (the CUDA library and its Python binding) never links, loads
 * or calls anything in this directory, and this directory includes nothing
 * from the product.
 *
 * Everything is computed in IEEE FP64, round-to-nearest, compiled with
 * -ffp-contract=off (no fused multiply-add) so that every setup float is a
 * fixed function of the inputs.
 *
 * Parity status of each part (see the test files under tests/ for the pins):
 *   Laplacian assembly, GS sweeps, affinity, energy ratio, hub test,
 *   Galerkin operator, coarsest solve, the solution x, the adjoint: pinned.
 *   Aggregate ids themselves: the paper defers the complete aggregation
 *   algorithm to an e-print that is not available; the parallel handshake
 *   rule below is this build's reading.  Its invariants (Sec. 3.4 rules 1,2,5,
 *   q <= 2.5, nesting of stages) are pinned; the particular ids are
 *   "parity unpinned" by the paper and are fixed only by this oracle.
 */
#ifndef LAMG_ORACLE_H
#define LAMG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double   gamma;            /* cycle index, Sec. 4.1 ("gamma = 1.5")             */
    int32_t  k_finest;         /* TVs at the finest level, Sec. 4.1 (4)              */
    int32_t  k_max;            /* TVs at coarse levels grow up to this, Sec. 4.1 (10) */
    int32_t  k_step;           /* TV increase per level (reading: 1)                 */
    int32_t  nu_tv;            /* GS sweeps per TV, Sec. 4.1 (3)                     */
    int32_t  nu1, nu2;         /* pre/post sweeps, Eq. (4.1) (1, 2)                  */
    int32_t  n_coarsest;       /* stop coarsening below this size, Sec. 4.1 (150)    */
    double   q_max;            /* energy-ratio acceptance, Sec. 3.4.5 (2.5)          */
    double   hub_factor;       /* hub test factor, Sec. 3.4.1 footnote (8)           */
    double   weak_tol;         /* weak-edge threshold (reading: 1e-8)                */
    double   alpha_stall;      /* coarsening ratio above which a level is final      */
    double   relax_fast_ratio; /* TV energy ratio per sweep below which GS is "fast" */
    int32_t  max_rounds;       /* aggregation stages per level (reading: 8)          */
    int32_t  max_levels;       /* hierarchy depth limit                              */
    int32_t  dense_max;        /* largest coarsest level solved directly             */
    int32_t  coarse_sweeps;    /* GS sweeps when the coarsest level is too large     */
    double   mu_flat;          /* flat energy correction, Eq. (3.9) (4/3)            */
    uint64_t seed;             /* seed of the counter-based generator                */
    int32_t  agg_rule;         /* the aggregation stages (Sec. 3.4.2):
                                  0: the parallel handshake (reading R9);
                                  1: the paper's sequential scan in node-index order;
                                  2 (default): the same scan in decreasing hashed
                                  priority order (reading R9); at most two stages
                                  for 1 and 2                                         */
    int32_t  elim;             /* 1: low-degree elimination levels before each
                                  aggregation, Sec. 3.2 (default 0: none, as the library) */
    double   elim_min_frac;    /* an elimination round is kept only if it removes at
                                  least this fraction of the level's nodes (reading: 0.1) */
    int32_t  lgmg_nx;          /* > 0: Lean Geometric Multigrid (Sec. 6) on an
                                  lgmg_nx x lgmg_nx periodic 5-point grid: 2x2 aggregates
                                  and red-black colours at every level, gamma at every
                                  level; solve in flat mode with mu_flat = 2.  Default 0 */
    double   mu_adaptive;      /* restriction factor of the adaptive cycle (reading R15: 1) */
    double   gamma_coarse_max; /* cap of the cycle index at coarse levels, Eq. (4.1): 2    */
    int32_t  plain_sums;       /* 1: every setup sum left to right from +0.0 (the plain
                                  definition) instead of the tiered canonical order;
                                  0 (default): the tiered order                         */
    int32_t  gamma_fine_printed; /* 1: gamma^l = gamma wherever |E^l| > .1|E| (Eq. (4.1) as
                                  printed); 0 (default): bounded there as at coarse levels */
    int32_t  recomb_finest;    /* 1 (default): the adaptive cycle recombines at the finest
                                  level too (reading R15); 0: below the finest level only */
    int32_t  relax_rule;       /* 0 (default): multicolour GS on the JP colouring (R2);
                                  1: lexicographic GS (Eq. (2.3)), swept as the level
                                  sets of the lower-triangular dependency graph       */
    int32_t  colour_rule;      /* JP priority (reading R2): 0 (default) degree, then
                                  splitmix64(key + u), then the lower index; 1 degree,
                                  then the lower index (greedy in that order)         */
    int32_t  negative_weights; /* 1: accept nonzero weights of either sign whose rows
                                  have a positive sum (Sec. 5, grids with negative
                                  weights); 0 (default): positive weights only       */
} orc_opts;

typedef struct orc_hier orc_hier;

/* status codes (same meaning as the library's, values fixed here) */
enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_NOT_SYMMETRIC = 2, ORC_ERR_BAD_WEIGHT = 3,
       ORC_ERR_DISCONNECTED = 4, ORC_ERR_RHS_NOT_ZERO_SUM = 5 };

void     orc_default_opts(orc_opts *o);

/* ---- building blocks, exported so the tests can pin each one ---- */
uint64_t orc_splitmix64(uint64_t key);
double   orc_canon_sum(const double *t, int64_t len);
double   orc_canon_dot(const double *a, const double *b, int64_t len);
double   orc_canon_sum_global(const double *t, int64_t len);
int32_t  orc_validate(int64_t n, const int64_t *rp, const int32_t *col, const double *w);
/* the same for signed weights: nonzero and finite, every row's sum positive */
int32_t  orc_validate_signed(int64_t n, const int64_t *rp, const int32_t *col, const double *w);
/* Several graphs as one block-diagonal union: graph g owns nodes
 * [gptr[g], gptr[g+1]).  No edge may join two graphs (ORC_ERR_ARG); each graph
 * must be connected (ORC_ERR_DISCONNECTED). */
int32_t  orc_validate_graphs(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                             int32_t ngraphs, const int64_t *gptr);
void     orc_laplacian_dense(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                             double *A /* n*n row-major */);
int32_t  orc_colour(int64_t n, const int64_t *rp, const int32_t *col, uint64_t key,
                    int32_t *colour /* out n */);
/* the lexicographic order's level sets (relax_rule 1): returns the colour count */
int32_t  orc_colour_lex(int64_t n, const int64_t *rp, const int32_t *col, int32_t *colour /* out n */);
void     orc_gs_sweep_lex(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                          const double *b, double *x);
void     orc_gs_sweep_colour(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                             const int32_t *colour, int32_t ncolours, const double *b, double *x);
void     orc_edge_scores(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                         int32_t K, const double *X, double q_max, double weak_tol,
                         double *aff, double *q, double *score);
void     orc_hubs(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                  double hub_factor, uint8_t *hub);
int32_t  orc_dense_pinv_solve(int64_t n, const double *A, const double *b, double *x);

/* ---- setup ---- */
int32_t  orc_setup(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                   const orc_opts *o, orc_hier **out);
/* The hierarchy of the block-diagonal union of ngraphs graphs (same setup
 * rules on the union; the coarsest direct solve, the level-1 mean projection,
 * the zero-sum test and the stopping test act per component / per graph). */
int32_t  orc_setup_graphs(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                          int32_t ngraphs, const int64_t *gptr, const orc_opts *o, orc_hier **out);
void     orc_free(orc_hier *h);
int32_t  orc_num_levels(const orc_hier *h);
/* info[0..15]: n, nnz, ncolours, K, nc, rounds, sel_round, coarsest, stop_reason,
 * alpha (as double bits), gamma_l (double bits), tv_ratio (double bits), jp_rounds */
void     orc_level_info(const orc_hier *h, int32_t l, int64_t *info);
void     orc_level_csr(const orc_hier *h, int32_t l, int64_t *rp, int32_t *col, double *w);
void     orc_level_colour(const orc_hier *h, int32_t l, int32_t *colour);
void     orc_level_tv(const orc_hier *h, int32_t l, double *X);
void     orc_level_scores(const orc_hier *h, int32_t l, double *aff, double *q, double *score);
void     orc_level_agg(const orc_hier *h, int32_t l, int32_t *agg, int32_t *state, uint8_t *hub);
/* One level's aggregation from its CSR, edge scores and hub flags (the setup's
 * rule).  info[0..3]: nc, rounds, selected round, alpha (double bits). */
void     orc_aggregate(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                       const double *score, const uint8_t *hub, const orc_opts *o, int32_t level,
                       int32_t *agg, int32_t *state, int64_t *info);
/* One level's Galerkin operator from its CSR and aggregates; col_c and w_c hold
 * up to rp[n] entries.  Returns the coarse nnz. */
int64_t  orc_galerkin(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                      const int32_t *agg, int64_t nc, int64_t *rp_c, int32_t *col_c, double *w_c);
/* the eliminated set of a graph (Sec. 3.2, reading R20) for the sweep key `key`:
 * cidx[u] = rank of u among the kept nodes, -1 for u in F; returns |F| */
int64_t  orc_elim_set(int64_t n, const int64_t *rp, const int32_t *col, uint64_t key, int32_t *cidx);
/* level l followed by an elimination level: cidx[u] = coarse index of u, or -1 for u in F */
void     orc_level_elim(const orc_hier *h, int32_t l, int32_t *cidx);

/* ---- solve ---- */
/* Cycles until ||b - A x||_2 <= tol ||b||_2 or max_cycles. x: in = initial guess, out = result.
 * res_hist (may be NULL): max_cycles+1 entries, ||b-Ax|| before the first cycle and after each. */
int32_t  orc_solve(const orc_hier *h, const double *b, double *x, double tol, int32_t max_cycles,
                   int32_t adaptive, double *res_hist, int32_t *cycles_out);
/* Exactly one cycle followed by the mean projection (for cycle-level comparisons). */
int32_t  orc_cycle(const orc_hier *h, const double *b, double *x, int32_t adaptive);
/* Solve A lambda = g - mean(g) and the edge gradient dw_e = -(lam_u - lam_v)(x_u - x_v). */
int32_t  orc_adjoint(const orc_hier *h, const double *x, const double *g, double *lambda,
                     const int32_t *eu, const int32_t *ev, int64_t m, double *dw,
                     double tol, int32_t max_cycles, int32_t adaptive);

#ifdef __cplusplus
}
#endif
#endif
