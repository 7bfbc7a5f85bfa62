/*
 * lamg_oracle.c -- plain serial FP64 CPU reference of the LAMG path
 * (Livne & Brandt, arXiv 1108.1310).  TEST INFRASTRUCTURE ONLY: used by the
 * tests, the smoke check and the benchmark's CPU-baseline leg; never by the
 * product.  Compile with -ffp-contract=off.
 *
 * Section/equation references are to the paper.  Where the paper is silent or
 * garbled the build's reading is stated at the function that implements it.
 */
#include "lamg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Options                                                                    */
/* ------------------------------------------------------------------------- */

void orc_default_opts(orc_opts *o) {
    o->gamma = 1.5;            /* Sec. 4.1 */
    o->k_finest = 4;           /* Sec. 4.1 */
    o->k_max = 10;             /* Sec. 4.1 */
    o->k_step = 1;             /* reading: K grows by 1 per level up to k_max */
    o->nu_tv = 3;              /* Sec. 4.1 */
    o->nu1 = 1;                /* Eq. (4.1) */
    o->nu2 = 2;                /* Eq. (4.1) */
    o->n_coarsest = 150;       /* Sec. 4.1 */
    o->q_max = 2.5;            /* Sec. 3.4.5, after Eq. (3.12) */
    o->hub_factor = 8.0;       /* Sec. 3.4.1 footnote */
    o->weak_tol = 1e-8;        /* weak-edge filter threshold (reading), Sec. 3.4.2 */
    o->alpha_stall = 0.95;     /* reading: aggregation that removes <5% of nodes stops */
    o->relax_fast_ratio = 0.0; /* fast-relaxation stopping test, Sec. 4.1: off by default (<= 0) */
    o->max_rounds = 8;
    o->max_levels = 100;
    o->dense_max = 1024;
    o->coarse_sweeps = 5;
    o->mu_flat = 4.0 / 3.0;    /* Eq. (3.10) with Q = 2 */
    o->seed = 1;
    o->agg_rule = 2;           /* the paper's scan (Sec. 3.4.2) in hashed priority order */
    o->elim = 0;               /* no elimination levels (as the library) */
    o->elim_min_frac = 0.1;    /* elimination rounds stop when F is small (reading), Sec. 3.2 */
    o->lgmg_nx = 0;            /* algebraic coarsening */
    o->mu_adaptive = 1.0;      /* reading R15: recombination replaces the flat correction */
    o->gamma_coarse_max = 2.0; /* Eq. (4.1): min{2, ...} at coarse levels */
    o->plain_sums = 0;         /* the tiered canonical order of the setup sums */
    o->gamma_fine_printed = 0; /* reading R13: the fine-level index is bounded too */
    o->recomb_finest = 1;      /* reading R15: recombination at the finest level too */
    o->relax_rule = 0;         /* multicolour GS on the JP colouring (reading R2) */
    o->colour_rule = 0;        /* JP priority: degree, then the hashed key, then index */
    o->negative_weights = 0;   /* positive weights only (as the library) */
}

/* ------------------------------------------------------------------------- */
/* Counter-based generator: splitmix64 (Steele, Lea & Flood 2014).             */
/* orc_splitmix64(k) is the first output of splitmix64 seeded with k.          */
/* ------------------------------------------------------------------------- */

uint64_t orc_splitmix64(uint64_t key) {
    uint64_t z = key + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Stream keys per level: JP priorities (odd slot) and TV draws (even slot). */
static uint64_t colour_key(uint64_t seed, int32_t level) {
    return orc_splitmix64(orc_splitmix64(seed) ^ (0x100000000ULL * (uint64_t)(2 * level + 1)));
}
static uint64_t tv_key(uint64_t seed, int32_t level) {
    return orc_splitmix64(orc_splitmix64(seed) ^ (0x100000000ULL * (uint64_t)(2 * level + 2)));
}
/* elimination scan order: the colour key's form with the top bit set */
static uint64_t elim_key(uint64_t seed, int32_t level) {
    return orc_splitmix64(orc_splitmix64(seed) ^ (0x100000000ULL * (uint64_t)(2 * level + 1)) ^ (1ULL << 63));
}

/* aggregation scan order (agg_rule 2): the TV key's form with the top bit set */
static uint64_t agg_key(uint64_t seed, int32_t level) {
    return orc_splitmix64(orc_splitmix64(seed) ^ (0x100000000ULL * (uint64_t)(2 * level + 2)) ^ (1ULL << 63));
}

/* TV initial value "random[-1,1]" (Sec. 3.3.1): the top 53 bits of the draw as a
 * uniform t in [0,1), then 2t - 1 (both steps exact in FP64). */
static double tv_uniform(uint64_t z) {
    double t = (double)(z >> 11) * 0x1.0p-53;
    return 2.0 * t - 1.0;
}

/* ------------------------------------------------------------------------- */
/* Canonical summation order (build reading; every setup float that feeds an   */
/* integer decision is summed this way on both sides).                         */
/*   len <= 32   : left to right from +0.0.                                    */
/*   len <= 512  : 32 partial sums p_j = t_j + t_{j+32} + ... (left to right), */
/*                 then the halving tree p_j += p_{j+h}, h = 16, 8, 4, 2, 1;   */
/*                 the result is p_0.                                          */
/*   len  > 512  : 1024 partial sums p_j = t_j + t_{j+1024} + ...; each group  */
/*                 of 32 consecutive p_j is reduced by the halving tree, and   */
/*                 the 32 group results by the halving tree again.             */
/* ------------------------------------------------------------------------- */

/* Plain order (option plain_sums): every canonical sum becomes one left-to-right
 * sum from +0.0, the textbook definition.  The setup sets this switch for the
 * duration of one hierarchy build; the oracle is serial. */
static int g_plain_sums = 0;

static double sum_left_to_right(const double *t, int64_t len) {
    double s = 0.0;
    for (int64_t i = 0; i < len; i++) s = s + t[i];
    return s;
}

static double tree32(double *p) {
    for (int h = 16; h >= 1; h /= 2)
        for (int j = 0; j < h; j++) p[j] = p[j] + p[j + h];
    return p[0];
}

double orc_canon_sum(const double *t, int64_t len) {
    if (g_plain_sums || len <= 32) return sum_left_to_right(t, len);
    if (len <= 512) {
        double p[32];
        for (int j = 0; j < 32; j++) {
            p[j] = 0.0;
            for (int64_t i = j; i < len; i += 32) p[j] = p[j] + t[i];
        }
        return tree32(p);
    }
    double p[1024], q[32];
    for (int j = 0; j < 1024; j++) {
        p[j] = 0.0;
        for (int64_t i = j; i < len; i += 1024) p[j] = p[j] + t[i];
    }
    for (int g = 0; g < 32; g++) q[g] = tree32(p + 32 * g);
    return tree32(q);
}

/* Canonical sum of products a_i b_i (the terms of Eq. (3.5), (3.12) and the
 * TV relaxation): the order above, with each running lane sum advanced by a
 * fused multiply-add, p = fma(a_i, b_i, p), one rounding per term.  The GPU
 * kernels advance their lane sums the same way. */
static double dot_left_to_right(const double *a, const double *b, int64_t len) {
    double s = 0.0;
    for (int64_t i = 0; i < len; i++) s = fma(a[i], b[i], s);
    return s;
}

double orc_canon_dot(const double *a, const double *b, int64_t len) {
    if (g_plain_sums || len <= 32) return dot_left_to_right(a, b, len);
    if (len <= 512) {
        double p[32];
        for (int j = 0; j < 32; j++) {
            p[j] = 0.0;
            for (int64_t i = j; i < len; i += 32) p[j] = fma(a[i], b[i], p[j]);
        }
        return tree32(p);
    }
    double p[1024], q[32];
    for (int j = 0; j < 1024; j++) {
        p[j] = 0.0;
        for (int64_t i = j; i < len; i += 1024) p[j] = fma(a[i], b[i], p[j]);
    }
    for (int g = 0; g < 32; g++) q[g] = tree32(p + 32 * g);
    return tree32(q);
}

/* Long vectors: chunks of 512 terms, each summed canonically; the chunk sums
 * are summed the same way, recursively. */
double orc_canon_sum_global(const double *t, int64_t len) {
    const int64_t C = 512;
    if (g_plain_sums) return sum_left_to_right(t, len);
    if (len <= C) return orc_canon_sum(t, len);
    int64_t nch = (len + C - 1) / C;
    double *part = (double *)malloc(sizeof(double) * (size_t)nch);
    for (int64_t c = 0; c < nch; c++) {
        int64_t lo = c * C, cnt = len - lo < C ? len - lo : C;
        part[c] = orc_canon_sum(t + lo, cnt);
    }
    double s = orc_canon_sum_global(part, nch);
    free(part);
    return s;
}

/* ------------------------------------------------------------------------- */
/* Input checks and the Laplacian (Eqs. (1.1)-(1.2), (1.3))                    */
/* ------------------------------------------------------------------------- */

static int64_t find_entry(const int64_t *rp, const int32_t *col, int64_t u, int32_t v) {
    int64_t lo = rp[u], hi = rp[u + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (col[mid] == v) return mid;
        if (col[mid] < v) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* The input is the off-diagonal pattern of A as a CSR with both directions of
 * every edge, columns strictly increasing per row, no self loops, w > 0 finite
 * and w_uv == w_vu (Eq. (1.2)); the graph must be connected (Sec. 1).
 * With several graphs (block-diagonal union, nodes of graph g in
 * [gptr[g], gptr[g+1])), no edge may join two graphs (ORC_ERR_ARG) and every
 * graph must be connected (ORC_ERR_DISCONNECTED). */
static int32_t validate_core(int64_t n, const int64_t *rp, const int32_t *col, const double *w, int32_t signed_w) {
    if (n < 1 || rp[0] != 0) return ORC_ERR_ARG;
    for (int64_t u = 0; u < n; u++) {
        if (rp[u + 1] < rp[u]) return ORC_ERR_ARG;
        for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
            if (col[e] < 0 || col[e] >= n || col[e] == u) return ORC_ERR_ARG;
            if (e > rp[u] && col[e] <= col[e - 1]) return ORC_ERR_ARG;
        }
    }
    for (int64_t u = 0; u < n; u++)
        for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
            if (!isfinite(w[e])) return ORC_ERR_BAD_WEIGHT;
            if (signed_w ? !(w[e] != 0.0) : !(w[e] > 0.0)) return ORC_ERR_BAD_WEIGHT;
        }
    /* signed weights (Sec. 5, grids with negative weights): Gauss-Seidel divides by
     * a_uu = sum_v w_uv, so every row with entries needs a positive sum */
    if (signed_w)
        for (int64_t u = 0; u < n; u++)
            if (rp[u + 1] > rp[u] && !(orc_canon_sum(w + rp[u], rp[u + 1] - rp[u]) > 0.0)) return ORC_ERR_BAD_WEIGHT;
    for (int64_t u = 0; u < n; u++)
        for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
            int64_t f = find_entry(rp, col, col[e], (int32_t)u);
            if (f < 0 || w[f] != w[e]) return ORC_ERR_NOT_SYMMETRIC;
        }
    return ORC_OK;
}

/* Connected components by breadth-first search: comp[u] = index of the
 * component in order of its smallest node; returns the count. */
static int32_t components(int64_t n, const int64_t *rp, const int32_t *col, int32_t *comp) {
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    for (int64_t u = 0; u < n; u++) comp[u] = -1;
    int32_t nc = 0;
    for (int64_t s0 = 0; s0 < n; s0++) {
        if (comp[s0] >= 0) continue;
        int64_t head = 0, tail = 0;
        comp[s0] = nc; queue[tail++] = (int32_t)s0;
        while (head < tail) {
            int32_t u = queue[head++];
            for (int64_t e = rp[u]; e < rp[u + 1]; e++)
                if (comp[col[e]] < 0) { comp[col[e]] = nc; queue[tail++] = col[e]; }
        }
        nc++;
    }
    free(queue);
    return nc;
}

static int32_t validate_graphs(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                               int32_t ngraphs, const int64_t *gptr, int32_t signed_w) {
    if (ngraphs < 1 || gptr[0] != 0 || gptr[ngraphs] != n) return ORC_ERR_ARG;
    for (int32_t g = 0; g < ngraphs; g++)
        if (gptr[g + 1] <= gptr[g]) return ORC_ERR_ARG;
    int32_t st = validate_core(n, rp, col, w, signed_w);
    if (st != ORC_OK) return st;
    for (int32_t g = 0; g < ngraphs; g++)
        for (int64_t u = gptr[g]; u < gptr[g + 1]; u++)
            for (int64_t e = rp[u]; e < rp[u + 1]; e++)
                if (col[e] < gptr[g] || col[e] >= gptr[g + 1]) return ORC_ERR_ARG;
    int32_t *comp = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t nc = components(n, rp, col, comp);
    free(comp);
    return nc == ngraphs ? ORC_OK : ORC_ERR_DISCONNECTED;
}

int32_t orc_validate_graphs(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                            int32_t ngraphs, const int64_t *gptr) {
    return validate_graphs(n, rp, col, w, ngraphs, gptr, 0);
}

int32_t orc_validate(int64_t n, const int64_t *rp, const int32_t *col, const double *w) {
    if (n < 1) return ORC_ERR_ARG;
    int64_t gptr[2] = {0, n};
    return orc_validate_graphs(n, rp, col, w, 1, gptr);
}

int32_t orc_validate_signed(int64_t n, const int64_t *rp, const int32_t *col, const double *w) {
    if (n < 1) return ORC_ERR_ARG;
    int64_t gptr[2] = {0, n};
    return validate_graphs(n, rp, col, w, 1, gptr, 1);
}

/* Eq. (1.2): a_uu = sum of incident weights, a_uv = -w_uv. */
void orc_laplacian_dense(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                         double *A) {
    memset(A, 0, sizeof(double) * (size_t)(n * n));
    for (int64_t u = 0; u < n; u++)
        for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
            A[u * n + col[e]] = -w[e];
            A[u * n + u] += w[e];
        }
}

/* a_uu by the canonical order (used wherever the diagonal feeds a setup float). */
static void diag_canon(int64_t n, const int64_t *rp, const double *w, double *diag) {
    for (int64_t u = 0; u < n; u++) diag[u] = orc_canon_sum(w + rp[u], rp[u + 1] - rp[u]);
}

/* ------------------------------------------------------------------------- */
/* Colouring (build reading of the relaxation order; the paper's GS of         */
/* Eq. (2.3) is lexicographic).  Jones-Plassmann, largest degree first: node u */
/* beats v iff (deg u, h u) > (deg v, h v) lexicographically, h = splitmix64(  */
/* key + u), ties to the lower index; each round, every uncoloured node that   */
/* beats all its uncoloured neighbours takes the smallest colour unused by its */
/* neighbours.  Returns the number of colours; *rounds if requested.           */
/* ------------------------------------------------------------------------- */

static int beats(int64_t du, uint64_t pu, int64_t u, int64_t dv, uint64_t pv, int64_t v) {
    if (du != dv) return du > dv;
    return pu > pv || (pu == pv && u < v);
}

static int32_t colour_impl(int64_t n, const int64_t *rp, const int32_t *col, uint64_t key, int32_t hashed,
                           int32_t *colour, int32_t *rounds_out) {
    uint64_t *pri = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    int32_t *sel = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t u = 0; u < n; u++) { pri[u] = hashed ? orc_splitmix64(key + (uint64_t)u) : 0; colour[u] = -1; }
    int64_t left = n; int32_t ncol = 0, rounds = 0;
    int64_t maxdeg = 0;
    for (int64_t u = 0; u < n; u++) if (rp[u + 1] - rp[u] > maxdeg) maxdeg = rp[u + 1] - rp[u];
    uint8_t *used = (uint8_t *)calloc((size_t)maxdeg + 2, 1);
    while (left > 0) {
        int64_t ns = 0;
        for (int64_t u = 0; u < n; u++) {
            if (colour[u] >= 0) continue;
            int is_max = 1;
            for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
                int32_t v = col[e];
                if (colour[v] < 0 && beats(rp[v + 1] - rp[v], pri[v], v, rp[u + 1] - rp[u], pri[u], u)) {
                    is_max = 0;
                    break;
                }
            }
            if (is_max) sel[ns++] = (int32_t)u;
        }
        /* the selected nodes are pairwise non-adjacent, so the order below is immaterial */
        for (int64_t i = 0; i < ns; i++) {
            int32_t u = sel[i];
            int64_t deg = rp[u + 1] - rp[u];
            memset(used, 0, (size_t)deg + 2);
            for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
                int32_t c = colour[col[e]];
                if (c >= 0 && c <= deg) used[c] = 1;
            }
            int32_t c = 0;
            while (used[c]) c++;
            colour[u] = c;
            if (c + 1 > ncol) ncol = c + 1;
        }
        left -= ns; rounds++;
    }
    free(pri); free(sel); free(used);
    if (rounds_out) *rounds_out = rounds;
    return ncol;
}

int32_t orc_colour(int64_t n, const int64_t *rp, const int32_t *col, uint64_t key, int32_t *colour) {
    return colour_impl(n, rp, col, key, 1, colour, NULL);
}

/* ------------------------------------------------------------------------- */
/* Gauss-Seidel, Eq. (2.3): x_u <- (b_u - sum_{v in E_u} a_uv x_v) / a_uu,     */
/* with a_uv = -w_uv.  Lexicographic order and colour order.                   */
/* ------------------------------------------------------------------------- */

static void gs_update(int64_t u, const int64_t *rp, const int32_t *col, const double *w,
                      const double *b, double *x) {
    double s = b[u], d = 0.0;
    if (rp[u + 1] == rp[u]) return;   /* isolated node (a whole graph of a union, coarsened away): unchanged */
    for (int64_t e = rp[u]; e < rp[u + 1]; e++) { s = s + w[e] * x[col[e]]; d = d + w[e]; }
    x[u] = s / d;
}

void orc_gs_sweep_lex(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                      const double *b, double *x) {
    for (int64_t u = 0; u < n; u++) gs_update(u, rp, col, w, b, x);
}

void orc_gs_sweep_colour(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                         const int32_t *colour, int32_t ncolours, const double *b, double *x) {
    for (int32_t c = 0; c < ncolours; c++)
        for (int64_t u = 0; u < n; u++)
            if (colour[u] == c) gs_update(u, rp, col, w, b, x);
}

/* ------------------------------------------------------------------------- */
/* Affinity (Eq. (3.5)) and energy ratio (Eq. (3.12)) per directed entry.     */
/* ------------------------------------------------------------------------- */

/* aff_uv = (X_u,X_v)^2 / ((X_u,X_u)(X_v,X_v)), i.e. 1 - c_uv of Eq. (3.5); the
 * closest neighbour has the LARGEST aff.  (X,Y) summed over k left to right;
 * aff = 0 when the denominator is 0.
 *
 * q_uv: the paper's Eq. (3.12) prints min_y E / E(x_s), which never exceeds 1
 * and would make the "q <= 2.5" test vacuous; the text describes the energy
 * after aggregation over the energy after a local relaxation, so this build
 * reads q_us = max_k E_u(x^k; x^k_s) / min_y E_u(x^k; y).  With
 * y*_k = B_u^k / a_uu and the identity E_u(x; y) = Emin + a_uu (y - y*)^2 / 2:
 *   Emin_k = 1/2 sum_v w_uv (y*_k - x^k_v)^2     (canonical row sum)
 *   E_s,k  = Emin_k + (a_uu / 2) (x^k_s - y*_k)^2
 *   ratio_k = E_s,k / Emin_k  (Emin_k == 0: 1 if E_s,k == 0 else +inf).
 * Strong entry: |w_uv| >= weak_tol * max(max_t |w_ut|, max_t |w_vt|)  (reading
 * of the weak-edge filter of Sec. 3.4.2).
 * score = aff if strong and q <= q_max, else -1 (never a candidate). */
void orc_edge_scores(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                     int32_t K, const double *X, double q_max, double weak_tol,
                     double *aff, double *q, double *score) {
    double *diag = (double *)malloc(sizeof(double) * (size_t)n);
    double *XX = (double *)malloc(sizeof(double) * (size_t)n);
    double *maxw = (double *)malloc(sizeof(double) * (size_t)n);
    double *ystar = (double *)malloc(sizeof(double) * (size_t)(n * K));
    double *emin = (double *)malloc(sizeof(double) * (size_t)(n * K));
    int64_t maxdeg = 0;
    for (int64_t u = 0; u < n; u++) if (rp[u + 1] - rp[u] > maxdeg) maxdeg = rp[u + 1] - rp[u];
    double *t = (double *)malloc(sizeof(double) * (size_t)(maxdeg + 1));
    double *aw = (double *)malloc(sizeof(double) * (size_t)(maxdeg + 1));
    /* the nodal energies use |w_uv| (reading R22): identical for positive weights,
     * and with negative weights min_y E_u stays non-negative, so the ratio keeps
     * its meaning of an energy inflation */
    for (int64_t u = 0; u < n; u++) {
        for (int64_t e = rp[u]; e < rp[u + 1]; e++) t[e - rp[u]] = fabs(w[e]);
        diag[u] = orc_canon_sum(t, rp[u + 1] - rp[u]);
    }
    for (int64_t u = 0; u < n; u++) {
        double s = 0.0;
        for (int k = 0; k < K; k++) s = fma(X[u * K + k], X[u * K + k], s);
        XX[u] = s;
        double m = 0.0;
        for (int64_t e = rp[u]; e < rp[u + 1]; e++) if (fabs(w[e]) > m) m = fabs(w[e]);
        maxw[u] = m;
        int64_t deg = rp[u + 1] - rp[u];
        for (int64_t e = rp[u]; e < rp[u + 1]; e++) aw[e - rp[u]] = fabs(w[e]);
        for (int k = 0; k < K; k++) {
            for (int64_t e = rp[u]; e < rp[u + 1]; e++) t[e - rp[u]] = X[(int64_t)col[e] * K + k];
            double B = orc_canon_dot(aw, t, deg);
            double y = B / diag[u];
            for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
                double d = y - X[(int64_t)col[e] * K + k];
                t[e - rp[u]] = d * d;
            }
            ystar[u * K + k] = y;
            emin[u * K + k] = 0.5 * orc_canon_dot(aw, t, deg);
        }
    }
    for (int64_t u = 0; u < n; u++) {
        double half_a = 0.5 * diag[u];
        for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
            int64_t v = col[e];
            double dot = 0.0;
            for (int k = 0; k < K; k++) dot = fma(X[u * K + k], X[v * K + k], dot);
            double num = dot * dot, den = XX[u] * XX[v];
            double a = den > 0.0 ? num / den : 0.0;
            double qq = 0.0;
            for (int k = 0; k < K; k++) {
                double d = X[v * K + k] - ystar[u * K + k];
                double em = emin[u * K + k];
                double es = em + half_a * (d * d);
                double r = em > 0.0 ? es / em : (es == 0.0 ? 1.0 : INFINITY);
                if (r > qq) qq = r;
            }
            double mw = maxw[u] > maxw[v] ? maxw[u] : maxw[v];
            int strong = fabs(w[e]) >= weak_tol * mw;
            if (aff) aff[e] = a;
            if (q) q[e] = qq;
            if (score) score[e] = (strong && qq <= q_max) ? a : -1.0;
        }
    }
    free(diag); free(XX); free(maxw); free(ystar); free(emin); free(t); free(aw);
}

/* Hub test, Sec. 3.4.1 footnote: |E_u| >= 8 sum_v |w_uv||E_v| / sum_v |w_uv|,
 * compared cross-multiplied: |E_u| * sum|w| >= 8 * sum |w_uv| |E_v|. */
void orc_hubs(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
              double hub_factor, uint8_t *hub) {
    int64_t maxdeg = 0;
    for (int64_t u = 0; u < n; u++) if (rp[u + 1] - rp[u] > maxdeg) maxdeg = rp[u + 1] - rp[u];
    double *t1 = (double *)malloc(sizeof(double) * (size_t)(maxdeg + 1));
    double *t2 = (double *)malloc(sizeof(double) * (size_t)(maxdeg + 1));
    for (int64_t u = 0; u < n; u++) {
        int64_t deg = rp[u + 1] - rp[u];
        for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
            int64_t v = col[e];
            t1[e - rp[u]] = fabs(w[e]);
            t2[e - rp[u]] = fabs(w[e]) * (double)(rp[v + 1] - rp[v]);
        }
        double lhs = (double)deg * orc_canon_sum(t1, deg);
        double rhs = hub_factor * orc_canon_sum(t2, deg);
        hub[u] = (deg > 0 && lhs >= rhs) ? 1 : 0;
    }
    free(t1); free(t2);
}

/* ------------------------------------------------------------------------- */
/* Dense solves: the coarsest level (Sec. 4.2, "direct solver on an augmented  */
/* system").  For a connected Laplacian, A + (1/n) 1 1^T is SPD and its        */
/* inverse maps a zero-sum b to the zero-mean solution of A x = b.             */
/* ------------------------------------------------------------------------- */

static int chol_factor(int64_t n, double *M) {   /* in place, lower triangle */
    for (int64_t j = 0; j < n; j++) {
        double s = M[j * n + j];
        for (int64_t k = 0; k < j; k++) s -= M[j * n + k] * M[j * n + k];
        if (!(s > 0.0)) return 1;
        double d = sqrt(s);
        M[j * n + j] = d;
        for (int64_t i = j + 1; i < n; i++) {
            double t = M[i * n + j];
            for (int64_t k = 0; k < j; k++) t -= M[i * n + k] * M[j * n + k];
            M[i * n + j] = t / d;
        }
    }
    return 0;
}

static void chol_solve(int64_t n, const double *L, const double *b, double *x) {
    for (int64_t i = 0; i < n; i++) {
        double t = b[i];
        for (int64_t k = 0; k < i; k++) t -= L[i * n + k] * x[k];
        x[i] = t / L[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; i--) {
        double t = x[i];
        for (int64_t k = i + 1; k < n; k++) t -= L[k * n + i] * x[k];
        x[i] = t / L[i * n + i];
    }
}

static void subtract_mean(int64_t n, double *x) {
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += x[i];
    double m = s / (double)n;
    for (int64_t i = 0; i < n; i++) x[i] -= m;
}

/* Mean subtraction on each component separately (comp[u] in [0, ncomp)):
 * the sums run over the nodes in index order, as subtract_mean does. */
static void subtract_mean_comp(int64_t n, double *x, const int32_t *comp, int32_t ncomp) {
    if (ncomp <= 1) { subtract_mean(n, x); return; }
    double *s = (double *)calloc((size_t)ncomp, sizeof(double));
    int64_t *c = (int64_t *)calloc((size_t)ncomp, sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) { s[comp[i]] += x[i]; c[comp[i]]++; }
    for (int32_t k = 0; k < ncomp; k++) s[k] /= (double)c[k];
    for (int64_t i = 0; i < n; i++) x[i] -= s[comp[i]];
    free(s); free(c);
}

/* Mean subtraction on each graph's contiguous node range. */
static void subtract_mean_ranges(double *x, int32_t ngraphs, const int64_t *gptr) {
    for (int32_t g = 0; g < ngraphs; g++) subtract_mean(gptr[g + 1] - gptr[g], x + gptr[g]);
}

int32_t orc_dense_pinv_solve(int64_t n, const double *A, const double *b, double *x) {
    double *M = (double *)malloc(sizeof(double) * (size_t)(n * n));
    for (int64_t i = 0; i < n * n; i++) M[i] = A[i] + 1.0 / (double)n;
    int bad = chol_factor(n, M);
    if (!bad) { chol_solve(n, M, b, x); subtract_mean(n, x); }
    free(M);
    return bad ? ORC_ERR_ARG : ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Hierarchy                                                                   */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t n, nnz;
    int64_t *rp; int32_t *col; double *w;
    double *diag;
    int32_t *colour; int32_t ncolours, jp_rounds;
    int32_t coarsest, stop_reason;   /* 1 small, 2 relaxation fast, 3 stall, 4 depth */
    int32_t K;
    double *X, *aff, *q, *score;
    uint8_t *hub;
    int32_t *state, *agg;
    int64_t nc;
    double alpha, gamma_l, tv_ratio;
    int32_t rounds, sel_round;
    double *chol;                     /* coarsest dense factor, if direct */
    int32_t *comp; int32_t ncomp;     /* coarsest: connected components */
    int32_t elim;                     /* 1: the next level is this level's Schur complement */
    int64_t nF;                       /* eliminated nodes */
    int32_t *cidx;                    /* coarse index of each C node, -1 for F nodes */
} orc_level;

struct orc_hier {
    orc_opts o;
    int32_t L;
    int32_t ngraphs;                  /* graphs of the block-diagonal union */
    int64_t *gptr;                    /* level-1 node ranges of the graphs */
    orc_level lv[128];
};

enum { ST_U = 0, ST_S = 1, ST_A = 2, ST_D = 3 };

static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s); }

/* TV relaxation, Sec. 3.3.1 and Sec. 4.1: K vectors from random[-1,1], nu GS
 * sweeps on A x = 0 in colour order, each update x_u = (sum_v w_uv x_v) / a_uu
 * with the canonical row sum.  Also returns the largest per-TV energy ratio of
 * the last sweep, E(nu) / E(nu-1), E = sum_u E_u (Eq. (3.11a)). */
static double relax_tvs(orc_level *L, const orc_opts *o, int32_t level) {
    int64_t n = L->n; int32_t K = L->K;
    uint64_t key = tv_key(o->seed, level);
    for (int64_t u = 0; u < n; u++)
        for (int k = 0; k < K; k++)
            L->X[u * K + k] = tv_uniform(orc_splitmix64(key + (uint64_t)(u * K + k)));
    int64_t maxdeg = 0;
    for (int64_t u = 0; u < n; u++) if (L->rp[u + 1] - L->rp[u] > maxdeg) maxdeg = L->rp[u + 1] - L->rp[u];
    double *t = (double *)malloc(sizeof(double) * (size_t)(maxdeg + 1));
    double *eu = (double *)malloc(sizeof(double) * (size_t)n);
    double eprev[16], ecur[16];
    double worst = 0.0;
    for (int sw = 1; sw <= o->nu_tv; sw++) {
        for (int32_t c = 0; c < L->ncolours; c++)
            for (int64_t u = 0; u < n; u++) {
                if (L->colour[u] != c) continue;
                int64_t deg = L->rp[u + 1] - L->rp[u];
                if (deg == 0) continue;   /* isolated node: its TVs keep their random values */
                for (int k = 0; k < K; k++) {
                    for (int64_t e = L->rp[u]; e < L->rp[u + 1]; e++)
                        t[e - L->rp[u]] = L->X[(int64_t)L->col[e] * K + k];
                    L->X[u * K + k] = orc_canon_dot(L->w + L->rp[u], t, deg) / L->diag[u];
                }
            }
        if (o->relax_fast_ratio > 0.0 && sw >= o->nu_tv - 1) {
            for (int k = 0; k < K; k++) {
                for (int64_t u = 0; u < n; u++) {
                    int64_t deg = L->rp[u + 1] - L->rp[u];
                    for (int64_t e = L->rp[u]; e < L->rp[u + 1]; e++) {
                        double d = L->X[u * K + k] - L->X[(int64_t)L->col[e] * K + k];
                        t[e - L->rp[u]] = d * d;
                    }
                    eu[u] = 0.5 * orc_canon_dot(L->w + L->rp[u], t, deg);
                }
                double E = orc_canon_sum_global(eu, n);
                if (sw == o->nu_tv - 1) eprev[k] = E; else ecur[k] = E;
            }
        }
    }
    if (o->relax_fast_ratio > 0.0 && o->nu_tv >= 2) {
        for (int k = 0; k < K; k++) {
            double r = eprev[k] > 0.0 ? ecur[k] / eprev[k] : 0.0;
            if (r > worst) worst = r;
        }
    } else {
        worst = INFINITY;
    }
    free(t); free(eu);
    return worst;
}

/* Aggregation, Sec. 3.4.1-3.4.2, build reading (the complete algorithm is in an
 * e-print that is not available).  States U(ndecided)/S(eed)/A(ssociate)/
 * D(ummy).  Start: nodes without strong entries -> D; hubs -> S; rest -> U.
 *
 * agg_rule 2 (default) and 1: the paper's scan.  Each stage visits the U nodes
 * one at a time, in decreasing priority splitmix64(key_l + u) (ties to the lower
 * index; rule 2) or in increasing index (rule 1); each decides on the states left
 * by the nodes before it.  u joins the admissible neighbour v (score >= 0, not A
 * or D) with the largest score, ties to the lower index (the smallest c_uv among
 * those with q_uv <= 2.5, Sec. 3.4.5); an undecided v thereby becomes a seed.
 * At most two stages are run, as in the paper.
 *
 * agg_rule 0: the parallel handshake.  Each round (one stage), from the
 * start-of-round state only:
 *   best(u), u in U: the entry with the largest score >= 0 whose neighbour is
 *     not A (ties -> lower neighbour index), or none.
 *   best(u) = v in S                 -> u becomes A with seed v;
 *   best(u) = v in U, best(v) = u    -> min(u,v) becomes S, the other A of it;
 *   otherwise u stays U.
 *
 * After stage r, alpha_r = (#S + #U + [#D > 0]) / n (left-over U become seeds).
 * Stages stop when alpha_r <= alpha_max = 0.7/gamma, when a stage changes
 * nothing, or after the stage limit.  The stage whose alpha_r is closest to
 * alpha_max is selected (ties -> earlier).  Numbering: seeds by ascending node
 * index, the dummy aggregate last. */
typedef struct { uint64_t p; int64_t u; } scan_prio;

static int scan_prio_cmp(const void *a, const void *b) {
    const scan_prio *x = (const scan_prio *)a, *y = (const scan_prio *)b;
    if (x->p != y->p) return x->p > y->p ? -1 : 1;
    return x->u < y->u ? -1 : (x->u > y->u);
}

static void aggregate(orc_level *L, const orc_opts *o, uint64_t key) {
    int64_t n = L->n;
    int32_t *state = L->state;
    int32_t *seed = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *best = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *nstate = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *nseed = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *bstate = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *bseed = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *maxw = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t u = 0; u < n; u++) {
        double m = 0.0;
        for (int64_t e = L->rp[u]; e < L->rp[u + 1]; e++) if (fabs(L->w[e]) > m) m = fabs(L->w[e]);
        maxw[u] = m;
    }
    int64_t nd = 0;
    for (int64_t u = 0; u < n; u++) {
        int has_strong = 0;
        for (int64_t e = L->rp[u]; e < L->rp[u + 1]; e++) {
            int64_t v = L->col[e];
            double mw = maxw[u] > maxw[v] ? maxw[u] : maxw[v];
            if (fabs(L->w[e]) >= o->weak_tol * mw) { has_strong = 1; break; }
        }
        seed[u] = -1;
        if (!has_strong) { state[u] = ST_D; nd++; }
        else state[u] = L->hub[u] ? ST_S : ST_U;
    }
    double amax = 0.7 / o->gamma;
    double best_alpha = INFINITY; int32_t best_round = 0, r;
    const int32_t max_stages = o->agg_rule >= 1 ? (o->max_rounds < 2 ? o->max_rounds : 2) : o->max_rounds;
    int64_t *order = NULL;
    if (o->agg_rule >= 1) {
        order = (int64_t *)xcalloc((size_t)n, sizeof(int64_t));
        if (o->agg_rule == 2) {
            scan_prio *sp = (scan_prio *)xcalloc((size_t)n, sizeof(scan_prio));
            for (int64_t u = 0; u < n; u++) { sp[u].p = orc_splitmix64(key + (uint64_t)u); sp[u].u = u; }
            qsort(sp, (size_t)n, sizeof(scan_prio), scan_prio_cmp);
            for (int64_t i = 0; i < n; i++) order[i] = sp[i].u;
            free(sp);
        } else {
            for (int64_t i = 0; i < n; i++) order[i] = i;
        }
    }
    for (r = 1; r <= max_stages; r++) {
        int changed = 0;
        if (o->agg_rule >= 1) {
            for (int64_t i = 0; i < n; i++) {
                const int64_t u = order[i];
                if (state[u] != ST_U) continue;
                int32_t bv = -1;
                double bs = -1.0;
                for (int64_t e = L->rp[u]; e < L->rp[u + 1]; e++) {
                    int32_t v = L->col[e];
                    double s = L->score[e];
                    if (s < 0.0 || state[v] == ST_A || state[v] == ST_D) continue;
                    if (s > bs || (s == bs && v < bv)) { bs = s; bv = v; }
                }
                if (bv < 0) continue;
                if (state[bv] == ST_U) state[bv] = ST_S;
                state[u] = ST_A;
                seed[u] = bv;
                changed = 1;
            }
        } else {
            for (int64_t u = 0; u < n; u++) {
                best[u] = -1;
                if (state[u] != ST_U) continue;
                double bs = -1.0;
                for (int64_t e = L->rp[u]; e < L->rp[u + 1]; e++) {
                    int32_t v = L->col[e];
                    double s = L->score[e];
                    if (s < 0.0 || state[v] == ST_A) continue;
                    if (s > bs || (s == bs && best[u] >= 0 && v < best[u])) { bs = s; best[u] = v; }
                }
            }
            memcpy(nstate, state, sizeof(int32_t) * (size_t)n);
            memcpy(nseed, seed, sizeof(int32_t) * (size_t)n);
            for (int64_t u = 0; u < n; u++) {
                if (state[u] != ST_U || best[u] < 0) continue;
                int32_t v = best[u];
                if (state[v] == ST_S) { nstate[u] = ST_A; nseed[u] = v; changed = 1; }
                else if (state[v] == ST_U && best[v] == (int32_t)u) {
                    int32_t lo = (int32_t)u < v ? (int32_t)u : v, hi = (int32_t)u < v ? v : (int32_t)u;
                    nstate[lo] = ST_S; nstate[hi] = ST_A; nseed[hi] = lo; changed = 1;
                }
            }
            memcpy(state, nstate, sizeof(int32_t) * (size_t)n);
            memcpy(seed, nseed, sizeof(int32_t) * (size_t)n);
        }
        int64_t nc = (nd > 0 ? 1 : 0);
        for (int64_t u = 0; u < n; u++) if (state[u] == ST_S || state[u] == ST_U) nc++;
        double alpha = (double)nc / (double)n;
        if (fabs(alpha - amax) < fabs(best_alpha - amax)) {
            best_alpha = alpha; best_round = r;
            memcpy(bstate, state, sizeof(int32_t) * (size_t)n);
            memcpy(bseed, seed, sizeof(int32_t) * (size_t)n);
        }
        if (alpha <= amax || !changed) break;
    }
    free(order);
    L->rounds = r > max_stages ? max_stages : r;
    L->sel_round = best_round;
    L->alpha = best_alpha;
    memcpy(state, bstate, sizeof(int32_t) * (size_t)n);
    int64_t nc = 0;
    for (int64_t u = 0; u < n; u++)
        if (state[u] == ST_S || state[u] == ST_U) L->agg[u] = (int32_t)nc++;
    for (int64_t u = 0; u < n; u++) {
        if (state[u] == ST_A) L->agg[u] = L->agg[bseed[u]];
        else if (state[u] == ST_D) L->agg[u] = (int32_t)nc;
    }
    L->nc = nc + (nd > 0 ? 1 : 0);
    free(seed); free(best); free(nstate); free(nseed); free(bstate); free(bseed); free(maxw);
}

/* Galerkin coarse operator, Eq. (2.5) with caliber-1 P (p_uU = 1 iff u in T_U):
 * W^c_UV = sum of w_uv over fine edges between T_U and T_V (U != V), and the
 * coarse Laplacian follows from Eq. (1.2).  Summation order (build reading):
 * for U < V the fine entries (u -> v), u in T_U, v in T_V, in increasing
 * (u, v), summed canonically; W^c_VU is the same number. */
typedef struct { int32_t U, V; int64_t pos; double w; } gal_entry;

static int gal_cmp(const void *a, const void *b) {
    const gal_entry *x = (const gal_entry *)a, *y = (const gal_entry *)b;
    if (x->U != y->U) return x->U < y->U ? -1 : 1;
    if (x->V != y->V) return x->V < y->V ? -1 : 1;
    if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;
    return 0;
}

static void galerkin(const orc_level *F, orc_level *C) {
    int64_t cnt = 0;
    for (int64_t u = 0; u < F->n; u++)
        for (int64_t e = F->rp[u]; e < F->rp[u + 1]; e++)
            if (F->agg[u] < F->agg[F->col[e]]) cnt++;
    gal_entry *E = (gal_entry *)xcalloc((size_t)cnt, sizeof(gal_entry));
    int64_t k = 0;
    for (int64_t u = 0; u < F->n; u++)
        for (int64_t e = F->rp[u]; e < F->rp[u + 1]; e++)
            if (F->agg[u] < F->agg[F->col[e]]) {
                E[k].U = F->agg[u]; E[k].V = F->agg[F->col[e]]; E[k].pos = e; E[k].w = F->w[e]; k++;
            }
    qsort(E, (size_t)cnt, sizeof(gal_entry), gal_cmp);
    /* unique pairs with canonical sums, then both directions into a sorted CSR */
    gal_entry *D = (gal_entry *)xcalloc((size_t)(2 * cnt), sizeof(gal_entry));
    double *t = (double *)xcalloc((size_t)cnt, sizeof(double));
    int64_t nd = 0;
    for (int64_t i = 0; i < cnt;) {
        int64_t j = i;
        while (j < cnt && E[j].U == E[i].U && E[j].V == E[i].V) { t[j - i] = E[j].w; j++; }
        double W = orc_canon_sum(t, j - i);
        D[nd].U = E[i].U; D[nd].V = E[i].V; D[nd].pos = 0; D[nd].w = W; nd++;
        D[nd].U = E[i].V; D[nd].V = E[i].U; D[nd].pos = 0; D[nd].w = W; nd++;
        i = j;
    }
    qsort(D, (size_t)nd, sizeof(gal_entry), gal_cmp);
    C->n = F->nc;
    C->nnz = nd;
    C->rp = (int64_t *)xcalloc((size_t)(C->n + 1), sizeof(int64_t));
    C->col = (int32_t *)xcalloc((size_t)nd, sizeof(int32_t));
    C->w = (double *)xcalloc((size_t)nd, sizeof(double));
    for (int64_t i = 0; i < nd; i++) { C->rp[D[i].U + 1]++; C->col[i] = D[i].V; C->w[i] = D[i].w; }
    for (int64_t u = 0; u < C->n; u++) C->rp[u + 1] += C->rp[u];
    free(E); free(D); free(t);
}

/* The aggregation of one level from its CSR, its edge scores and hub flags
 * (Sec. 3.4.1-3.4.2 with readings R9-R11), as the setup runs it.
 * info[0..3] = nc, rounds, selected round, alpha (double bits). */
void orc_aggregate(int64_t n, const int64_t *rp, const int32_t *col, const double *w, const double *score,
                   const uint8_t *hub, const orc_opts *o, int32_t level, int32_t *agg, int32_t *state,
                   int64_t *info) {
    orc_level L;
    memset(&L, 0, sizeof(L));
    L.n = n; L.nnz = rp[n];
    L.rp = (int64_t *)rp; L.col = (int32_t *)col; L.w = (double *)w;
    L.score = (double *)score; L.hub = (uint8_t *)hub;
    L.agg = agg; L.state = state;
    aggregate(&L, o, agg_key(o->seed, level));
    info[0] = L.nc; info[1] = L.rounds; info[2] = L.sel_round;
    memcpy(&info[3], &L.alpha, sizeof(double));
}

/* The Galerkin operator of one level (Eq. (2.5), reading R12) from its CSR and
 * aggregates 0..nc-1.  The caller sizes rp_c as nc + 1 and col_c, w_c as the
 * fine nnz (a bound on the coarse nnz).  Returns the coarse nnz. */
int64_t orc_galerkin(int64_t n, const int64_t *rp, const int32_t *col, const double *w, const int32_t *agg,
                     int64_t nc, int64_t *rp_c, int32_t *col_c, double *w_c) {
    orc_level F, C;
    memset(&F, 0, sizeof(F));
    memset(&C, 0, sizeof(C));
    F.n = n; F.nnz = rp[n];
    F.rp = (int64_t *)rp; F.col = (int32_t *)col; F.w = (double *)w;
    F.agg = (int32_t *)agg; F.nc = nc;
    galerkin(&F, &C);
    memcpy(rp_c, C.rp, sizeof(int64_t) * (size_t)(nc + 1));
    memcpy(col_c, C.col, sizeof(int32_t) * (size_t)C.nnz);
    memcpy(w_c, C.w, sizeof(double) * (size_t)C.nnz);
    int64_t nnz = C.nnz;
    free(C.rp); free(C.col); free(C.w);
    return nnz;
}

/* Low-degree elimination, Sec. 3.2.  F is an independent set of nodes of
 * degree 1..4 (unweighted, |E_u|), taken by one sweep through the nodes: an
 * eligible node joins F and its neighbours become ineligible.  The paper does
 * not fix the sweep order; this build sweeps by decreasing priority
 * splitmix64(elim_key + u), ties to the lower index, so that the same set can
 * be found in parallel rounds of small depth (each candidate waits only for
 * its higher-priority candidate neighbours).  Degree 0 is left out: an
 * isolated node has a_uu = 0.  C = N \ F keeps the fine order: cidx[u] = rank
 * of u among the C nodes, -1 for u in F.  Returns |F|. */
typedef struct { uint64_t p; int64_t u; } elim_prio;

static int elim_prio_cmp(const void *a, const void *b) {
    const elim_prio *x = (const elim_prio *)a, *y = (const elim_prio *)b;
    if (x->p != y->p) return x->p > y->p ? -1 : 1;
    return x->u < y->u ? -1 : (x->u > y->u);
}

static int64_t elim_select(const orc_level *L, uint64_t key, int32_t *cidx) {
    int64_t n = L->n, nF = 0, nc = 0;
    uint8_t *inel = (uint8_t *)xcalloc((size_t)n, 1);
    elim_prio *ord = (elim_prio *)xcalloc((size_t)n, sizeof(elim_prio));
    for (int64_t u = 0; u < n; u++) { ord[u].p = orc_splitmix64(key + (uint64_t)u); ord[u].u = u; cidx[u] = 0; }
    qsort(ord, (size_t)n, sizeof(elim_prio), elim_prio_cmp);
    for (int64_t i = 0; i < n; i++) {
        int64_t u = ord[i].u;
        int64_t deg = L->rp[u + 1] - L->rp[u];
        if (inel[u] || deg < 1 || deg > 4) continue;
        cidx[u] = -1;
        nF++;
        for (int64_t e = L->rp[u]; e < L->rp[u + 1]; e++) inel[L->col[e]] = 1;
    }
    for (int64_t u = 0; u < n; u++) if (cidx[u] != -1) cidx[u] = (int32_t)nc++;
    free(inel); free(ord);
    return nF;
}

int64_t orc_elim_set(int64_t n, const int64_t *rp, const int32_t *col, uint64_t key, int32_t *cidx) {
    orc_level L;
    memset(&L, 0, sizeof(L));
    L.n = n;
    L.rp = (int64_t *)rp;
    L.col = (int32_t *)col;
    return elim_select(&L, key, cidx);
}

typedef struct { int32_t col; int64_t key; double v; } elim_term;

static int elim_cmp(const void *a, const void *b) {
    const elim_term *x = (const elim_term *)a, *y = (const elim_term *)b;
    if (x->col != y->col) return x->col < y->col ? -1 : 1;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return 0;
}

/* Schur complement of F, Eq. (3.1): A^c = A_CC - A_CF A_FF^-1 A_FC, again a
 * graph Laplacian.  A_FF is diagonal (F independent), so the coarse weight of
 * c1 != c2 is W^c = w_{c1 c2} + sum over f in F adjacent to both of
 * (w_{f c1} w_{f c2}) / a_ff.  Summation order (build reading): the direct
 * edge first, then the fill terms by increasing f, summed canonically; the
 * product is commutative, so W^c is bit-symmetric.  Coarse rows and columns
 * follow cidx; the diagonal is the row sum (Eq. (1.2)). */
static void eliminate(const orc_level *F, const int32_t *cidx, orc_level *C) {
    int64_t n = F->n, nc = 0, maxt = 0;
    for (int64_t u = 0; u < n; u++) if (cidx[u] >= 0) nc++;
    C->n = nc;
    C->rp = (int64_t *)xcalloc((size_t)(nc + 1), sizeof(int64_t));
    /* terms of each coarse row: first count them */
    int64_t *cnt = (int64_t *)xcalloc((size_t)(nc + 1), sizeof(int64_t));
    for (int64_t u = 0; u < n; u++) {
        if (cidx[u] < 0) continue;
        int64_t t = 0;
        for (int64_t e = F->rp[u]; e < F->rp[u + 1]; e++) {
            int32_t v = F->col[e];
            t += cidx[v] >= 0 ? 1 : (F->rp[v + 1] - F->rp[v] - 1);
        }
        cnt[cidx[u]] = t;
        if (t > maxt) maxt = t;
    }
    elim_term *T = (elim_term *)xcalloc((size_t)maxt, sizeof(elim_term));
    double *t = (double *)xcalloc((size_t)maxt, sizeof(double));
    /* two passes over the rows: sizes, then entries */
    int64_t cap = 0;
    for (int64_t U = 0; U < nc; U++) cap += cnt[U];
    C->col = (int32_t *)xcalloc((size_t)cap, sizeof(int32_t));
    C->w = (double *)xcalloc((size_t)cap, sizeof(double));
    int64_t nnz = 0;
    for (int64_t u = 0; u < n; u++) {
        if (cidx[u] < 0) continue;
        int64_t k = 0;
        for (int64_t e = F->rp[u]; e < F->rp[u + 1]; e++) {
            int32_t v = F->col[e];
            if (cidx[v] >= 0) {
                T[k].col = cidx[v]; T[k].key = -1; T[k].v = F->w[e]; k++;
                continue;
            }
            for (int64_t e2 = F->rp[v]; e2 < F->rp[v + 1]; e2++) {
                int32_t c2 = F->col[e2];
                if (c2 == (int32_t)u) continue;
                T[k].col = cidx[c2]; T[k].key = v; T[k].v = (F->w[e] * F->w[e2]) / F->diag[v]; k++;
            }
        }
        qsort(T, (size_t)k, sizeof(elim_term), elim_cmp);
        for (int64_t i = 0; i < k;) {
            int64_t j = i;
            while (j < k && T[j].col == T[i].col) { t[j - i] = T[j].v; j++; }
            C->col[nnz] = T[i].col;
            C->w[nnz] = orc_canon_sum(t, j - i);
            nnz++;
            i = j;
        }
        C->rp[cidx[u] + 1] = nnz;
    }
    C->nnz = nnz;
    free(cnt); free(T); free(t);
}

/* Cycle index per level, Eq. (4.1).  As printed, the second branch
 * min{2, .7|E^{l+1}|/|E^l|} is below 0.7 < 1 whenever the coarse level has
 * fewer edges; the text says gamma^l is raised at coarse levels at a bounded
 * work increase, so this build reads the ratio inverted,
 * g = .7 |E^l| / |E^{l+1}| (coarse work per fine visit stays at .7), and
 * applies the same bound at the fine levels, where the cap is gamma instead
 * of 2:  gamma^l = min{cap, max{1, g}}, cap = gamma if |E^l| > .1|E| else
 * gamma_coarse_max (2, as printed).
 * (With the printed fine-level rule gamma^l = gamma, a level that coarsens
 * slowly, alpha ~ .85, makes the work per cycle grow without bound.) */
static void cycle_indices(orc_hier *h) {
    double m1 = (double)h->lv[0].nnz / 2.0;
    for (int32_t l = 0; l < h->L - 1; l++) {
        if (h->lv[l].elim) { h->lv[l].gamma_l = 1.0; continue; }   /* Sec. 4.2: gamma = 1 before elimination */
        if (h->o.lgmg_nx > 0) { h->lv[l].gamma_l = h->o.gamma; continue; }   /* Sec. 6: a standard gamma-cycle */
        double ml = (double)h->lv[l].nnz / 2.0, mn = (double)h->lv[l + 1].nnz / 2.0;
        double g = mn > 0.0 ? 0.7 * ml / mn : 2.0;
        double gmax = ml > 0.1 * m1 ? h->o.gamma : h->o.gamma_coarse_max;
        if (g > gmax) g = gmax;
        if (g < 1.0) g = 1.0;
        if (h->o.gamma_fine_printed && ml > 0.1 * m1) g = h->o.gamma;   /* Eq. (4.1) as printed */
        h->lv[l].gamma_l = g;
    }
    h->lv[h->L - 1].gamma_l = 0.0;
}

/* Lean Geometric Multigrid (Sec. 6): red-black colours of an nx x nx torus */
static void level_colour_rb(orc_level *L, int32_t nx) {
    L->colour = (int32_t *)xcalloc((size_t)L->n, sizeof(int32_t));
    for (int64_t u = 0; u < L->n; u++) L->colour[u] = (int32_t)(((u % nx) + (u / nx)) & 1);
    L->ncolours = 2;
    L->jp_rounds = 0;
}

static void level_diag(orc_level *L) {
    L->diag = (double *)xcalloc((size_t)L->n, sizeof(double));
    diag_canon(L->n, L->rp, L->w, L->diag);
}

/* The JP colouring of a level that relaxes.  A level followed by elimination
 * never relaxes (Sec. 4.2: nu = 0 there), so it gets one colour, 0, instead. */
/* Lexicographic Gauss-Seidel (Eq. (2.3)) as a colour-ordered sweep: colour[u] =
 * 1 + the largest colour of a lower-index neighbour (0 if none), the level sets of
 * the lower-triangular dependency graph.  Neighbours never share a colour, every
 * lower-index neighbour of u has a smaller colour and every higher-index one a
 * larger colour, so sweeping the colours in order updates each node from the new
 * values of its lower-index neighbours and the old values of the others: the
 * lexicographic sweep exactly.  Returns the number of colours. */
int32_t orc_colour_lex(int64_t n, const int64_t *rp, const int32_t *col, int32_t *colour) {
    int32_t nc = 0;
    for (int64_t u = 0; u < n; u++) {
        int32_t c = 0;
        for (int64_t e = rp[u]; e < rp[u + 1]; e++)
            if (col[e] < u && colour[col[e]] + 1 > c) c = colour[col[e]] + 1;
        colour[u] = c;
        if (c + 1 > nc) nc = c + 1;
    }
    return nc;
}

static void level_colour(orc_level *L, uint64_t seed, int32_t level, int relaxes, int32_t relax_rule,
                         int32_t colour_rule) {
    L->colour = (int32_t *)xcalloc((size_t)L->n, sizeof(int32_t));
    if (relaxes && relax_rule == 1) {
        L->ncolours = orc_colour_lex(L->n, L->rp, L->col, L->colour);
        L->jp_rounds = 0;
    } else if (relaxes) {
        L->ncolours = colour_impl(L->n, L->rp, L->col, colour_key(seed, level), colour_rule == 0, L->colour,
                                  &L->jp_rounds);
    } else {
        L->ncolours = 1;
        L->jp_rounds = 0;
    }
}

/* Coarsest level: the direct solve uses (A + sum_K 1_K 1_K^T / n_K)^-1 over the
 * connected components K of the level (one component for a connected input),
 * which maps a right-hand side that is zero-sum on every component to the
 * solution with zero mean on every component. */
static int make_coarsest(orc_level *L, const orc_opts *o) {
    L->coarsest = 1;
    int64_t n = L->n;
    L->comp = (int32_t *)xcalloc((size_t)n, sizeof(int32_t));
    L->ncomp = components(n, L->rp, L->col, L->comp);
    if (n <= o->dense_max) {
        int64_t *size = (int64_t *)calloc((size_t)L->ncomp, sizeof(int64_t));
        for (int64_t i = 0; i < n; i++) size[L->comp[i]]++;
        L->chol = (double *)xcalloc((size_t)(n * n), sizeof(double));
        orc_laplacian_dense(n, L->rp, L->col, L->w, L->chol);
        for (int64_t i = 0; i < n; i++)
            for (int64_t j = 0; j < n; j++)
                if (L->comp[i] == L->comp[j]) L->chol[i * n + j] += 1.0 / (double)size[L->comp[i]];
        free(size);
        if (chol_factor(n, L->chol)) return ORC_ERR_ARG;
    }
    return ORC_OK;
}

/* Setup phase, Sec. 4.1: coarsen by caliber-1 aggregation until n < 150, or
 * until relaxation is fast (TV energy ratio per sweep <= 0.1, when enabled), or the
 * aggregation stalls (alpha > 0.9), or the depth limit. */
static int32_t setup_graphs(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                            int32_t ngraphs, const int64_t *gptr, const orc_opts *o, orc_hier **out) {
    *out = NULL;
    int32_t st = validate_graphs(n, rp, col, w, ngraphs, gptr, o->negative_weights);
    if (st != ORC_OK) return st;
    orc_hier *h = (orc_hier *)calloc(1, sizeof(orc_hier));
    h->o = *o;
    h->ngraphs = ngraphs;
    h->gptr = (int64_t *)xcalloc((size_t)ngraphs + 1, sizeof(int64_t));
    memcpy(h->gptr, gptr, sizeof(int64_t) * ((size_t)ngraphs + 1));
    orc_level *L0 = &h->lv[0];
    L0->n = n; L0->nnz = rp[n];
    L0->rp = (int64_t *)xcalloc((size_t)(n + 1), sizeof(int64_t));
    L0->col = (int32_t *)xcalloc((size_t)L0->nnz, sizeof(int32_t));
    L0->w = (double *)xcalloc((size_t)L0->nnz, sizeof(double));
    memcpy(L0->rp, rp, sizeof(int64_t) * (size_t)(n + 1));
    memcpy(L0->col, col, sizeof(int32_t) * (size_t)L0->nnz);
    memcpy(L0->w, w, sizeof(double) * (size_t)L0->nnz);
    int32_t maxl = o->max_levels < 128 ? o->max_levels : 128;
    int32_t nagg = 0;   /* aggregation levels so far (the TV count grows with them) */
    int32_t nxl = o->lgmg_nx;   /* Lean Geometric MG: the current grid side */
    if (nxl > 0 && (int64_t)nxl * nxl != n) { orc_free(h); return ORC_ERR_ARG; }
    for (int32_t l = 0;; l++) {
        orc_level *L = &h->lv[l];
        level_diag(L);
        h->L = l + 1;
        if (L->n < o->n_coarsest || l + 1 >= maxl || (nxl > 0 && (nxl % 2 != 0 || nxl < 6))) {
            if (nxl > 0) level_colour_rb(L, nxl);
            else level_colour(L, o->seed, l, 1, o->relax_rule, o->colour_rule);
            L->stop_reason = L->n < o->n_coarsest ? 1 : 4;
            st = make_coarsest(L, o);
            break;
        }
        if (nxl > 0) {   /* Lean Geometric MG: 1:2 coarsening in both directions, 2x2 aggregates */
            level_colour_rb(L, nxl);
            const int32_t nc2 = nxl / 2;
            L->agg = (int32_t *)xcalloc((size_t)L->n, sizeof(int32_t));
            L->state = (int32_t *)xcalloc((size_t)L->n, sizeof(int32_t));
            L->hub = (uint8_t *)xcalloc((size_t)L->n, 1);
            for (int64_t u = 0; u < L->n; u++)
                L->agg[u] = (int32_t)((u / nxl) / 2 * nc2 + (u % nxl) / 2);
            L->nc = (int64_t)nc2 * nc2;
            L->alpha = (double)L->nc / (double)L->n;
            galerkin(L, &h->lv[l + 1]);
            nxl = nc2;
            continue;
        }
        if (o->elim) {   /* low-degree elimination before aggregating, Sec. 3.2 */
            int32_t *cidx = (int32_t *)xcalloc((size_t)L->n, sizeof(int32_t));
            int64_t nF = elim_select(L, elim_key(o->seed, l), cidx);
            if (nF >= 1 && (double)nF >= o->elim_min_frac * (double)L->n) {
                level_colour(L, o->seed, l, 0, o->relax_rule, o->colour_rule);
                L->elim = 1;
                L->nF = nF;
                L->cidx = cidx;
                L->nc = L->n - nF;
                eliminate(L, cidx, &h->lv[l + 1]);
                continue;
            }
            free(cidx);
        }
        level_colour(L, o->seed, l, 1, o->relax_rule, o->colour_rule);
        int32_t K = o->k_finest + o->k_step * nagg;
        if (K > o->k_max) K = o->k_max;
        if (K > 16) K = 16;
        if (K < 1) K = 1;
        L->K = K;
        L->X = (double *)xcalloc((size_t)(L->n * K), sizeof(double));
        L->tv_ratio = relax_tvs(L, o, l);
        if (L->tv_ratio <= o->relax_fast_ratio) {
            L->stop_reason = 2;
            st = make_coarsest(L, o);
            break;
        }
        L->aff = (double *)xcalloc((size_t)L->nnz, sizeof(double));
        L->q = (double *)xcalloc((size_t)L->nnz, sizeof(double));
        L->score = (double *)xcalloc((size_t)L->nnz, sizeof(double));
        orc_edge_scores(L->n, L->rp, L->col, L->w, K, L->X, o->q_max, o->weak_tol,
                        L->aff, L->q, L->score);
        L->hub = (uint8_t *)xcalloc((size_t)L->n, 1);
        orc_hubs(L->n, L->rp, L->col, L->w, o->hub_factor, L->hub);
        L->state = (int32_t *)xcalloc((size_t)L->n, sizeof(int32_t));
        L->agg = (int32_t *)xcalloc((size_t)L->n, sizeof(int32_t));
        aggregate(L, o, agg_key(o->seed, l));
        if (L->alpha > o->alpha_stall) {
            L->stop_reason = 3;
            st = make_coarsest(L, o);
            break;
        }
        galerkin(L, &h->lv[l + 1]);
        nagg++;
    }
    cycle_indices(h);
    if (st != ORC_OK) { orc_free(h); return st; }
    *out = h;
    return ORC_OK;
}

int32_t orc_setup_graphs(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                         int32_t ngraphs, const int64_t *gptr, const orc_opts *o, orc_hier **out) {
    const int saved = g_plain_sums;
    g_plain_sums = o->plain_sums != 0;
    int32_t st = setup_graphs(n, rp, col, w, ngraphs, gptr, o, out);
    g_plain_sums = saved;
    return st;
}

int32_t orc_setup(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                  const orc_opts *o, orc_hier **out) {
    *out = NULL;
    if (n < 1) return ORC_ERR_ARG;
    int64_t gptr[2] = {0, n};
    return orc_setup_graphs(n, rp, col, w, 1, gptr, o, out);
}

void orc_free(orc_hier *h) {
    if (!h) return;
    free(h->gptr);
    for (int32_t l = 0; l < h->L; l++) {
        orc_level *L = &h->lv[l];
        free(L->rp); free(L->col); free(L->w); free(L->diag); free(L->colour);
        free(L->X); free(L->aff); free(L->q); free(L->score); free(L->hub);
        free(L->state); free(L->agg); free(L->chol); free(L->comp); free(L->cidx);
    }
    free(h);
}

int32_t orc_num_levels(const orc_hier *h) { return h->L; }

void orc_level_info(const orc_hier *h, int32_t l, int64_t *info) {
    const orc_level *L = &h->lv[l];
    memset(info, 0, sizeof(int64_t) * 16);
    info[0] = L->n; info[1] = L->nnz; info[2] = L->ncolours; info[3] = L->K; info[4] = L->nc;
    info[5] = L->rounds; info[6] = L->sel_round; info[7] = L->coarsest; info[8] = L->stop_reason;
    memcpy(&info[9], &L->alpha, 8); memcpy(&info[10], &L->gamma_l, 8); memcpy(&info[11], &L->tv_ratio, 8);
    info[12] = L->jp_rounds;
    info[13] = L->elim; info[14] = L->nF;
}

void orc_level_csr(const orc_hier *h, int32_t l, int64_t *rp, int32_t *col, double *w) {
    const orc_level *L = &h->lv[l];
    memcpy(rp, L->rp, sizeof(int64_t) * (size_t)(L->n + 1));
    memcpy(col, L->col, sizeof(int32_t) * (size_t)L->nnz);
    memcpy(w, L->w, sizeof(double) * (size_t)L->nnz);
}

void orc_level_colour(const orc_hier *h, int32_t l, int32_t *colour) {
    memcpy(colour, h->lv[l].colour, sizeof(int32_t) * (size_t)h->lv[l].n);
}

void orc_level_tv(const orc_hier *h, int32_t l, double *X) {
    const orc_level *L = &h->lv[l];
    if (L->X) memcpy(X, L->X, sizeof(double) * (size_t)(L->n * L->K));
}

void orc_level_scores(const orc_hier *h, int32_t l, double *aff, double *q, double *score) {
    const orc_level *L = &h->lv[l];
    if (!L->aff) return;
    memcpy(aff, L->aff, sizeof(double) * (size_t)L->nnz);
    memcpy(q, L->q, sizeof(double) * (size_t)L->nnz);
    memcpy(score, L->score, sizeof(double) * (size_t)L->nnz);
}

void orc_level_elim(const orc_hier *h, int32_t l, int32_t *cidx) {
    const orc_level *L = &h->lv[l];
    if (L->cidx) memcpy(cidx, L->cidx, sizeof(int32_t) * (size_t)L->n);
}

void orc_level_agg(const orc_hier *h, int32_t l, int32_t *agg, int32_t *state, uint8_t *hub) {
    const orc_level *L = &h->lv[l];
    if (!L->agg) return;
    memcpy(agg, L->agg, sizeof(int32_t) * (size_t)L->n);
    memcpy(state, L->state, sizeof(int32_t) * (size_t)L->n);
    memcpy(hub, L->hub, (size_t)L->n);
}

/* ------------------------------------------------------------------------- */
/* Solve phase, Sec. 4.2 and Fig. 4.2                                          */
/* ------------------------------------------------------------------------- */

typedef struct {
    const orc_hier *h;
    int adaptive;
    double mu;
    double **x, **b, **r;   /* per-level iterate, right-hand side, residual */
    int32_t *visits;        /* per-level counter of coarse corrections, reset per cycle */
} solve_ctx;

static void relax(const orc_level *L, const double *b, double *x) {
    orc_gs_sweep_colour(L->n, L->rp, L->col, L->w, L->colour, L->ncolours, b, x);
}

static void residual(const orc_level *L, const double *b, const double *x, double *r) {
    for (int64_t u = 0; u < L->n; u++) {
        double s = b[u] - L->diag[u] * x[u];
        for (int64_t e = L->rp[u]; e < L->rp[u + 1]; e++) s += L->w[e] * x[L->col[e]];
        r[u] = s;
    }
}

static double dot(int64_t n, const double *a, const double *b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

static void coarsest_solve(const orc_level *L, const orc_opts *o, const double *b, double *x) {
    if (L->chol) { chol_solve(L->n, L->chol, b, x); subtract_mean_comp(L->n, x, L->comp, L->ncomp); return; }
    for (int64_t i = 0; i < L->n; i++) x[i] = 0.0;
    for (int s = 0; s < o->coarse_sweeps; s++) relax(L, b, x);
    subtract_mean_comp(L->n, x, L->comp, L->ncomp);
}

/* Iterate recombination, Eq. (3.13): y = x + sum_i alpha_i (x_i - x) with alpha
 * minimising ||b - A y||_2.  With r = b - A x and r_i = b - A x_i,
 * A(x_i - x) = r - r_i, so alpha solves G alpha = h, G_ij = <r - r_i, r - r_j>,
 * h_i = <r, r - r_i> (theta <= 2 unknowns; a singular G gives alpha = 0). */
static void recombine(const orc_level *L, const double *b, double *x, int theta,
                      double **xs, double **rs, double *r) {
    int64_t n = L->n;
    residual(L, b, x, r);
    double G[2][2] = {{0, 0}, {0, 0}}, hv[2] = {0, 0}, al[2] = {0, 0};
    double *d0 = (double *)malloc(sizeof(double) * (size_t)n);
    double *d1 = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t u = 0; u < n; u++) d0[u] = r[u] - rs[0][u];
    if (theta == 2) for (int64_t u = 0; u < n; u++) d1[u] = r[u] - rs[1][u];
    G[0][0] = dot(n, d0, d0); hv[0] = dot(n, r, d0);
    if (theta == 2) { G[0][1] = G[1][0] = dot(n, d0, d1); G[1][1] = dot(n, d1, d1); hv[1] = dot(n, r, d1); }
    if (theta == 1) {
        if (G[0][0] > 0.0) al[0] = hv[0] / G[0][0];
    } else {
        double det = G[0][0] * G[1][1] - G[0][1] * G[1][0];
        if (det > 1e-14 * G[0][0] * G[1][1] && det > 0.0) {
            al[0] = (hv[0] * G[1][1] - G[0][1] * hv[1]) / det;
            al[1] = (G[0][0] * hv[1] - G[1][0] * hv[0]) / det;
        } else if (G[0][0] > 0.0) {
            al[0] = hv[0] / G[0][0];
        }
    }
    for (int64_t u = 0; u < n; u++) {
        double y = x[u] + al[0] * (xs[0][u] - x[u]);
        if (theta == 2) y += al[1] * (xs[1][u] - x[u]);
        x[u] = y;
    }
    free(d0); free(d1);
}

static void visit(solve_ctx *c, int32_t l, int theta);

/* One step of a level whose next level is its Schur complement (Sec. 3.2 and
 * Sec. 4.2: gamma = 1, no relaxation, no energy correction).  With r = b - A x,
 * the coarse right-hand side is r_C - A_CF A_FF^-1 r_F, i.e.
 * b^c_c = r_c + sum over f in F of w_cf r_f / a_ff; after the coarse visit
 * x_C += x^c, and x_F is recomputed exactly, x_f = (b_f + sum_c w_fc x_c) / a_ff
 * (back-substitution; with an exact coarse solve the level is solved exactly). */
static void elim_step(solve_ctx *c, int32_t l) {
    const orc_hier *h = c->h;
    const orc_level *F = &h->lv[l], *C = &h->lv[l + 1];
    int64_t n = F->n;
    double *x = c->x[l], *b = c->b[l], *r = c->r[l];
    double *bc = c->b[l + 1], *xc = c->x[l + 1];
    residual(F, b, x, r);
    for (int64_t u = 0; u < n; u++) {
        int32_t U = F->cidx[u];
        if (U < 0) continue;
        double s = r[u];
        for (int64_t e = F->rp[u]; e < F->rp[u + 1]; e++) {
            int32_t f = F->col[e];
            if (F->cidx[f] < 0) s += F->w[e] * r[f] / F->diag[f];
        }
        bc[U] = s;
        xc[U] = 0.0;
    }
    if (C->coarsest) coarsest_solve(C, &h->o, bc, xc);
    else if (C->elim) elim_step(c, l + 1);
    else visit(c, l + 1, 1);
    for (int64_t u = 0; u < n; u++) if (F->cidx[u] >= 0) x[u] += xc[F->cidx[u]];
    for (int64_t f = 0; f < n; f++) {
        if (F->cidx[f] >= 0) continue;
        double s = b[f];
        for (int64_t e = F->rp[f]; e < F->rp[f + 1]; e++) s += F->w[e] * x[F->col[e]];
        x[f] = s / F->diag[f];
    }
}

/* theta visits of level l: elimination steps, or the two-level steps below */
static void visit_level(solve_ctx *c, int32_t l, int theta) {
    if (c->h->lv[l].elim) {
        for (int i = 0; i < theta; i++) elim_step(c, l);
        return;
    }
    visit(c, l, theta);
}

/* One visit to level l (< L-1) consisting of theta two-level steps, Sec. 3.4.6
 * and Fig. 4.2: pre-relax nu1, [save x_i, r_i], b^{l+1} = mu P^T r, coarse
 * visit, x += P x^{l+1}, post-relax nu2; then recombine when adaptive and l is
 * not the finest level.  The coarse visit's own theta comes from the fractional
 * cycle index (build reading): the k-th coarse correction of a level (counted
 * from 0 within the cycle) performs ceil((k+1) g) - ceil(k g) visits, g = gamma^l. */
static void visit(solve_ctx *c, int32_t l, int theta) {
    const orc_hier *h = c->h;
    const orc_level *F = &h->lv[l], *C = &h->lv[l + 1];
    const orc_opts *o = &h->o;
    int64_t n = F->n;
    double *x = c->x[l], *b = c->b[l], *r = c->r[l];
    int recomb = c->adaptive && (l >= 1 || h->o.recomb_finest);
    double *xs[2] = {NULL, NULL}, *rs[2] = {NULL, NULL};
    for (int i = 0; i < theta; i++) {
        for (int s = 0; s < o->nu1; s++) relax(F, b, x);
        residual(F, b, x, r);
        if (recomb) {
            xs[i] = (double *)malloc(sizeof(double) * (size_t)n);
            rs[i] = (double *)malloc(sizeof(double) * (size_t)n);
            memcpy(xs[i], x, sizeof(double) * (size_t)n);
            memcpy(rs[i], r, sizeof(double) * (size_t)n);
        }
        double *bc = c->b[l + 1], *xc = c->x[l + 1];
        for (int64_t U = 0; U < C->n; U++) { bc[U] = 0.0; xc[U] = 0.0; }
        for (int64_t u = 0; u < n; u++) bc[F->agg[u]] += r[u];
        for (int64_t U = 0; U < C->n; U++) bc[U] *= c->mu;
        if (C->coarsest) {
            coarsest_solve(C, o, bc, xc);
        } else {
            int32_t k = c->visits[l]++;
            double g = F->gamma_l;
            int th = (int)(ceil((double)(k + 1) * g) - ceil((double)k * g));
            if (th < 1) th = 1;
            if (th > 2) th = 2;
            visit_level(c, l + 1, th);
        }
        for (int64_t u = 0; u < n; u++) x[u] += xc[F->agg[u]];
        for (int s = 0; s < o->nu2; s++) relax(F, b, x);
    }
    if (recomb) recombine(F, b, x, theta, xs, rs, r);
    for (int i = 0; i < 2; i++) { free(xs[i]); free(rs[i]); }
}

static void ctx_init(solve_ctx *c, const orc_hier *h, int adaptive) {
    c->h = h; c->adaptive = adaptive;
    c->mu = adaptive ? h->o.mu_adaptive : h->o.mu_flat;
    c->x = (double **)calloc((size_t)h->L, sizeof(double *));
    c->b = (double **)calloc((size_t)h->L, sizeof(double *));
    c->r = (double **)calloc((size_t)h->L, sizeof(double *));
    c->visits = (int32_t *)calloc((size_t)h->L, sizeof(int32_t));
    for (int32_t l = 0; l < h->L; l++) {
        c->x[l] = (double *)xcalloc((size_t)h->lv[l].n, sizeof(double));
        c->b[l] = (double *)xcalloc((size_t)h->lv[l].n, sizeof(double));
        c->r[l] = (double *)xcalloc((size_t)h->lv[l].n, sizeof(double));
    }
}

static void ctx_free(solve_ctx *c) {
    for (int32_t l = 0; l < c->h->L; l++) { free(c->x[l]); free(c->b[l]); free(c->r[l]); }
    free(c->x); free(c->b); free(c->r); free(c->visits);
}

/* One cycle on the finest level followed by the mean subtraction M (Sec. 4.2). */
static void cycle_once(solve_ctx *c, const double *b, double *x) {
    const orc_hier *h = c->h;
    const orc_level *F = &h->lv[0];
    int64_t n = F->n;
    if (F->coarsest) {
        coarsest_solve(F, &h->o, b, x);
        return;
    }
    memcpy(c->x[0], x, sizeof(double) * (size_t)n);
    memcpy(c->b[0], b, sizeof(double) * (size_t)n);
    for (int32_t l = 0; l < h->L; l++) c->visits[l] = 0;
    visit_level(c, 0, 1);
    memcpy(x, c->x[0], sizeof(double) * (size_t)n);
    subtract_mean_ranges(x, h->ngraphs, h->gptr);
}

static double norm2(int64_t n, const double *v) { return sqrt(dot(n, v, v)); }

int32_t orc_cycle(const orc_hier *h, const double *b, double *x, int32_t adaptive) {
    solve_ctx c;
    ctx_init(&c, h, adaptive);
    cycle_once(&c, b, x);
    ctx_free(&c);
    return ORC_OK;
}

/* Cycles until every graph g of the union has ||b_g - A x_g|| <= tol ||b_g||
 * (one graph: the plain relative residual test).  res_hist holds the norm of
 * the whole residual. */
int32_t orc_solve(const orc_hier *h, const double *b, double *x, double tol, int32_t max_cycles,
                  int32_t adaptive, double *res_hist, int32_t *cycles_out) {
    const orc_level *F = &h->lv[0];
    int64_t n = F->n;
    int32_t G = h->ngraphs;
    for (int32_t g = 0; g < G; g++) {
        double sb = 0.0, ab = 0.0;
        for (int64_t i = h->gptr[g]; i < h->gptr[g + 1]; i++) { sb += b[i]; ab += fabs(b[i]); }
        if (fabs(sb) > 1e-10 * (ab > 0 ? ab : 1.0)) return ORC_ERR_RHS_NOT_ZERO_SUM;
    }
    solve_ctx c;
    ctx_init(&c, h, adaptive);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *bn = (double *)malloc(sizeof(double) * (size_t)G);
    for (int32_t g = 0; g < G; g++) bn[g] = norm2(h->gptr[g + 1] - h->gptr[g], b + h->gptr[g]);
    residual(F, b, x, r);
    double rn = norm2(n, r);
    if (res_hist) res_hist[0] = rn;
    int32_t it = 0;
    for (;;) {
        int pending = 0;
        for (int32_t g = 0; g < G && !pending; g++)
            if (norm2(h->gptr[g + 1] - h->gptr[g], r + h->gptr[g]) > tol * bn[g]) pending = 1;
        if (!pending || it >= max_cycles) break;
        cycle_once(&c, b, x);
        residual(F, b, x, r);
        rn = norm2(n, r);
        it++;
        if (res_hist) res_hist[it] = rn;
    }
    if (cycles_out) *cycles_out = it;
    free(r); free(bn);
    ctx_free(&c);
    return ORC_OK;
}

int32_t orc_adjoint(const orc_hier *h, const double *x, const double *g, double *lambda,
                    const int32_t *eu, const int32_t *ev, int64_t m, double *dw,
                    double tol, int32_t max_cycles, int32_t adaptive) {
    int64_t n = h->lv[0].n;
    double *gz = (double *)malloc(sizeof(double) * (size_t)n);
    memcpy(gz, g, sizeof(double) * (size_t)n);
    subtract_mean_ranges(gz, h->ngraphs, h->gptr);
    for (int64_t i = 0; i < n; i++) lambda[i] = 0.0;
    int32_t st = orc_solve(h, gz, lambda, tol, max_cycles, adaptive, NULL, NULL);
    free(gz);
    if (st != ORC_OK) return st;
    /* dL/dw_uv = -(lambda_u - lambda_v)(x_u - x_v): dA/dw_uv = (e_u - e_v)(e_u - e_v)^T, Eq. (1.2) */
    if (dw)
        for (int64_t e = 0; e < m; e++)
            dw[e] = -(lambda[eu[e]] - lambda[ev[e]]) * (x[eu[e]] - x[ev[e]]);
    return ORC_OK;
}
