// lamg_internal.cuh -- internal data structures and helpers of the GB300 LAMG
// library (Livne & Brandt, arXiv 1108.1310).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/lamg.h"

namespace lamg {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------

struct Error {
    lamg_status status;
    std::string msg;
};

void set_last_error(const std::string &msg);

#define LAMG_CUDA(expr)                                                                  \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            throw ::lamg::Error{e_ == cudaErrorMemoryAllocation ? LAMG_ERR_OOM : LAMG_ERR_CUDA, \
                                std::string(#expr) + ": " + cudaGetErrorString(e_) +     \
                                    " (" + __FILE__ + ":" + std::to_string(__LINE__) + ")"}; \
        }                                                                                \
    } while (0)

// Every kernel launch is followed by LAMG_CHECK_LAUNCH(), which also counts it.
void note_launch();
int64_t launch_count();

#define LAMG_CHECK_LAUNCH()                  \
    do {                                     \
        ::lamg::note_launch();               \
        LAMG_CUDA(cudaGetLastError());       \
    } while (0)

#define LAMG_REQUIRE(cond, status, text)                                                 \
    do {                                                                                 \
        if (!(cond)) throw ::lamg::Error{(status), std::string(text)};                   \
    } while (0)

// Row tiers.  Setup: rows of <= kLongRow terms are handled by one thread,
// up to kHugeRow by one warp, longer ones by a block of kBlk threads; the
// canonical summation order (left to right / 32-lane tree / 1024-lane tree)
// switches at the same lengths.  The solve uses kHugeSolve for its block tier.
constexpr int kLongRow = 32;
constexpr int kHugeRow = 512;
constexpr int kHugeSolve = 512;
constexpr int kTailChunk = 128;   // entries of a tail row summed by one warp in a tail colour step
constexpr int kBlk = 1024;

// ---------------------------------------------------------------------------
// Device buffers (owned, freed with the handle)
// ---------------------------------------------------------------------------

template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DBuf() { release(); }
    void alloc(size_t count) {
        release();
        n = count;
        if (count) LAMG_CUDA(cudaMalloc((void **)&p, sizeof(T) * count));
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    T *get() const { return p; }
    size_t bytes() const { return sizeof(T) * n; }
};

// ---------------------------------------------------------------------------
// Hierarchy
// ---------------------------------------------------------------------------

// Setup-phase view of one level, natural node order (Sec. 4.1).
struct SetupLevel {
    int32_t n = 0;
    int64_t nnz = 0;
    DBuf<int32_t> rp, col;         // CSR, int32 row pointers (nnz < 2^31)
    DBuf<double> w;                // FP64 weights
    DBuf<int32_t> colour;          // Jones-Plassmann colour
    int32_t ncolours = 0, jp_rounds = 0;
    DBuf<int32_t> sorder;          // nodes sorted by (colour, row tier, id)
    std::vector<int32_t> cb;       // colour c, tier t: sorder[cb[4c+t], cb[4c+t+1]); cb[4c+3] = end
    DBuf<int32_t> cb_dev;          // same on the device
    DBuf<int32_t> agg, state;      // aggregation result (non-coarsest levels)
    DBuf<uint8_t> hub;
    DBuf<double> tv, aff, q, score;  // kept only with keep_setup_data
    int32_t K = 0, nc = 0, rounds = 0, sel_round = 0;
    int32_t coarsest = 0, stop_reason = 0;
    double alpha = 0.0, gamma_l = 0.0, tv_ratio = 0.0;
    // low-degree elimination (Sec. 3.2): the next level is the Schur complement on C
    int32_t elim = 0;
    int64_t nF = 0;
    DBuf<int32_t> cidx;            // coarse index of each C node, -1 for F nodes
};

// Solve-phase layout of one level: rows permuted so that each colour is a
// contiguous range, short rows (<= kLongRow entries) before long rows within
// each colour; vectors live in this order.
struct SolveLevel {
    int32_t n = 0;
    int64_t nnz = 0;
    DBuf<int32_t> rp, col;         // permuted CSR (columns in permuted ids)
    DBuf<double> w64;
    DBuf<float> w32;
    DBuf<int32_t> perm;            // perm[i] = natural id of permuted row i
    std::vector<int32_t> cb;       // colour c, tier t rows: [cb[4c+t], cb[4c+t+1]); cb[4c+3] = end
    DBuf<int32_t> cb_dev;
    // sweep plan per precision (0 = FP64, 1 = FP32): segments (c0, c1, single);
    // single = 1: colours c0..c1-1 in one single-block launch, else colour c0 alone
    std::vector<int32_t> seg[2];
    DBuf<int32_t> wrows, brows;    // all warp-tier / block-tier rows (permuted ids)
    int32_t nw = 0, nb = 0;
    // transfer to the next coarser level (absent on the coarsest level)
    DBuf<int32_t> pagg;            // permuted fine row -> permuted coarse id
    DBuf<int32_t> mptr, mlist;     // members of each coarse id (permuted fine ids)
    DBuf<int32_t> wagg, bagg;      // coarse ids whose member lists are warp / block tier
    int32_t nwagg = 0, nbagg = 0;
    // tail colours (power-law levels: many colours of a few long hub rows at the
    // end of the colour order): rows tt0 .. n-1, colours tc0 .. ncolours-1.  The
    // sweep splits each tail row into its part outside the tail (fixed while the
    // tail colours run) and its part inside (trp/tcol local CSR, tw weights).
    int32_t tc0 = -1, tt0 = 0, tn = 0, tnc = 0;
    int64_t tnnz = 0;
    DBuf<int32_t> trp, tcol, tcb;  // local CSR of the tail block, tail colour bounds (local rows)
    DBuf<int32_t> trq;             // per local row: first chunk (kTailChunk entries) of its local row
    int32_t tmaxq = 0;             // most chunks in one tail colour
    DBuf<double> tw64, tdeg64;     // weights and full weighted degrees of tail rows
    DBuf<float> tw32, tdeg32;
    // transfer to a Schur-complement next level (Sec. 3.2) instead of pagg/mlist
    int32_t elim = 0;
    DBuf<int32_t> ecx;             // permuted row -> permuted coarse id, -1 for eliminated rows
    DBuf<double> ed64;             // a_ii of each row (used for the eliminated rows)
    DBuf<float> ed32;
    // coarsest level
    int32_t dense = 0;
    DBuf<double> minv;             // (A + 11^T/n)^-1, n x n, if dense
    // sliced ELL of the thread-tier rows (<= kLongRow entries): slices of 32
    // consecutive rows of one colour; sl[k] = {first row, rows, pairs, first pair}.
    // Entry pair p of the row in lane l of slice k sits at (first pair + p) * 32 + l,
    // so a warp's load of pair p is 32 consecutive 16-byte vectors.  FP32:
    // {c0, c1, w0 bits, w1 bits}; FP64: {c0, c1} and {w0, w1}.  Short rows are
    // padded with (own row, weight 0).
    int32_t nsl = 0;
    std::vector<int32_t> csl;      // colour c: slices [csl[c], csl[c+1])
    DBuf<int32_t> csl_dev;
    DBuf<int4> sl;
    DBuf<uint4> ell32;
    DBuf<int2> ellc;
    DBuf<double2> ellw64;
};

// Per-level vectors of one precision.
template <class T>
struct LevelVecs {
    DBuf<T> x, b, r, xs0, xs1, rs0, rs1;
};

// Workspace of batched solves: level vectors of n x ld interleaved columns
// (ld = 4 * groups), their descriptors, programs and engine scratch.
struct BatchState {
    int32_t groups = 0, ld = 0, grid = 0;
    std::vector<LevelVecs<double>> v64;
    std::vector<LevelVecs<float>> v32;
    DBuf<double> r64;              // FP64 outer residual, n x ld (permuted)
    DBuf<double> out;              // per-column results, 4 x ld
    DBuf<char> lv64, lv32;         // level descriptors (MKLevel)
    DBuf<double> part;             // grid x 8 x ld partial sums
    DBuf<unsigned int> bar;
    DBuf<int32_t> err;
    DBuf<int32_t> prog[6];         // (FP64 step, FP32-IR step, residual only) x adaptive
    int32_t len[6] = {0, 0, 0, 0, 0, 0};
    int32_t prof_pending = 0;      // a timed launch whose events are not read yet
    int64_t prof_bytes = 0;        // its algorithmic bytes
};

struct Hierarchy;

}  // namespace lamg

struct lamg_ctx {
    lamg_options opt;
    std::vector<lamg::SetupLevel> sl;
    std::vector<lamg::SolveLevel> lv;
    int32_t L = 0;
    int64_t n = 0;
    double t_setup_s = 0.0;
    // solve workspaces
    std::vector<lamg::LevelVecs<double>> v64;
    std::vector<lamg::LevelVecs<float>> v32;
    lamg::DBuf<double> scratch;     // reductions, recombination coefficients
    lamg::DBuf<double> xnat, bnat;  // level-1 vectors for host-array solves
    lamg::DBuf<double> r64;         // FP64 outer residual (permuted)
    double *host_pinned = nullptr;  // pinned readback slots
    // cycle engine: level descriptors, programs (FP64 step, FP32-IR step, one cycle) x adaptive
    lamg::DBuf<char> eng_lv64, eng_lv32;
    lamg::DBuf<int32_t> eng_prog[6];
    int32_t eng_len[6] = {0, 0, 0, 0, 0, 0};
    lamg::DBuf<double> eng_part;
    lamg::DBuf<unsigned int> eng_bar;
    lamg::DBuf<int32_t> eng_err;
    lamg::DBuf<unsigned long long> eng_optime;
    int32_t eng_grid = 0;
    // profiling of the engine launches
    int32_t prof_on = 0;
    std::vector<cudaEvent_t> prof_ev;
    double prof_ms = 0.0;
    int64_t prof_count = 0;
    int64_t prof_bytes = 0;
    lamg_stats last{};
    std::unique_ptr<lamg::BatchState> mr;   // batched-solve workspace (lazily built)
    int32_t batch_cols = 0;                 // columns per batched engine run (0: the largest)
    // block-diagonal union of several graphs (ngraphs == 1: one connected graph)
    int32_t ngraphs = 1;
    std::vector<int64_t> gptr;              // host: level-1 node range of each graph
    lamg::DBuf<int64_t> gptr_d;
    lamg::DBuf<int32_t> iperm0;             // natural level-1 id -> permuted row
    lamg::DBuf<int32_t> gid0, gidnat;       // graph of each permuted / natural level-1 row
    lamg::DBuf<double> gsum, gnorm, gstat;  // per-graph means, ||r||^2, and b statistics (3 per graph)
    std::vector<double> grel;               // per-graph ||r_g|| / ||b_g|| of the last solve
};

namespace lamg {

// setup.cu
void build_hierarchy(lamg_ctx *h, int64_t n, const int64_t *row_ptr, const int32_t *col,
                     const void *w, int32_t w_is_fp32, cudaStream_t s);
void validate_graph(int64_t n, const int64_t *row_ptr, const int32_t *col, const void *w,
                    int32_t w_is_fp32, cudaStream_t s, int32_t ngraphs = 1, const int64_t *gptr = nullptr,
                    int32_t signed_w = 0);

// Single-block thresholds of the cycle engine: a level whose n + nnz is at most
// sb_work(prec) runs every op on one block (no grid barrier); a colour of at
// most tail_work(prec) entries joins a single-block run.  One SM streams FP32
// rows from L2 faster than a grid-wide phase completes, up to a few hundred
// KB; FP64 arithmetic on one SM is slow (1/64 rate), so its limits are lower.
int64_t sb_work(const lamg_options &o, int prec);    // prec 0 = FP64, 1 = FP32
int64_t tail_work(const lamg_options &o, int prec);
constexpr int64_t kSBWork = 16384;

// cycle.cu
void engine_prepare(lamg_ctx *h);
void engine_run(lamg_ctx *h, int kind, int adaptive, double mu, cudaStream_t s);
bool engine_failed(lamg_ctx *h, cudaStream_t s);
// op timer table: (level < 128) x (op type < 32) x (grid, single block) x (ns, count)
constexpr int kOpTimeSlots = 128 * 32 * 2 * 2;
void engine_op_times(lamg_ctx *h, int mode, std::vector<unsigned long long> &out);
// algorithmic bytes of one cycle with `cols` right-hand sides (weights of wb bytes)
int64_t cycle_bytes(lamg_ctx *h, int wb, int cols);
void build_program(lamg_ctx *h, int kind, int adaptive, std::vector<int32_t> &out, int groups = 0);
bool engine_noalloc_ready(lamg_ctx *h, int adaptive);
int32_t barrier_selftest(int32_t hold_one, cudaStream_t s);
int32_t *engine_run_noalloc(lamg_ctx *h, int adaptive, double mu, cudaStream_t s);

// solve.cu
void build_solve_layout(lamg_ctx *h, cudaStream_t s);
void build_graph_maps(lamg_ctx *h, cudaStream_t s);
void solve_device(lamg_ctx *h, const double *b, double *x, double tol, lamg_precision p,
                  cudaStream_t s, lamg_stats *st);
void solve_batched_device(lamg_ctx *h, int32_t nrhs, const double *B, double *X, int64_t ld,
                          double tol, lamg_precision p, cudaStream_t s, lamg_stats *st);
void set_batch_cols(lamg_ctx *h, int32_t cols);
void autotune_batched(lamg_ctx *h, int32_t nrhs, lamg_precision p, cudaStream_t s, int32_t *chosen,
                      double *ms_out);
void prepare_solve(lamg_ctx *h);
void cycle_device(lamg_ctx *h, const double *b, double *x, int32_t adaptive, cudaStream_t s);
void cycle_device_noalloc(lamg_ctx *h, const double *b, double *x, int32_t adaptive, cudaStream_t s);
void adjoint_device(lamg_ctx *h, const double *x, const double *g, double *lambda,
                    const int32_t *eu, const int32_t *ev, int64_t m, void *dw, int32_t dw32,
                    double tol, lamg_precision p, cudaStream_t s, lamg_stats *st);
void release_solve(lamg_ctx *h);

// prims.cu
void exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);
template <class K, class V>
void radix_sort_pairs(K *keys, V *vals, K *ktmp, V *vtmp, int64_t n, int nbits, cudaStream_t s);
int64_t compact_indices(const uint8_t *flags, int32_t *out_idx, int64_t n, cudaStream_t s);
int32_t reduce_max_i32(const int32_t *a, int64_t n, cudaStream_t s);
int64_t count_equal_i32(const int32_t *a, int64_t n, int32_t value, cudaStream_t s);

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Temporary device memory from the stream-ordered pool, freed at scope exit.
template <class T>
struct Tmp {
    T *p = nullptr;
    cudaStream_t s;
    Tmp(size_t count, cudaStream_t st) : s(st) {
        if (count) LAMG_CUDA(cudaMallocAsync((void **)&p, sizeof(T) * count, st));
    }
    ~Tmp() {
        if (p) cudaFreeAsync(p, s);
    }
    Tmp(const Tmp &) = delete;
    Tmp &operator=(const Tmp &) = delete;
    T *get() const { return p; }
};

// true when the hierarchy has a level followed by elimination (Sec. 3.2)
inline bool has_elim(const lamg_ctx *h) {
    for (int l = 0; l + 1 < h->L; l++)
        if (h->sl[l].elim) return true;
    return false;
}

template <class T>
inline T read_scalar(const T *dptr, cudaStream_t s) {
    T v;
    LAMG_CUDA(cudaMemcpyAsync(&v, dptr, sizeof(T), cudaMemcpyDeviceToHost, s));
    LAMG_CUDA(cudaStreamSynchronize(s));
    return v;
}

}  // namespace lamg
