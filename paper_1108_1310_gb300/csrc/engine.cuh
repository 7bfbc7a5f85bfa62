// engine.cuh -- definitions shared by the single- and multi-right-hand-side
// cycle engines: level descriptors, the op codes of a cycle program, the
// bounded grid barrier and the fixed-order block reductions.
#pragma once

#include "solve_rows.cuh"

namespace lamg {

constexpr int kEngThreads = 1024;
constexpr long long kMaxSpins = 1ll << 21;  // one to two seconds of polling

template <class T>
struct MKLevel {
    int32_t n, nc;
    const int32_t *rp, *col;
    const T *w;
    const int32_t *cb;
    const int32_t *wrows, *brows;
    int32_t nw, nb;
    const int32_t *pagg, *mptr, *mlist, *wagg, *bagg;
    int32_t nwagg, nbagg;
    T *x, *b, *r, *xs0, *xs1, *rs0, *rs1;
    const double *minv;
    // tail colours (tn == 0: none)
    int32_t tt0, tn, tnc, tnnz, tmaxq;
    const int32_t *trp, *tcol, *tcb, *trq;
    const T *tw, *tdeg;
    // next level is this level's Schur complement (Sec. 3.2)
    const int32_t *ecx;   // permuted coarse id, -1 for an eliminated row
    const T *ed;          // a_ii of the eliminated rows
    // sliced ELL of the thread-tier rows (see SolveLevel)
    int32_t nsl;
    const int32_t *csl;
    const int4 *sl;
    const uint4 *ell32;
    const int2 *ellc;
    const double2 *ellw;
};

constexpr int kSellStage = 6;   // pairs of a slice staged in shared memory (rows of up to 12 entries)
// A warp with a single slice in an op has both slots to itself and stages up to
// 2 kSellStage pairs (rows of up to 24 entries: the coarse levels of a 3-D grid).
constexpr int kSellWide = 2 * kSellStage;
constexpr int kSellChunk = 3;   // staged pairs moved to registers at a time (a 7-point row has 3)
// per-warp staging of the FP32 sliced ELL in the engine's dynamic shared memory:
// two slots of kSellStage pairs x 32 lanes of 16 bytes
constexpr int kSellStageBytes = 2 * kSellStage * 32 * 16;

// 16-byte asynchronous copy global -> shared (L2 only), commit, wait
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ uint4 *sell_warp_buf() {
    extern __shared__ __align__(16) unsigned char smem[];
    return (uint4 *)(smem + (size_t)(threadIdx.x >> 5) * kSellStageBytes);
}

// Stage the first min(m.z, cap) pairs of slice m at slot `slot` of this warp's
// buffer (each lane copies its own 16-byte pairs; one commit group per call,
// possibly empty).  cap = kSellWide fills both slots from slot 0.
__device__ __forceinline__ void sell_stage(const MKLevel<float> &L, const int4 m, int lane, uint4 *wbuf, int slot,
                                           int cap) {
    uint4 *dst = wbuf + slot * kSellStage * 32 + lane;
    const uint4 *src = L.ell32 + (size_t)m.w * 32 + lane;
    const int nq = min(m.z, cap);
#pragma unroll 1
    for (int q = 0; q < nq; q++) cp_async16(dst + q * 32, src + (size_t)q * 32);
    cp_async_commit();
}

// A warp's first slice of an op, staged ahead: while its block waits in the
// barrier before the op, each warp loads the descriptor of its first slice and
// stages that slice's pairs (neither depends on x), so that after the barrier
// only the gathers of x remain on the op's critical path.  The descriptor
// waits in shared memory (one per warp).
struct SellPre {
    bool on;
};
__device__ __forceinline__ int4 &sell_pre_desc() {
    __shared__ int4 desc[kEngThreads / 32];
    return desc[threadIdx.x >> 5];
}

// Issue the staging of slice k0 of a walk [k0, k1) with step `step`, as
// sell_walk32 would at its start; false when the warp has no slice.
__device__ __forceinline__ bool sell_prestage(const MKLevel<float> &L, int64_t k0, int64_t k1, int64_t step,
                                              SellPre &pre) {
    pre.on = false;
    if (k0 >= k1) return false;
    const int4 m = L.sl[k0];
    sell_stage(L, m, threadIdx.x & 31, sell_warp_buf(), 0, k0 + step >= k1 ? kSellWide : kSellStage);
    if ((threadIdx.x & 31) == 0) sell_pre_desc() = m;
    __syncwarp();
    pre.on = true;
    return true;
}

// Walk the FP32 slices [k0, k1) with step `step`, the next slice's first pairs
// staged in shared memory while the current slice is processed (a warp with a
// single slice stages up to kSellWide pairs of it).  fn(m, st, nst) gets the
// slice, this lane's staged pairs (st[q * 32], q < nst) and their count.  A
// staged first slice (pre.on, from sell_prestage with the same range) is taken
// over and pre is cleared.  Every copy issued is waited for before returning.
template <class F>
__device__ __forceinline__ void sell_walk32(const MKLevel<float> &L, int64_t k0, int64_t k1, int64_t step,
                                            SellPre &pre, F fn) {
    const int lane = threadIdx.x & 31;
    uint4 *wbuf = sell_warp_buf();
    const bool single = k0 + step >= k1;
    int4 mc;
    if (pre.on) {
        mc = sell_pre_desc();
        pre.on = false;
    } else {
        if (k0 >= k1) return;
        mc = L.sl[k0];
        sell_stage(L, mc, lane, wbuf, 0, single ? kSellWide : kSellStage);
    }
    int slot = 0;
    for (int64_t k = k0; k < k1; k += step) {
        const bool more = k + step < k1;
        int4 mn = mc;
        if (more) {
            mn = L.sl[k + step];
            sell_stage(L, mn, lane, wbuf, slot ^ 1, kSellStage);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        fn(mc, (const uint4 *)(wbuf + slot * kSellStage * 32 + lane), min(mc.z, single ? kSellWide : kSellStage));
        slot ^= 1;
        mc = mn;
    }
}

// The dot products of a staged slice row: acc += sum w x[col] (res: w (x[col] - xi)),
// d += sum w over its nst staged pairs, in pair order, kSellChunk pairs at a time.
__device__ __forceinline__ void sell_row32(const uint4 *st, int nst, const float *__restrict__ x, float xi, bool res,
                                           float &acc, float &d) {
    for (int q0 = 0; q0 < nst; q0 += kSellChunk) {
        uint4 v[kSellChunk];
#pragma unroll
        for (int q = 0; q < kSellChunk; q++) v[q] = q0 + q < nst ? st[(q0 + q) * 32] : make_uint4(0, 0, 0, 0);
        float xv[2 * kSellChunk];
#pragma unroll
        for (int q = 0; q < kSellChunk; q++) {
            xv[2 * q] = x[v[q].x];
            xv[2 * q + 1] = x[v[q].y];
        }
#pragma unroll
        for (int q = 0; q < kSellChunk; q++) {
            const float w0 = __uint_as_float(v[q].z), w1 = __uint_as_float(v[q].w);
            if (res) acc += w0 * (xv[2 * q] - xi) + w1 * (xv[2 * q + 1] - xi);
            else acc += w0 * xv[2 * q] + w1 * xv[2 * q + 1];
            d += w0 + w1;
        }
    }
}

__device__ __forceinline__ float pw(const uint4 &v, int h) { return __uint_as_float(h ? v.w : v.z); }

// Slice dot products: lane l holds row m.x + l of slice m; acc += sum w x[col],
// d += sum w over the row's entries (padding adds 0).  The pairs are loaded four
// at a time before their gathers, so eight gathers are in flight per lane.
__device__ __forceinline__ void sell_dot(const MKLevel<float> &L, const int4 m, int lane, const float *__restrict__ x,
                                         float &acc, float &d) {
    const uint4 *__restrict__ p = L.ell32 + (size_t)m.w * 32 + lane;
    for (int q = 0; q < m.z; q += 4) {
        uint4 v[4];
#pragma unroll
        for (int k = 0; k < 4; k++) v[k] = q + k < m.z ? __ldg(p + (size_t)(q + k) * 32) : make_uint4(0, 0, 0, 0);
        float xv[8];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            xv[2 * k] = x[v[k].x];
            xv[2 * k + 1] = x[v[k].y];
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float w0 = __uint_as_float(v[k].z), w1 = __uint_as_float(v[k].w);
            acc += w0 * xv[2 * k] + w1 * xv[2 * k + 1];
            d += w0 + w1;
        }
    }
}
__device__ __forceinline__ void sell_dot(const MKLevel<double> &L, const int4 m, int lane,
                                         const double *__restrict__ x, double &acc, double &d) {
    const size_t base = (size_t)m.w * 32 + lane;
    for (int q = 0; q < m.z; q += 4) {
        int2 c[4];
        double2 w[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            c[k] = q + k < m.z ? __ldg(L.ellc + base + (size_t)(q + k) * 32) : make_int2(0, 0);
            w[k] = q + k < m.z ? __ldg(L.ellw + base + (size_t)(q + k) * 32) : make_double2(0.0, 0.0);
        }
        double xv[8];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            xv[2 * k] = x[c[k].x];
            xv[2 * k + 1] = x[c[k].y];
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            acc += w[k].x * xv[2 * k] + w[k].y * xv[2 * k + 1];
            d += w[k].x + w[k].y;
        }
    }
}
// pairs nst.. of a slice (the pairs that were not staged)
template <class T>
__device__ __forceinline__ void sell_rest(const MKLevel<T> &L, int4 m, int lane, int nst, const T *__restrict__ x,
                                          T xi, bool res, T &acc, T &d) {
    if (m.z <= nst) return;
    int4 m2 = m;
    m2.w += nst;
    m2.z -= nst;
    if (res) sell_res(L, m2, lane, x, xi, acc);
    else sell_dot(L, m2, lane, x, acc, d);
}

// residual form: acc += sum w (x[col] - xi)  (differences: no cancellation)
__device__ __forceinline__ void sell_res(const MKLevel<float> &L, const int4 m, int lane, const float *__restrict__ x,
                                         float xi, float &acc) {
    const uint4 *__restrict__ p = L.ell32 + (size_t)m.w * 32 + lane;
    for (int q = 0; q < m.z; q += 4) {
        uint4 v[4];
#pragma unroll
        for (int k = 0; k < 4; k++) v[k] = q + k < m.z ? __ldg(p + (size_t)(q + k) * 32) : make_uint4(0, 0, 0, 0);
        float xv[8];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            xv[2 * k] = x[v[k].x];
            xv[2 * k + 1] = x[v[k].y];
        }
#pragma unroll
        for (int k = 0; k < 4; k++)
            acc += __uint_as_float(v[k].z) * (xv[2 * k] - xi) + __uint_as_float(v[k].w) * (xv[2 * k + 1] - xi);
    }
}
__device__ __forceinline__ void sell_res(const MKLevel<double> &L, const int4 m, int lane,
                                         const double *__restrict__ x, double xi, double &acc) {
    const size_t base = (size_t)m.w * 32 + lane;
    for (int q = 0; q < m.z; q += 4) {
        int2 c[4];
        double2 w[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            c[k] = q + k < m.z ? __ldg(L.ellc + base + (size_t)(q + k) * 32) : make_int2(0, 0);
            w[k] = q + k < m.z ? __ldg(L.ellw + base + (size_t)(q + k) * 32) : make_double2(0.0, 0.0);
        }
        double xv[8];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            xv[2 * k] = x[c[k].x];
            xv[2 * k + 1] = x[c[k].y];
        }
#pragma unroll
        for (int k = 0; k < 4; k++) acc += w[k].x * (xv[2 * k] - xi) + w[k].y * (xv[2 * k + 1] - xi);
    }
}

enum : int32_t {
    OP_SWEEP = 0,     // level, colour a (all blocks)
    OP_SWEEP_RUN,     // level, colours a..b-1 (single block, __syncthreads between colours)
    OP_RESID,         // r = b - A x; a >= 0: also save x, r into slot a (recombination)
    OP_RESTRICT,      // b^c = mu P^T r, x^c = 0
    OP_ZERO,          // x = 0 (coarsest solved by sweeps)
    OP_COARSE,        // x = M^-1 b (dense coarsest, FP64 arithmetic)
    OP_PROLONG,       // x += P x^c
    OP_RECOMB_DOTS,   // partial dot products, theta = a
    OP_RECOMB_APPLY,  // alpha from the partials, y = x + sum alpha_i (x_i - x)
    OP_MEAN_PART,     // partial sums of x (cycle precision)
    OP_MEAN_APPLY,    // x -= mean
    OP_IR_PREP,       // b32 = (float) r64, x32 = 0
    OP_IR_UPDATE,     // x64 += (double) x32
    OP_MEAN64_PART,   // partial sums of x64
    OP_MEAN64_APPLY,  // x64 -= mean
    OP_RES64,         // r64 = b64 - A x64 (FP64) and partial sums of r64^2
    OP_NORM64_FIN,    // out[0] = sum of the partials
    OP_SWEEP_SMEM,    // level, a = sweeps: whole sweeps from shared memory (single block)
    // union of several graphs: level-1 projection and norms per graph
    OP_GMEAN_PART,    // gsum[g] = mean of x over graph g (cycle precision, level 1)
    OP_GMEAN_APPLY,   // x -= gsum[graph of the row]
    OP_GMEAN64_PART,  // same on the FP64 iterate
    OP_GMEAN64_APPLY,
    OP_GNORM64,       // gnorm[g] = ||r64 on graph g||^2
    OP_TAIL_PRE,      // tail rows: r_i = b_i + sum over neighbours outside the tail (grid)
    OP_TAIL_RUN,      // tail colours in order from shared memory (single block)
    // a level followed by elimination (Sec. 3.2): no relaxation, gamma = 1
    OP_ELIM_RESTRICT, // b^c_c = r_c + sum over eliminated f of w_cf r_f / a_ff, x^c = 0
    OP_ELIM_PROLONG,  // x_c += x^c_c on the kept rows
    OP_ELIM_BACK,     // x_f = (b_f + sum_c w_fc x_c) / a_ff on the eliminated rows
};

constexpr int kEngSmem = 200 * 1024;  // dynamic shared memory of the engine block

// bytes the shared-memory sweep needs for a level: rp, col, w, x, b, colour bounds
template <class T>
__host__ __device__ __forceinline__ int64_t smem_bytes(int64_t n, int64_t nnz, int64_t ncol) {
    auto al = [](int64_t b) { return (b + 15) & ~int64_t(15); };
    return al(4 * (n + 1)) + al(4 * nnz) + al((int64_t)sizeof(T) * nnz) + 2 * al((int64_t)sizeof(T) * n) +
           al(16 * ncol);
}

struct Op {
    int32_t type, level, a, b, sb;
};

// colour count of a level is carried in the op (b) for the shared-memory sweep

template <class T>
struct EngineArgs {
    const Op *prog;
    int32_t begin, end;
    const MKLevel<T> *lv;
    MKLevel<double> L0;     // FP64 finest level (outer refinement / residual)
    T mu;
    double *part;           // gridDim * 8 partial sums
    double *alpha;          // 2 per level
    double *out;            // results
    unsigned int *bar;      // barrier: count, generation
    int32_t *err;
    unsigned long long *optime;  // optional per (level, op, single-block) time and count
    // union of several graphs (ngraphs > 1 only)
    int32_t ngraphs;
    const int64_t *gptr;     // level-1 natural node range of each graph
    const int32_t *iperm0;   // natural level-1 id -> permuted row
    const int32_t *gid0;     // graph of each permuted level-1 row
    double *gsum, *gnorm;    // per-graph means, ||r64||^2
    int32_t nlev;            // levels in lv (the first kLvShared are copied to shared memory)
};

// Level descriptors kept in each block's shared memory for the whole launch: an op
// then reads its level's pointers and sizes from shared memory instead of
// starting with dependent loads from global memory.
constexpr int kLvShared = 20;
template <class T>
__device__ __forceinline__ const MKLevel<T> &lvl(const EngineArgs<T> &a, const MKLevel<T> *s, int l) {
    return l < kLvShared ? s[l] : a.lv[l];
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------
// grid barrier (bounded spin)
// ---------------------------------------------------------------------------

// Thread index of a grid-wide op executed by nb blocks (this one is bid) that
// deals work out in chunks of 32 consecutive items, consecutive chunks going to
// consecutive blocks: a warp's items stay contiguous (coalesced) while even a
// small op spreads over every SM.  (tid >> 5) is the matching warp index.
__device__ __forceinline__ int64_t spread_tid(int bid, int nb) {
    return ((int64_t)(threadIdx.x >> 5) * nb + bid) * 32 + (threadIdx.x & 31);
}

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Counting grid barrier: bar[0] counts every block's arrivals over the whole
// launch and must be zero when the launch starts (the host clears it before
// each launch).  Barrier number e (1, 2, ...) completes when bar[0] reaches
// e * gridDim.x, so no block resets anything and a single atomic per block
// and barrier suffices.  Ordering: the block's __syncthreads puts its threads'
// writes before thread 0's arrival, a release reduction (cumulative at GPU
// scope); thread 0 polls with acquire loads, and the closing __syncthreads
// puts that acquire before every thread's next access.  On GB300 this pair
// costs about a microsecond less per barrier inside the engine than full
// fences around a relaxed atomic.  The spin is bounded: after kMaxSpins polls
// (or when another block has given up) it sets the error word and every block
// returns.

__device__ __forceinline__ void red_release_gpu(unsigned int *p) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
}

// The barrier comes in two halves, so that a block can issue work that does
// not depend on the other blocks (loads of the next op's constant data)
// between its arrival and its wait.
__device__ __forceinline__ void grid_arrive(unsigned int *bar, unsigned int &epoch) {
    __syncthreads();
    if (threadIdx.x == 0) {
        ++epoch;
        red_release_gpu(bar);
    }
}
// grid_wait: false when the wait gave up
__device__ __forceinline__ bool grid_wait(unsigned int *bar, int32_t *err, unsigned int epoch) {
    __shared__ int bad;
    if (threadIdx.x == 0) {
        bad = 0;
        const unsigned int target = epoch * gridDim.x;
        long long spins = 0;
        while (ld_acquire_gpu(bar) < target) {
            if ((++spins & 255) == 0) {
                if (*(volatile int32_t *)err) { bad = 1; break; }
                if (spins > kMaxSpins) { atomicExch(err, 1); bad = 1; break; }
            }
        }
    }
    __syncthreads();
    return bad == 0;
}
__device__ __forceinline__ bool grid_sync(unsigned int *bar, int32_t *err, unsigned int &epoch) {
    grid_arrive(bar, epoch);
    return grid_wait(bar, err, epoch);
}

// Block sums of N values of type A, result in every thread.  The cross-warp
// step runs in warp 0 alone: with FP64 (1/64 of the FP32 rate on this GPU)
// a sum done by every thread would cost 32 adds per thread.
template <class A, int N>
__device__ __forceinline__ void block_sum_n(A (&v)[N]) {
    __shared__ A sh[N][32];
    __shared__ A res[N];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
#pragma unroll
    for (int k = 0; k < N; k++) v[k] = warp_allsum(v[k]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < N; k++) sh[k][warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < N; k++) {
            A t = lane < nw ? sh[k][lane] : A(0);
            t = warp_allsum(t);
            if (lane == 0) res[k] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; k++) v[k] = res[k];
    __syncthreads();
}

template <class A>
__device__ __forceinline__ A block_sum(A v) {
    A t[1] = {v};
    block_sum_n<A, 1>(t);
    return t[0];
}

template <class T>
__device__ __forceinline__ double block_sum_d(double v) { return block_sum<double>(v); }

// out[k] = sum of the nb block partials at slots k0 .. k0+N-1 (warp 0 sums, fixed
// order; the result is broadcast to every thread)
template <int N>
__device__ __forceinline__ void sum_partials_n(const double *part, int nb, int k0, double (&out)[N]) {
    __shared__ double res[N];
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        // all N sums in one pass over the partials, so that their loads are in
        // flight together; each sum still adds its partials in block order
        const int lane = threadIdx.x & 31;
        double t[N];
#pragma unroll
        for (int k = 0; k < N; k++) t[k] = 0.0;
#pragma unroll 4
        for (int b = lane; b < nb; b += 32) {
#pragma unroll
            for (int k = 0; k < N; k++) t[k] += part[(int64_t)b * 8 + k0 + k];
        }
#pragma unroll
        for (int k = 0; k < N; k++) {
            const double v = warp_allsum(t[k]);
            if (lane == 0) res[k] = v;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; k++) out[k] = res[k];
    __syncthreads();
}

__device__ __forceinline__ double sum_partials(const double *part, int nb, int k) {
    double o[1];
    sum_partials_n<1>(part, nb, k, o);
    return o[0];
}

template <class T>
inline MKLevel<T> describe(lamg_ctx *h, int l, LevelVecs<T> &v, const T *w) {
    const SolveLevel &V = h->lv[l];
    MKLevel<T> d{};
    d.n = V.n;
    d.nc = (l + 1 < h->L) ? h->lv[l + 1].n : 0;
    d.rp = V.rp.get();
    d.col = V.col.get();
    d.w = w;
    d.cb = V.cb_dev.get();
    d.wrows = V.wrows.get();
    d.brows = V.brows.get();
    d.nw = V.nw;
    d.nb = V.nb;
    d.pagg = V.pagg.get();
    d.mptr = V.mptr.get();
    d.mlist = V.mlist.get();
    d.wagg = V.wagg.get();
    d.bagg = V.bagg.get();
    d.nwagg = V.nwagg;
    d.nbagg = V.nbagg;
    d.x = v.x.get();
    d.b = v.b.get();
    d.r = v.r.get();
    d.xs0 = v.xs0.get();
    d.xs1 = v.xs1.get();
    d.rs0 = v.rs0.get();
    d.rs1 = v.rs1.get();
    d.minv = V.minv.get();
    d.tt0 = V.tt0;
    d.tn = V.tn;
    d.tnc = V.tnc;
    d.tnnz = (int32_t)V.tnnz;
    d.trp = V.trp.get();
    d.tcol = V.tcol.get();
    d.tcb = V.tcb.get();
    d.trq = V.trq.get();
    d.tmaxq = V.tmaxq;
    if constexpr (sizeof(T) == 8) {
        d.tw = (const T *)V.tw64.get();
        d.tdeg = (const T *)V.tdeg64.get();
        d.ed = (const T *)V.ed64.get();
    } else {
        d.tw = (const T *)V.tw32.get();
        d.tdeg = (const T *)V.tdeg32.get();
        d.ed = (const T *)V.ed32.get();
    }
    d.ecx = V.ecx.get();
    d.nsl = V.nsl;
    d.csl = V.csl_dev.get();
    d.sl = V.sl.get();
    d.ell32 = V.ell32.get();
    d.ellc = V.ellc.get();
    d.ellw = V.ellw64.get();
    return d;
}

// shared memory of the tail run: x, s, d (T each), trp, tcb, trq, the chunk
// partial sums of one colour, and (when it fits) the tail block's local CSR
template <class T>
__host__ __device__ __forceinline__ int64_t tail_smem_base(int64_t tn, int64_t tnc, int64_t tmaxq) {
    auto al = [](int64_t b) { return (b + 15) & ~int64_t(15); };
    return 3 * al((int64_t)sizeof(T) * tn) + 2 * al(4 * (tn + 1)) + al(4 * (tnc + 1)) + al((int64_t)sizeof(T) * tmaxq);
}
template <class T>
__host__ __device__ __forceinline__ int64_t tail_smem_csr(int64_t tnnz) {
    auto al = [](int64_t b) { return (b + 15) & ~int64_t(15); };
    return al(4 * tnnz) + al((int64_t)sizeof(T) * tnnz);
}

}  // namespace lamg
