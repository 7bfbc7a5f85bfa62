// cycle.cu -- the cycle engine: one persistent cooperative kernel per cycle
// (or per FP32-in-FP64 refinement step) that interprets a program of ops
// built on the host by replaying the cycle schedule of Sec. 4.2 / Fig. 4.2
// (Livne & Brandt, arXiv 1108.1310).
//
// LAMG's cycles visit the coarse levels many times (fractional cycle index
// up to 2, Eq. (4.1)), and multicolour Gauss-Seidel needs one dependent phase
// per colour, so a cycle is thousands of short dependent phases.  Launching
// them as separate kernels makes the cycle latency-bound.  Here every phase is
// an op executed by all blocks between grid barriers; ops of small levels (and
// runs of tiny colours) are flagged single-block and run by block 0 alone with
// __syncthreads between them, costing one grid barrier per run.
//
// The grid barrier spins with a bounded count; when it runs out the kernel
// sets an error word and every block returns (the host reports
// LAMG_ERR_TIMEOUT).  The launch is cooperative, so all blocks are resident.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "engine.cuh"

namespace lamg {

static_assert((kEngThreads / 32) * kSellStageBytes <= kEngSmem, "sliced-ELL staging must fit the engine's shared memory");

// ---------------------------------------------------------------------------
// ops; (bid, nb) = this block's index among the nb blocks executing the op
// ---------------------------------------------------------------------------

template <class T>
__device__ __forceinline__ void sweep_colour(const MKLevel<T> &L, int c, int bid, int nb, SellPre &pre) {
    const int32_t t1 = L.cb[4 * c + 1], t2 = L.cb[4 * c + 2], t3 = L.cb[4 * c + 3];
    const int64_t nthr = (int64_t)nb * blockDim.x, tid = spread_tid(bid, nb);
    const int64_t nwarp = nthr >> 5, wid = tid >> 5;
    const int lane = threadIdx.x & 31;
    // thread-tier rows: one warp per slice of 32 rows (sliced ELL, 16-byte loads)
    if constexpr (sizeof(T) == 4) {
        // FP32: the next slice's first pairs are staged in shared memory while this
        // slice's gathers are in flight
        sell_walk32(L, L.csl[c] + wid, L.csl[c + 1], nwarp, pre, [&](const int4 m, const uint4 *st, int nst) {
            // b does not depend on x: its load goes out before the gathers
            const int32_t i = m.x + (lane < m.y ? lane : 0);
            const float bi = L.b[i];
            float acc = 0.0f, d = 0.0f;
            sell_row32(st, nst, L.x, 0.0f, false, acc, d);
            sell_rest(L, m, lane, nst, L.x, 0.0f, false, acc, d);
            if (lane < m.y && d != 0.0f) L.x[i] = (bi + acc) / d;
        });
    } else {
        for (int64_t k = L.csl[c] + wid; k < L.csl[c + 1]; k += nwarp) {
            const int4 m = L.sl[k];
            T acc = T(0), d = T(0);
            sell_dot(L, m, lane, L.x, acc, d);
            const int32_t i = m.x + lane;
            if (lane < m.y && d != T(0)) L.x[i] = (L.b[i] + acc) / d;
        }
    }
    for (int64_t i = t1 + wid; i < t2; i += nwarp) gs_row<M_WARP, T>((int32_t)i, L.rp, L.col, L.w, L.b, L.x);
    for (int64_t i = t2 + bid; i < t3; i += nb) gs_row<M_BLK, T>((int32_t)i, L.rp, L.col, L.w, L.b, L.x);
}

template <class T>
__device__ __forceinline__ void residual(const MKLevel<T> &L, const T *b, const T *x, T *r, T *xs, T *rs, int bid,
                                         int nb, SellPre &pre) {
    const int64_t nthr = (int64_t)nb * blockDim.x, tid = spread_tid(bid, nb);
    const int64_t nwarp = nthr >> 5, wid = tid >> 5;
    const int lane = threadIdx.x & 31;
    // thread-tier rows: one warp per slice of 32 rows (sliced ELL, 16-byte loads)
    if constexpr (sizeof(T) == 4) {
        // FP32: the next slice's first pairs are staged in shared memory while this
        // slice's gathers are in flight
        sell_walk32(L, wid, L.nsl, nwarp, pre, [&](const int4 m, const uint4 *st, int nst) {
            const int32_t i = m.x + (lane < m.y ? lane : 0);
            const float xi = x[i], bi = b[i];
            float acc = 0.0f, dummy = 0.0f;
            sell_row32(st, nst, x, xi, true, acc, dummy);
            sell_rest(L, m, lane, nst, x, xi, true, acc, dummy);
            if (lane < m.y) {
                const float ri = bi + acc;
                r[i] = ri;
                if (xs) { xs[i] = xi; rs[i] = ri; }
            }
        });
    } else {
        for (int64_t k = wid; k < L.nsl; k += nwarp) {
            const int4 m = L.sl[k];
            const int32_t i = m.x + (lane < m.y ? lane : 0);
            const T xi = x[i];
            T acc = T(0);
            sell_res(L, m, lane, x, xi, acc);
            if (lane < m.y) {
                const T ri = b[i] + acc;
                r[i] = ri;
                if (xs) { xs[i] = xi; rs[i] = ri; }
            }
        }
    }
    for (int64_t k = wid; k < L.nw; k += nwarp) {
        const int32_t ii = L.wrows[k];
        resid_row<M_WARP, T>(ii, L.rp, L.col, L.w, b, x, r);
        if (xs && (threadIdx.x & 31) == 0) { xs[ii] = x[ii]; rs[ii] = r[ii]; }
    }
    for (int64_t k = bid; k < L.nb; k += nb) {
        const int32_t ii = L.brows[k];
        resid_row<M_BLK, T>(ii, L.rp, L.col, L.w, b, x, r);
        if (xs && threadIdx.x == 0) { xs[ii] = x[ii]; rs[ii] = r[ii]; }
    }
}

template <class T>
__device__ __forceinline__ void restrict_op(const MKLevel<T> &F, const MKLevel<T> &C, T mu, int bid, int nb) {
    const int64_t nthr = (int64_t)nb * blockDim.x, tid = spread_tid(bid, nb);
    for (int64_t J = tid; J < C.n; J += nthr) {
        const int32_t jj = (int32_t)J;
        C.x[jj] = T(0);
        if (F.mptr[jj + 1] - F.mptr[jj] > kLongRow) continue;
        restrict_row<M_THR, T>(jj, F.mptr, F.mlist, F.r, mu, C.b);
    }
    const int64_t nwarp = nthr >> 5, wid = tid >> 5;
    for (int64_t k = wid; k < F.nwagg; k += nwarp) restrict_row<M_WARP, T>(F.wagg[k], F.mptr, F.mlist, F.r, mu, C.b);
    for (int64_t k = bid; k < F.nbagg; k += nb) restrict_row<M_BLK, T>(F.bagg[k], F.mptr, F.mlist, F.r, mu, C.b);
}

// kept row i of a level followed by elimination (Sec. 3.2): b^c = r_i + sum over
// its eliminated neighbours f of w_if r_f / a_ff; x^c = 0
template <int M, class T>
__device__ __forceinline__ void elim_restrict_row(int32_t i, const MKLevel<T> &L, const MKLevel<T> &C) {
    const int32_t e = L.rp[i + 1];
    const int st = sstride<M>();
    T acc = T(0), dummy = T(0);
    for (int32_t j = L.rp[i] + slane<M>(); j < e; j += st) {
        const int32_t f = L.col[j];
        if (L.ecx[f] < 0) acc += L.w[j] * L.r[f] / L.ed[f];
    }
    reduce2<M>(acc, dummy);
    if (slane<M>() == 0) {
        const int32_t c = L.ecx[i];
        C.b[c] = L.r[i] + acc;
        C.x[c] = T(0);
    }
}

// tail row i: r_i = b_i + sum of w_iv x_v over v < tt0 (outside the tail)
template <int M, class T>
__device__ __forceinline__ void tail_pre_row(int32_t i, const MKLevel<T> &L) {
    const int32_t e = L.rp[i + 1], t0 = L.tt0;
    const int st = sstride<M>();
    T acc = T(0), dummy = T(0);
    int32_t j = L.rp[i] + slane<M>();
    for (; j + 3 * st < e; j += 4 * st) {
        int32_t c[4];
        T wv[4], xv[4];
#pragma unroll
        for (int k = 0; k < 4; k++) c[k] = L.col[j + k * st];
#pragma unroll
        for (int k = 0; k < 4; k++) wv[k] = L.w[j + k * st];
#pragma unroll
        for (int k = 0; k < 4; k++) xv[k] = c[k] < t0 ? L.x[c[k]] : T(0);
#pragma unroll
        for (int k = 0; k < 4; k++) acc += wv[k] * xv[k];
    }
    for (; j < e; j += st) {
        const int32_t cj = L.col[j];
        if (cj < t0) acc += L.w[j] * L.x[cj];
    }
    reduce2<M>(acc, dummy);
    if (slane<M>() == 0) L.r[i] = L.b[i] + acc;
}

template <class T>
__device__ void exec_op(const EngineArgs<T> &a, const MKLevel<T> *slv, const Op &op, int bid, int nb, SellPre &pre) {
    const int64_t nthr = (int64_t)nb * blockDim.x, tid = spread_tid(bid, nb);
    const MKLevel<T> &L = lvl(a, slv, op.level);
    switch (op.type) {
        case OP_SWEEP:
            sweep_colour<T>(L, op.a, bid, nb, pre);
            break;
        case OP_SWEEP_RUN:
            for (int c = op.a; c < op.b; c++) {
                sweep_colour<T>(L, c, 0, 1, pre);
                if constexpr (sizeof(T) == 4) {
                    // the next colour's first slices are staged before the block syncs
                    if (c + 1 < op.b)
                        sell_prestage(L, L.csl[c + 1] + (threadIdx.x >> 5), L.csl[c + 2], blockDim.x >> 5, pre);
                }
                __syncthreads();
            }
            break;
        case OP_RESID: {
            T *xs = op.a == 0 ? L.xs0 : (op.a == 1 ? L.xs1 : nullptr);
            T *rs = op.a == 0 ? L.rs0 : (op.a == 1 ? L.rs1 : nullptr);
            residual<T>(L, L.b, L.x, L.r, xs, rs, bid, nb, pre);
            break;
        }
        case OP_RESTRICT:
            restrict_op<T>(L, lvl(a, slv, op.level + 1), a.mu, bid, nb);
            break;
        case OP_ZERO:
            for (int64_t i = tid; i < L.n; i += nthr) L.x[i] = T(0);
            break;
        case OP_COARSE: {
            const int64_t nwarp = nthr >> 5, wid = tid >> 5;
            const int lane = threadIdx.x & 31;
            for (int64_t i = wid; i < L.n; i += nwarp) {
                double acc = 0.0;
                for (int32_t j = lane; j < L.n; j += 32) acc += L.minv[i * L.n + j] * (double)L.b[j];
                acc = warp_allsum(acc);
                if (lane == 0) L.x[i] = (T)acc;
            }
            break;
        }
        case OP_PROLONG: {
            const MKLevel<T> &C = lvl(a, slv, op.level + 1);
            for (int64_t i = tid; i < L.n; i += nthr) L.x[i] += C.x[L.pagg[i]];
            break;
        }
        case OP_RECOMB_DOTS: {
            // in the cycle precision per thread and block; block partials in FP64
            T v[5] = {T(0), T(0), T(0), T(0), T(0)};  // G00, G01, G11, h0, h1
            for (int64_t i = tid; i < L.n; i += nthr) {
                const T ri = L.r[i];
                const T d0 = ri - L.rs0[i];
                v[0] += d0 * d0;
                v[3] += ri * d0;
                if (op.a == 2) {
                    const T d1 = ri - L.rs1[i];
                    v[1] += d0 * d1;
                    v[2] += d1 * d1;
                    v[4] += ri * d1;
                }
            }
            block_sum_n<T, 5>(v);
            if (threadIdx.x < 5) a.part[(int64_t)bid * 8 + threadIdx.x] = (double)v[threadIdx.x];
            break;
        }
        case OP_RECOMB_APPLY: {
            // Eq. (3.13): alpha minimises ||b - A y||_2; normal equations of size theta
            double G[5];
            sum_partials_n<5>(a.part, nb, 0, G);
            const double G00 = G[0], G01 = G[1], G11 = G[2], h0 = G[3], h1 = G[4];
            double a0 = 0.0, a1 = 0.0;
            if (op.a == 1) {
                if (G00 > 0.0) a0 = h0 / G00;
            } else {
                const double det = G00 * G11 - G01 * G01;
                if (det > 1e-14 * G00 * G11 && det > 0.0) {
                    a0 = (h0 * G11 - G01 * h1) / det;
                    a1 = (G00 * h1 - G01 * h0) / det;
                } else if (G00 > 0.0) {
                    a0 = h0 / G00;
                }
            }
            const T ta0 = (T)a0, ta1 = (T)a1;
            for (int64_t i = tid; i < L.n; i += nthr) {
                const T xi = L.x[i];
                T y = xi + ta0 * (L.xs0[i] - xi);
                if (op.a == 2) y += ta1 * (L.xs1[i] - xi);
                L.x[i] = y;
            }
            break;
        }
        case OP_MEAN_PART: {
            T v = T(0);
            for (int64_t i = tid; i < L.n; i += nthr) v += L.x[i];
            v = block_sum<T>(v);
            if (threadIdx.x == 0) a.part[(int64_t)bid * 8] = (double)v;
            break;
        }
        case OP_MEAN_APPLY: {
            const T m = (T)(sum_partials(a.part, nb, 0) / (double)L.n);
            for (int64_t i = tid; i < L.n; i += nthr) L.x[i] -= m;
            break;
        }
        case OP_IR_PREP:
            for (int64_t i = tid; i < L.n; i += nthr) {
                L.b[i] = (T)a.L0.r[i];
                L.x[i] = T(0);
            }
            break;
        case OP_IR_UPDATE:
            for (int64_t i = tid; i < L.n; i += nthr) a.L0.x[i] += (double)L.x[i];
            break;
        case OP_MEAN64_PART: {
            double v = 0.0;
            for (int64_t i = tid; i < a.L0.n; i += nthr) v += a.L0.x[i];
            v = block_sum_d<double>(v);
            if (threadIdx.x == 0) a.part[(int64_t)bid * 8] = v;
            break;
        }
        case OP_MEAN64_APPLY: {
            const double m = sum_partials(a.part, nb, 0) / (double)a.L0.n;
            for (int64_t i = tid; i < a.L0.n; i += nthr) a.L0.x[i] -= m;
            break;
        }
        case OP_RES64: {
            SellPre none{};
            residual<double>(a.L0, a.L0.b, a.L0.x, a.L0.r, nullptr, nullptr, bid, nb, none);
            // the residual entries this block wrote are not known here; sum squares after a barrier
            break;
        }
        case OP_NORM64_FIN: {
            double v = 0.0;
            for (int64_t i = tid; i < a.L0.n; i += nthr) {
                const double t = a.L0.r[i];
                v += t * t;
            }
            v = block_sum_d<double>(v);
            if (threadIdx.x == 0) a.part[(int64_t)bid * 8 + 5] = v;
            break;
        }
        case OP_GMEAN_PART:
        case OP_GMEAN64_PART:
        case OP_GNORM64:
            // one block per graph; natural ids of the graph are contiguous
            for (int32_t g = bid; g < a.ngraphs; g += nb) {
                const int64_t s0 = a.gptr[g], e0 = a.gptr[g + 1];
                double v = 0.0;
                if (op.type == OP_GMEAN_PART) {
                    T t = T(0);
                    for (int64_t u = s0 + threadIdx.x; u < e0; u += blockDim.x) t += L.x[a.iperm0[u]];
                    v = (double)block_sum<T>(t);
                } else {
                    for (int64_t u = s0 + threadIdx.x; u < e0; u += blockDim.x) {
                        const int32_t i = a.iperm0[u];
                        v += op.type == OP_GMEAN64_PART ? a.L0.x[i] : a.L0.r[i] * a.L0.r[i];
                    }
                    v = block_sum<double>(v);
                }
                if (threadIdx.x == 0) {
                    if (op.type == OP_GNORM64) a.gnorm[g] = v;
                    else a.gsum[g] = v / (double)(e0 - s0);
                }
            }
            break;
        case OP_GMEAN_APPLY:
            for (int64_t i = tid; i < L.n; i += nthr) L.x[i] -= (T)a.gsum[a.gid0[i]];
            break;
        case OP_GMEAN64_APPLY:
            for (int64_t i = tid; i < a.L0.n; i += nthr) a.L0.x[i] -= a.gsum[a.gid0[i]];
            break;
        case OP_ELIM_RESTRICT: {
            // the eliminated rows have degree <= 4: thread tier; warp/block-tier rows are kept rows
            const MKLevel<T> &C = lvl(a, slv, op.level + 1);
            for (int64_t i = tid; i < L.n; i += nthr) {
                const int32_t ii = (int32_t)i;
                if (L.ecx[ii] < 0 || L.rp[ii + 1] - L.rp[ii] > kLongRow) continue;
                elim_restrict_row<M_THR, T>(ii, L, C);
            }
            const int64_t nwarp = nthr >> 5, wid = tid >> 5;
            for (int64_t k = wid; k < L.nw; k += nwarp) {
                const int32_t ii = L.wrows[k];
                if (L.ecx[ii] >= 0) elim_restrict_row<M_WARP, T>(ii, L, C);
            }
            for (int64_t k = bid; k < L.nb; k += nb) {
                const int32_t ii = L.brows[k];
                if (L.ecx[ii] >= 0) elim_restrict_row<M_BLK, T>(ii, L, C);
            }
            break;
        }
        case OP_ELIM_PROLONG: {
            const MKLevel<T> &C = lvl(a, slv, op.level + 1);
            for (int64_t i = tid; i < L.n; i += nthr) {
                const int32_t c = L.ecx[i];
                if (c >= 0) L.x[i] += C.x[c];
            }
            break;
        }
        case OP_ELIM_BACK:
            // exact back-substitution x_f = (b_f + sum_c w_fc x_c) / a_ff (F is independent)
            for (int64_t i = tid; i < L.n; i += nthr) {
                if (L.ecx[i] >= 0) continue;
                T acc = L.b[i];
                for (int32_t j = L.rp[i]; j < L.rp[i + 1]; j++) acc += L.w[j] * L.x[L.col[j]];
                L.x[i] = acc / L.ed[i];
            }
            break;
        case OP_TAIL_PRE: {
            // r_i = b_i + sum of w_iv x_v over the neighbours v outside the tail; those
            // x_v do not change while the tail colours run (they come last in the order)
            const int32_t t0 = L.tt0, n = L.n;
            for (int32_t i = t0 + bid; i < n; i += nb) {
                if (L.rp[i + 1] - L.rp[i] <= kHugeSolve) continue;
                tail_pre_row<M_BLK, T>(i, L);
            }
            const int64_t nwarp = nthr >> 5, wid = tid >> 5;
            for (int64_t i = t0 + wid; i < n; i += nwarp) {
                if (L.rp[i + 1] - L.rp[i] > kHugeSolve) continue;
                tail_pre_row<M_WARP, T>((int32_t)i, L);
            }
            break;
        }
        case OP_TAIL_RUN: {
            // single block: x_i = (r_i + sum over tail neighbours) / a_ii, colour by colour.
            // Each colour's rows are cut into chunks of kTailChunk local entries spread over
            // all warps; the chunk sums of a row are then added in order (deterministic).
            extern __shared__ __align__(16) unsigned char smem[];
            auto al = [](int64_t v) { return (v + 15) & ~int64_t(15); };
            const int32_t tn = L.tn, tnc = L.tnc, t0 = L.tt0;
            unsigned char *p = smem;
            T *sx = (T *)p; p += al((int64_t)sizeof(T) * tn);
            T *ss = (T *)p; p += al((int64_t)sizeof(T) * tn);
            T *sd = (T *)p; p += al((int64_t)sizeof(T) * tn);
            int32_t *srp = (int32_t *)p; p += al(4 * (int64_t)(tn + 1));
            int32_t *srq = (int32_t *)p; p += al(4 * (int64_t)(tn + 1));
            int32_t *scb = (int32_t *)p; p += al(4 * (int64_t)(tnc + 1));
            T *cpart = (T *)p; p += al((int64_t)sizeof(T) * L.tmaxq);
            const int32_t *tcol = L.tcol;
            const T *tw = L.tw;
            if (op.a) {  // the local CSR fits: stage it too
                int32_t *c2 = (int32_t *)p; p += al(4 * (int64_t)L.tnnz);
                T *w2 = (T *)p;
                for (int32_t k = threadIdx.x; k < L.tnnz; k += blockDim.x) { c2[k] = L.tcol[k]; w2[k] = L.tw[k]; }
                tcol = c2;
                tw = w2;
            }
            for (int32_t k = threadIdx.x; k < tn; k += blockDim.x) {
                sx[k] = L.x[t0 + k];
                ss[k] = L.r[t0 + k];
                sd[k] = L.tdeg[k];
            }
            for (int32_t k = threadIdx.x; k <= tn; k += blockDim.x) { srp[k] = L.trp[k]; srq[k] = L.trq[k]; }
            for (int32_t k = threadIdx.x; k <= tnc; k += blockDim.x) scb[k] = L.tcb[k];
            __syncthreads();
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (int)(blockDim.x >> 5);
            // entry range [k0, k1) of chunk q of the colour with rows [R0, R1)
            auto chunk = [&](int32_t q, int32_t R0, int32_t R1, int32_t &k0, int32_t &k1) {
                int32_t lo = R0, hi = R1 - 1;   // last row of the colour whose first chunk is <= q
                while (lo < hi) {
                    const int32_t mid = (lo + hi + 1) >> 1;
                    if (srq[mid] <= q) lo = mid; else hi = mid - 1;
                }
                k0 = srp[lo] + (q - srq[lo]) * kTailChunk;
                k1 = min(k0 + kTailChunk, srp[lo + 1]);
            };
            // the entries (column, weight) of this warp's first chunk of the next colour are
            // loaded while the current colour finishes (they do not depend on x)
            constexpr int kPer = kTailChunk / 32;
            int32_t pc[kPer];
            T pw[kPer];
            int32_t pk0 = 0, pk1 = 0;
            auto prefetch = [&](int32_t c) {
                pk0 = pk1 = 0;
                if (c >= tnc) return;
                const int32_t R0 = scb[c], R1 = scb[c + 1], q = srq[R0] + warp;
                if (q >= srq[R1]) return;
                chunk(q, R0, R1, pk0, pk1);
#pragma unroll
                for (int m = 0; m < kPer; m++) {
                    const int32_t k = pk0 + lane + 32 * m;
                    pc[m] = k < pk1 ? tcol[k] : 0;
                    pw[m] = k < pk1 ? tw[k] : T(0);
                }
            };
            prefetch(0);
            for (int32_t c = 0; c < tnc; c++) {
                const int32_t R0 = scb[c], R1 = scb[c + 1], Q0 = srq[R0], Q1 = srq[R1];
                if (Q0 + warp < Q1) {   // the prefetched first chunk
                    T acc = T(0);
#pragma unroll
                    for (int m = 0; m < kPer; m++) acc += pw[m] * sx[pc[m]];
                    acc = warp_allsum(acc);
                    if (lane == 0) cpart[warp] = acc;
                }
                for (int32_t q = Q0 + warp + nw; q < Q1; q += nw) {
                    int32_t k0, k1;
                    chunk(q, R0, R1, k0, k1);
                    T acc = T(0);
#pragma unroll 4
                    for (int32_t k = k0 + lane; k < k1; k += 32) acc += tw[k] * sx[tcol[k]];
                    acc = warp_allsum(acc);
                    if (lane == 0) cpart[q - Q0] = acc;
                }
                prefetch(c + 1);
                __syncthreads();
                for (int32_t li = R0 + threadIdx.x; li < R1; li += blockDim.x) {
                    T acc = T(0);
                    for (int32_t q = srq[li]; q < srq[li + 1]; q++) acc += cpart[q - Q0];
                    if (sd[li] != T(0)) sx[li] = (ss[li] + acc) / sd[li];
                }
                __syncthreads();
            }
            for (int32_t k = threadIdx.x; k < tn; k += blockDim.x) L.x[t0 + k] = sx[k];
            break;
        }
        case OP_SWEEP_SMEM: {
            // single block: stage the level, run a sweeps of all b colours, write x back
            extern __shared__ __align__(16) unsigned char smem[];
            const int32_t n = L.n, nnz = L.rp[n], nc = op.b;
            auto al = [](int64_t v) { return (v + 15) & ~int64_t(15); };
            unsigned char *p = smem;
            int32_t *srp = (int32_t *)p; p += al(4 * (int64_t)(n + 1));
            int32_t *scol = (int32_t *)p; p += al(4 * (int64_t)nnz);
            T *sw = (T *)p; p += al((int64_t)sizeof(T) * nnz);
            T *sx = (T *)p; p += al((int64_t)sizeof(T) * n);
            T *sbv = (T *)p; p += al((int64_t)sizeof(T) * n);
            int32_t *scb = (int32_t *)p;
            for (int32_t k = threadIdx.x; k <= n; k += blockDim.x) srp[k] = L.rp[k];
            for (int32_t k = threadIdx.x; k < nnz; k += blockDim.x) { scol[k] = L.col[k]; sw[k] = L.w[k]; }
            for (int32_t k = threadIdx.x; k < n; k += blockDim.x) { sx[k] = L.x[k]; sbv[k] = L.b[k]; }
            for (int32_t k = threadIdx.x; k < 4 * nc; k += blockDim.x) scb[k] = L.cb[k];
            __syncthreads();
            const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
            for (int rep = 0; rep < op.a; rep++)
                for (int32_t c = 0; c < nc; c++) {
                    const int32_t t0 = scb[4 * c], t1 = scb[4 * c + 1], t2 = scb[4 * c + 2], t3 = scb[4 * c + 3];
                    // long rows: one warp each (shared-memory gathers are short; rows of a
                    // colour proceed in parallel instead of one block-wide row at a time)
                    for (int32_t i = t0 + threadIdx.x; i < t1; i += blockDim.x) gs_row<M_THR, T>(i, srp, scol, sw, sbv, sx);
                    for (int32_t i = t1 + warp; i < t3; i += nwarp) gs_row<M_WARP, T>(i, srp, scol, sw, sbv, sx);
                    __syncthreads();
                }
            for (int32_t k = threadIdx.x; k < n; k += blockDim.x) L.x[k] = sx[k];
            break;
        }
        default:
            break;
    }
}

// Stage this warp's first slice of op `nx` (run by nb blocks, this one bid),
// for the sliced-ELL walks that begin the FP32 sweep and residual ops.
template <class T>
__device__ __forceinline__ void prestage_op(const EngineArgs<T> &a, const MKLevel<T> *slv, const Op &nx, int bid,
                                            int nb, SellPre &pre) {
    if constexpr (sizeof(T) == 4) {
        const int64_t nwarp = ((int64_t)nb * blockDim.x) >> 5, wid = spread_tid(bid, nb) >> 5;
        if (nx.type == OP_SWEEP || (nx.type == OP_SWEEP_RUN && nx.a < nx.b)) {
            const MKLevel<T> &N = lvl(a, slv, nx.level);
            sell_prestage(N, N.csl[nx.a] + wid, N.csl[nx.a + 1], nwarp, pre);
        } else if (nx.type == OP_RESID) {
            const MKLevel<T> &N = lvl(a, slv, nx.level);
            sell_prestage(N, wid, N.nsl, nwarp, pre);
        }
    }
}

template <class T>
__global__ void __launch_bounds__(kEngThreads) k_engine(EngineArgs<T> a) {
    __shared__ MKLevel<T> slv[kLvShared];
    {
        static_assert(sizeof(MKLevel<T>) % 4 == 0, "level descriptors are copied as 4-byte words");
        const int words = min(a.nlev, kLvShared) * (int)(sizeof(MKLevel<T>) / 4);
        const int32_t *src = (const int32_t *)a.lv;
        for (int i = threadIdx.x; i < words; i += blockDim.x) ((int32_t *)slv)[i] = src[i];
        __syncthreads();
    }
    int32_t pc = a.begin;
    unsigned int epoch = 0;
    SellPre pre{};
    // the next op is read while the block waits in the barrier and carried over,
    // so that no op starts with a load of its own descriptor
    Op op = pc < a.end ? a.prog[pc] : Op{};
    while (pc < a.end) {
        const bool timed = a.optime && blockIdx.x == 0 && threadIdx.x == 0;
        const unsigned long long t0 = timed ? gtimer() : 0ull;
        if (op.sb) {
            int32_t q = pc;
            if (blockIdx.x == 0) {
                while (q < a.end && a.prog[q].sb) {
                    const int32_t t = a.prog[q].type;
                    exec_op<T>(a, slv, a.prog[q], 0, 1, pre);
                    // (ops that hold the level in shared memory may still be reading it)
                    if (q + 1 < a.end && a.prog[q + 1].sb && t != OP_TAIL_RUN && t != OP_SWEEP_SMEM)
                        prestage_op<T>(a, slv, a.prog[q + 1], 0, 1, pre);
                    __syncthreads();
                    q++;
                }
            } else {
                while (q < a.end && a.prog[q].sb) q++;
            }
            pc = q;
        } else {
            exec_op<T>(a, slv, op, blockIdx.x, gridDim.x, pre);
            pc++;
        }
        grid_arrive(a.bar, epoch);
        // stage this warp's first slice of the next op while the block waits
        Op nx{};
        if (pc < a.end) {
            nx = a.prog[pc];
            if (!nx.sb) prestage_op<T>(a, slv, nx, blockIdx.x, gridDim.x, pre);
            else if (blockIdx.x == 0) prestage_op<T>(a, slv, nx, 0, 1, pre);
        }
        if (!grid_wait(a.bar, a.err, epoch)) {
            cp_async_wait<0>();   // copies staged ahead land before the block leaves
            return;
        }
        if (timed) {
            const int key = (op.level * 32 + op.type) * 2 + (op.sb ? 1 : 0);
            a.optime[2 * key] += gtimer() - t0;
            a.optime[2 * key + 1] += 1;
        }
        op = nx;
    }
}

// Self-test of the grid barrier's bounded wait: every block except `held`
// (-1: none) enters one barrier.  With a block held back the others give up
// after kMaxSpins polls, set the error word and return; nothing faults.
__global__ void __launch_bounds__(kEngThreads) k_barrier_probe(unsigned int *bar, int32_t *err, int32_t held) {
    unsigned int epoch = 0;
    if ((int32_t)blockIdx.x == held) return;
    grid_sync(bar, err, epoch);
}

// ||r64||^2 from the per-block partials written by OP_NORM64_FIN
__global__ void k_engine_norm(const double *part, int nb, double *out) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[(int64_t)b * 8 + 5];
    v = block_sum_d<double>(v);
    if (threadIdx.x == 0) out[0] = v;
}

// ---------------------------------------------------------------------------
// Program builder (host): replays the cycle schedule of the oracle
// ---------------------------------------------------------------------------

struct Builder {
    lamg_ctx *h;
    int prec;            // 0 = FP64, 1 = FP32
    int adaptive;
    int groups;          // 0: one right-hand side; G >= 1: 4G interleaved columns
    std::vector<Op> prog;
    std::vector<int32_t> visits;

    // a level runs on block 0 alone when it is small and its sweep fits in shared memory
    // (with several columns: when its work times the column groups is small)
    bool level_sb(int l) const {
        const SolveLevel &V = h->lv[l];
        if (groups) return (V.nnz + V.n) * groups <= kSBWork;
        return V.nnz + V.n <= sb_work(h->opt, prec);
    }
    void emit(int type, int level, int a, int b, bool sb) { prog.push_back(Op{type, level, a, b, sb ? 1 : 0}); }

    // `count` consecutive sweeps of level l
    void sweeps(int l, int count) {
        if (count <= 0) return;
        const SolveLevel &V = h->lv[l];
        const int nc = (int)V.cb.size() / 4;
        if (level_sb(l) && !groups) {
            const int64_t need = prec == 0 ? smem_bytes<double>(V.n, V.nnz, nc) : smem_bytes<float>(V.n, V.nnz, nc);
            if (need <= kEngSmem) {
                emit(OP_SWEEP_SMEM, l, count, nc, true);
                return;
            }
        }
        for (int k = 0; k < count; k++) sweep(l);
    }
    void sweep(int l) {
        const SolveLevel &V = h->lv[l];
        const bool sb = level_sb(l);
        const int nc = (int)V.cb.size() / 4;
        if (sb) {
            emit(OP_SWEEP_RUN, l, 0, nc, true);
            return;
        }
        if (groups) {
            for (int c = 0; c < nc; c++) emit(OP_SWEEP, l, c, c + 1, false);
            return;
        }
        const int64_t tbase = V.tn > 0 ? (prec == 0 ? tail_smem_base<double>(V.tn, V.tnc, V.tmaxq)
                                                    : tail_smem_base<float>(V.tn, V.tnc, V.tmaxq)) : 0;
        const bool tail = V.tn > 0 && tbase <= kEngSmem;
        const int cend = tail ? V.tc0 : nc;   // colours before the tail
        const std::vector<int32_t> &seg = V.seg[prec];
        for (size_t q = 0; q < seg.size(); q += 3) {
            const int c0 = seg[q], c1 = std::min((int)seg[q + 1], cend);
            if (c0 >= cend) break;
            if (seg[q + 2]) emit(OP_SWEEP_RUN, l, c0, c1, true);
            else emit(OP_SWEEP, l, c0, c0 + 1, false);
        }
        if (tail) {
            const int64_t csr = prec == 0 ? tail_smem_csr<double>(V.tnnz) : tail_smem_csr<float>(V.tnnz);
            emit(OP_TAIL_PRE, l, 0, 0, false);
            emit(OP_TAIL_RUN, l, tbase + csr <= kEngSmem ? 1 : 0, 0, true);
        }
    }
    void coarsest(int l) {
        const SolveLevel &V = h->lv[l];
        if (V.dense) {
            emit(OP_COARSE, l, 0, 0, (int64_t)V.n * std::max(groups, 1) <= 64);
        } else {
            emit(OP_ZERO, l, 0, 0, level_sb(l));
            sweeps(l, h->opt.coarse_sweeps);
        }
    }
    void visit(int l, int theta) {
        const bool sb = level_sb(l);
        if (h->lv[l].elim) {
            // Sec. 3.2 / 4.2: a level above an elimination has gamma = 1 and no
            // relaxation; the step is exact, so no recombination and no mu
            for (int i = 0; i < theta; i++) {
                emit(OP_RESID, l, -1, 0, sb);
                emit(OP_ELIM_RESTRICT, l, 0, 0, sb);
                if (l + 1 == h->L - 1) {
                    coarsest(l + 1);
                } else {
                    const int32_t k = visits[l]++;
                    const double g = h->sl[l].gamma_l;
                    int th = (int)(std::ceil((double)(k + 1) * g) - std::ceil((double)k * g));
                    th = th < 1 ? 1 : (th > 2 ? 2 : th);
                    visit(l + 1, th);
                }
                emit(OP_ELIM_PROLONG, l, 0, 0, sb);
                emit(OP_ELIM_BACK, l, 0, 0, sb);
            }
            return;
        }
        const bool recomb = adaptive && (l >= 1 || h->opt.recomb_finest);
        for (int i = 0; i < theta; i++) {
            sweeps(l, h->opt.nu1);
            emit(OP_RESID, l, recomb ? i : -1, 0, sb);
            emit(OP_RESTRICT, l, 0, 0, sb);
            if (l + 1 == h->L - 1) {
                coarsest(l + 1);
            } else {
                const int32_t k = visits[l]++;
                const double g = h->sl[l].gamma_l;
                int th = (int)(std::ceil((double)(k + 1) * g) - std::ceil((double)k * g));
                th = th < 1 ? 1 : (th > 2 ? 2 : th);
                visit(l + 1, th);
            }
            emit(OP_PROLONG, l, 0, 0, sb);
            sweeps(l, h->opt.nu2);
        }
        if (recomb) {
            emit(OP_RESID, l, -1, 0, sb);
            emit(OP_RECOMB_DOTS, l, theta, 0, sb);
            emit(OP_RECOMB_APPLY, l, theta, 0, sb);
        }
    }
    void cycle() {
        visits.assign(h->L, 0);
        if (h->L == 1) coarsest(0);
        else visit(0, 1);
        if (h->ngraphs > 1) {
            emit(OP_GMEAN_PART, 0, 0, 0, false);
            emit(OP_GMEAN_APPLY, 0, 0, 0, false);
            return;
        }
        const bool sb = level_sb(0);
        emit(OP_MEAN_PART, 0, 0, 0, sb);
        emit(OP_MEAN_APPLY, 0, 0, 0, sb);
    }
};

// Build (and cache) the program of one step.
//   kind 0: FP64 cycle + mean + FP64 residual norm (solve step)
//   kind 1: FP32 refinement step: prep, ir_inner FP32 cycles, update, mean, FP64 residual norm
//   kind 2: one FP64 cycle + mean only
//   kind 3: FP64 residual norm only (initial residual of a batched solve)
// groups > 0 builds the program for 4*groups interleaved right-hand sides.
void build_program(lamg_ctx *h, int kind, int adaptive, std::vector<int32_t> &out, int groups) {
    Builder B{h, kind == 1 ? 1 : 0, adaptive, groups, {}, {}};
    if (kind == 3) {
        // nothing before the residual
    } else if (kind == 1) {
        B.emit(OP_IR_PREP, 0, 0, 0, false);
        for (int k = 0; k < std::max(1, h->opt.ir_inner); k++) B.cycle();
        B.emit(OP_IR_UPDATE, 0, 0, 0, false);
        B.emit(h->ngraphs > 1 ? OP_GMEAN64_PART : OP_MEAN64_PART, 0, 0, 0, false);
        B.emit(h->ngraphs > 1 ? OP_GMEAN64_APPLY : OP_MEAN64_APPLY, 0, 0, 0, false);
    } else {
        B.cycle();
    }
    if (kind != 2) {
        B.emit(OP_RES64, 0, 0, 0, false);
        B.emit(OP_NORM64_FIN, 0, 0, 0, false);
        if (h->ngraphs > 1) B.emit(OP_GNORM64, 0, 0, 0, false);
    }
    out.resize(B.prog.size() * 5);
    for (size_t i = 0; i < B.prog.size(); i++) {
        out[5 * i] = B.prog[i].type;
        out[5 * i + 1] = B.prog[i].level;
        out[5 * i + 2] = B.prog[i].a;
        out[5 * i + 3] = B.prog[i].b;
        out[5 * i + 4] = B.prog[i].sb;
    }
}

// ---------------------------------------------------------------------------
// Runner
// ---------------------------------------------------------------------------

void engine_prepare(lamg_ctx *h) {
    if (h->eng_lv64.get()) return;
    std::vector<MKLevel<double>> d64(h->L);
    std::vector<MKLevel<float>> d32(h->L);
    for (int l = 0; l < h->L; l++) {
        d64[l] = describe<double>(h, l, h->v64[l], h->lv[l].w64.get());
        d32[l] = describe<float>(h, l, h->v32[l], h->lv[l].w32.get());
    }
    h->eng_lv64.alloc(sizeof(MKLevel<double>) * h->L);
    h->eng_lv32.alloc(sizeof(MKLevel<float>) * h->L);
    LAMG_CUDA(cudaMemcpy(h->eng_lv64.get(), d64.data(), sizeof(MKLevel<double>) * h->L, cudaMemcpyHostToDevice));
    LAMG_CUDA(cudaMemcpy(h->eng_lv32.get(), d32.data(), sizeof(MKLevel<float>) * h->L, cudaMemcpyHostToDevice));
    int dev = 0, sms = 0, per = 0;
    LAMG_CUDA(cudaGetDevice(&dev));
    LAMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int p64 = 0, p32 = 0;
    LAMG_CUDA(cudaFuncSetAttribute(k_engine<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kEngSmem));
    LAMG_CUDA(cudaFuncSetAttribute(k_engine<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kEngSmem));
    LAMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p64, k_engine<double>, kEngThreads, kEngSmem));
    LAMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p32, k_engine<float>, kEngThreads, kEngSmem));
    per = std::min(std::min(p64, p32), 1);
    LAMG_REQUIRE(per >= 1, LAMG_ERR_CUDA, "cycle engine cannot be resident");
    h->eng_grid = sms * per;
    h->eng_part.alloc((size_t)h->eng_grid * 8);
    h->eng_bar.alloc(2);
    h->eng_err.alloc(1);
    LAMG_CUDA(cudaMemset(h->eng_bar.get(), 0, 2 * sizeof(unsigned int)));
    LAMG_CUDA(cudaMemset(h->eng_err.get(), 0, sizeof(int32_t)));
}

// The engine's op timer (lamg_op_times): block 0's clock around every op, summed
// per (level, op type, single-block flag) in eng_optime while it is allocated.
void engine_op_times(lamg_ctx *h, int mode, std::vector<unsigned long long> &out) {
    if (mode == 1) {
        if (!h->eng_optime.get()) h->eng_optime.alloc(kOpTimeSlots);
        LAMG_CUDA(cudaMemset(h->eng_optime.get(), 0, h->eng_optime.bytes()));
        return;
    }
    if (mode == -1) {
        h->eng_optime.release();
        return;
    }
    out.assign(kOpTimeSlots, 0ull);
    if (!h->eng_optime.get()) return;
    LAMG_CUDA(cudaMemcpy(out.data(), h->eng_optime.get(), h->eng_optime.bytes(), cudaMemcpyDeviceToHost));
    LAMG_CUDA(cudaMemset(h->eng_optime.get(), 0, h->eng_optime.bytes()));
}

template <class T>
static void set_graphs(EngineArgs<T> &a, lamg_ctx *h) {
    a.ngraphs = h->ngraphs;
    a.gptr = h->gptr_d.get();
    a.iperm0 = h->iperm0.get();
    a.gid0 = h->gid0.get();
    a.gsum = h->gsum.get();
    a.gnorm = h->gnorm.get();
}

// Run program `kind` once on stream s; returns after the launch is queued.
void engine_run(lamg_ctx *h, int kind, int adaptive, double mu, cudaStream_t s) {
    auto &slot = h->eng_prog[kind * 2 + (adaptive ? 1 : 0)];
    int32_t &len = h->eng_len[kind * 2 + (adaptive ? 1 : 0)];
    if (!slot.get()) {
        std::vector<int32_t> prog;
        build_program(h, kind, adaptive, prog);
        slot.alloc(prog.size());
        LAMG_CUDA(cudaMemcpy(slot.get(), prog.data(), sizeof(int32_t) * prog.size(), cudaMemcpyHostToDevice));
        len = (int32_t)(prog.size() / 5);
    }
    MKLevel<double> L0 = describe<double>(h, 0, h->v64[0], h->lv[0].w64.get());
    L0.r = h->r64.get();
    const dim3 grid(h->eng_grid), block(kEngThreads);
    LAMG_CUDA(cudaMemsetAsync(h->eng_bar.get(), 0, 2 * sizeof(unsigned int), s));  // the barrier counts from 0
    if (kind == 1) {
        EngineArgs<float> a{(const Op *)slot.get(), 0, len, (const MKLevel<float> *)h->eng_lv32.get(), L0,
                            (float)mu, h->eng_part.get(), nullptr, h->scratch.get(), h->eng_bar.get(),
                            h->eng_err.get(), h->eng_optime.get()};
        set_graphs(a, h);
        a.nlev = h->L;
        void *args[] = {&a};
        LAMG_CUDA(cudaLaunchCooperativeKernel((void *)k_engine<float>, grid, block, args, kEngSmem, s));
    } else {
        EngineArgs<double> a{(const Op *)slot.get(), 0, len, (const MKLevel<double> *)h->eng_lv64.get(), L0, mu,
                             h->eng_part.get(), nullptr, h->scratch.get(), h->eng_bar.get(), h->eng_err.get(),
                             h->eng_optime.get()};
        set_graphs(a, h);
        a.nlev = h->L;
        void *args[] = {&a};
        LAMG_CUDA(cudaLaunchCooperativeKernel((void *)k_engine<double>, grid, block, args, kEngSmem, s));
    }
    note_launch();
    if (kind != 2) {
        k_engine_norm<<<1, 256, 0, s>>>(h->eng_part.get(), h->eng_grid, h->scratch.get());
        LAMG_CHECK_LAUNCH();
    }
}

// Error word of the last runs (bounded barrier timeout); clears it.
bool engine_failed(lamg_ctx *h, cudaStream_t s) {
    int32_t e = 0;
    LAMG_CUDA(cudaMemcpyAsync(&e, h->eng_err.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LAMG_CUDA(cudaStreamSynchronize(s));
    if (e) {
        LAMG_CUDA(cudaMemsetAsync(h->eng_err.get(), 0, sizeof(int32_t), s));
        LAMG_CUDA(cudaMemsetAsync(h->eng_bar.get(), 0, 2 * sizeof(unsigned int), s));
    }
    return e != 0;
}

// ---------------------------------------------------------------------------
// Allocation-free one-cycle run (lamg_cycle_noalloc)
// ---------------------------------------------------------------------------
// The engine's per-launch scratch -- a row of 8 partial sums per block, the two
// grid-barrier words and the error word -- lives in this fixed array of the
// library's device image instead of the handle's buffers, so a run allocates
// nothing.  Layout: part[kNoAllocMaxBlocks * 8] doubles, then bar[2] (unsigned)
// at +0, err (int32) at +16 of the 256-byte tail.  The partial sums are always
// written before they are read; the barrier and error words must start at zero
// and are cleared by every call.  One array per device, shared by all handles.
constexpr int kNoAllocMaxBlocks = 512;
constexpr size_t kNoAllocPartBytes = (size_t)kNoAllocMaxBlocks * 8 * sizeof(double);
constexpr size_t kNoAllocBytes = kNoAllocPartBytes + 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
static unsigned char *noalloc_scratch() {
    int dev = -1;
    LAMG_CUDA(cudaGetDevice(&dev));
    LAMG_REQUIRE(dev >= 0 && dev < kNoAllocMaxDevices, LAMG_ERR_ARG, "lamg_cycle_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            throw Error{LAMG_ERR_CUDA, std::string("lamg_cycle_noalloc: scratch address lookup failed: ") +
                                           cudaGetErrorString(e)};
        g_noalloc_addr[dev] = (unsigned char *)p;
    }
    return g_noalloc_addr[dev];
}

bool engine_noalloc_ready(lamg_ctx *h, int adaptive) {
    return h->eng_lv64.get() && h->eng_prog[2 * 2 + (adaptive ? 1 : 0)].get() && h->eng_grid > 0;
}

// Launch the one-cycle program (kind 2) with the fixed scratch; queues the
// launch and returns the device address of the error word.
int32_t *engine_run_noalloc(lamg_ctx *h, int adaptive, double mu, cudaStream_t s) {
    LAMG_REQUIRE(engine_noalloc_ready(h, adaptive), LAMG_ERR_ARG,
                 "lamg_cycle_noalloc: handle not prepared (call lamg_cycle once with the same adaptive flag)");
    LAMG_REQUIRE(h->eng_grid <= kNoAllocMaxBlocks, LAMG_ERR_ARG,
                 "lamg_cycle_noalloc: engine grid of " + std::to_string(h->eng_grid) +
                     " blocks exceeds the fixed scratch limit of " + std::to_string(kNoAllocMaxBlocks));
    unsigned char *base = noalloc_scratch();
    double *part = (double *)base;
    unsigned int *bar = (unsigned int *)(base + kNoAllocPartBytes);
    int32_t *err = (int32_t *)(base + kNoAllocPartBytes + 16);
    LAMG_CUDA(cudaMemsetAsync(base + kNoAllocPartBytes, 0, 256, s));
    const int k = 2 * 2 + (adaptive ? 1 : 0);
    MKLevel<double> L0 = describe<double>(h, 0, h->v64[0], h->lv[0].w64.get());
    L0.r = h->r64.get();
    EngineArgs<double> a{(const Op *)h->eng_prog[k].get(), 0, h->eng_len[k],
                         (const MKLevel<double> *)h->eng_lv64.get(), L0, mu, part, nullptr, h->scratch.get(),
                         bar, err, nullptr};
    set_graphs(a, h);
    a.nlev = h->L;
    void *args[] = {&a};
    LAMG_CUDA(cudaLaunchCooperativeKernel((void *)k_engine<double>, dim3(h->eng_grid), dim3(kEngThreads), args,
                                          kEngSmem, s));
    note_launch();
    return err;
}

// Runs k_barrier_probe on the engine's grid; returns the error word.
int32_t barrier_selftest(int32_t hold_one, cudaStream_t s) {
    int dev = 0, sms = 0, per = 0;
    LAMG_CUDA(cudaGetDevice(&dev));
    LAMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LAMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_barrier_probe, kEngThreads, 0));
    LAMG_REQUIRE(per >= 1, LAMG_ERR_CUDA, "barrier probe cannot be resident");
    Tmp<unsigned int> bar(2, s);
    Tmp<int32_t> err(1, s);
    LAMG_CUDA(cudaMemsetAsync(bar.get(), 0, 2 * sizeof(unsigned int), s));
    LAMG_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int32_t), s));
    unsigned int *bp = bar.get();
    int32_t *ep = err.get();
    int32_t held = hold_one ? 0 : -1;
    void *args[] = {&bp, &ep, &held};
    LAMG_CUDA(cudaLaunchCooperativeKernel((void *)k_barrier_probe, dim3(sms), dim3(kEngThreads), args, 0, s));
    note_launch();
    return read_scalar(err.get(), s);
}

int64_t engine_program_ops(lamg_ctx *h, int kind, int adaptive) {
    return h->eng_len[kind * 2 + (adaptive ? 1 : 0)];
}

}  // namespace lamg
