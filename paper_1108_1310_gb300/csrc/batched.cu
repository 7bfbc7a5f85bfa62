// batched.cu -- lamg_solve_batched: many right-hand sides on one hierarchy.
//
// Re-solving with another b reuses the whole setup (Sec. 1 and Sec. 5: the
// setup is paid once, each solve costs only cycles).  Here up to kMaxCols
// right-hand sides run through the same cycle program at once.  Level vectors
// are stored row-interleaved, ld = 4 * G columns per node (G a power of two),
// so every relaxation, residual, restriction and prolongation gathers 4
// consecutive columns of a neighbour with one 16-byte (FP32) or two 16-byte
// (FP64) loads: an SpMM with the row's weights read once per column group
// instead of once per right-hand side.  Recombination (Eq. (3.13)), the mean
// projection and the outer residual norms are per column: each column keeps
// its own recombination coefficients, exactly as if it were solved alone.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "engine.cuh"

namespace lamg {

constexpr int kMaxCols = 128;  // columns per engine run: at most 32 groups of 4

// ---------------------------------------------------------------------------
// 4-wide loads and stores (ld is a multiple of 4: 16-byte aligned for FP32,
// 32-byte aligned for FP64)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void ld4(const float *p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&v)[4]) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double *p, const double (&v)[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}
template <class T>
__device__ __forceinline__ void zero4(T (&v)[4]) { v[0] = v[1] = v[2] = v[3] = T(0); }

// sum of N values over the tier's lanes (result in every lane of the tier)
template <int M, class T, int N>
__device__ __forceinline__ void reduce_n(T (&v)[N]) {
    if (M == M_WARP) {
#pragma unroll
        for (int k = 0; k < N; k++) v[k] = warp_allsum(v[k]);
    }
    if (M == M_BLK) block_sum_n<T, N>(v);
}

// ---------------------------------------------------------------------------
// row routines on one column group g of row i (tier M lanes share the row)
// ---------------------------------------------------------------------------

// x_i = (b_i + sum_v w_iv x_v) / sum_v w_iv for 4 columns
template <int M, class T>
__device__ __forceinline__ void gs_row4(int32_t i, int g, const MKLevel<T> &L, int ld) {
    const int32_t e = L.rp[i + 1];
    const int st = sstride<M>();
    const T *xg = L.x + 4 * g;
    T v[5] = {T(0), T(0), T(0), T(0), T(0)};  // 4 sums, then the weighted degree
    int32_t j = L.rp[i] + slane<M>();
    for (; j + 3 * st < e; j += 4 * st) {
        int32_t c[4];
        T wv[4], xv[4][4];
#pragma unroll
        for (int k = 0; k < 4; k++) c[k] = L.col[j + k * st];
#pragma unroll
        for (int k = 0; k < 4; k++) wv[k] = L.w[j + k * st];
#pragma unroll
        for (int k = 0; k < 4; k++) ld4(xg + (int64_t)c[k] * ld, xv[k]);
#pragma unroll
        for (int k = 0; k < 4; k++) {
#pragma unroll
            for (int q = 0; q < 4; q++) v[q] += wv[k] * xv[k][q];
            v[4] += wv[k];
        }
    }
    for (; j < e; j += st) {
        const T wj = L.w[j];
        T xv[4];
        ld4(xg + (int64_t)L.col[j] * ld, xv);
#pragma unroll
        for (int q = 0; q < 4; q++) v[q] += wj * xv[q];
        v[4] += wj;
    }
    reduce_n<M, T, 5>(v);
    if (slane<M>() == 0 && e > L.rp[i]) {
        T bv[4], o[4];
        ld4(L.b + (int64_t)i * ld + 4 * g, bv);
#pragma unroll
        for (int q = 0; q < 4; q++) o[q] = (bv[q] + v[q]) / v[4];
        st4(L.x + (int64_t)i * ld + 4 * g, o);
    }
}

// r_i = b_i + sum_v w_iv (x_v - x_i) for 4 columns; optionally save x_i, r_i
template <int M, class T>
__device__ __forceinline__ void resid_row4(int32_t i, int g, const MKLevel<T> &L, const T *b, const T *x, T *r,
                                           T *xs, T *rs, int ld) {
    const int32_t e = L.rp[i + 1];
    const int st = sstride<M>();
    const int64_t off = (int64_t)i * ld + 4 * g;
    T xi[4], v[4];
    ld4(x + off, xi);
    zero4(v);
    int32_t j = L.rp[i] + slane<M>();
    for (; j + 3 * st < e; j += 4 * st) {
        int32_t c[4];
        T wv[4], xv[4][4];
#pragma unroll
        for (int k = 0; k < 4; k++) c[k] = L.col[j + k * st];
#pragma unroll
        for (int k = 0; k < 4; k++) wv[k] = L.w[j + k * st];
#pragma unroll
        for (int k = 0; k < 4; k++) ld4(x + (int64_t)c[k] * ld + 4 * g, xv[k]);
#pragma unroll
        for (int k = 0; k < 4; k++)
#pragma unroll
            for (int q = 0; q < 4; q++) v[q] += wv[k] * (xv[k][q] - xi[q]);
    }
    for (; j < e; j += st) {
        const T wj = L.w[j];
        T xv[4];
        ld4(x + (int64_t)L.col[j] * ld + 4 * g, xv);
#pragma unroll
        for (int q = 0; q < 4; q++) v[q] += wj * (xv[q] - xi[q]);
    }
    reduce_n<M, T, 4>(v);
    if (slane<M>() == 0) {
        T bv[4], o[4];
        ld4(b + off, bv);
#pragma unroll
        for (int q = 0; q < 4; q++) o[q] = bv[q] + v[q];
        st4(r + off, o);
        if (xs) {
            st4(xs + off, xi);
            st4(rs + off, o);
        }
    }
}

// b^c_J = mu sum_{i in T_J} r_i for 4 columns
template <int M, class T>
__device__ __forceinline__ void restrict_row4(int32_t J, int g, const MKLevel<T> &F, const MKLevel<T> &C, T mu,
                                              int ld) {
    const int32_t e = F.mptr[J + 1];
    const int st = sstride<M>();
    T v[4];
    zero4(v);
    int32_t j = F.mptr[J] + slane<M>();
    for (; j + 1 * st < e; j += 2 * st) {
        T a[4], b[4];
        ld4(F.r + (int64_t)F.mlist[j] * ld + 4 * g, a);
        ld4(F.r + (int64_t)F.mlist[j + st] * ld + 4 * g, b);
#pragma unroll
        for (int q = 0; q < 4; q++) v[q] += a[q] + b[q];
    }
    for (; j < e; j += st) {
        T a[4];
        ld4(F.r + (int64_t)F.mlist[j] * ld + 4 * g, a);
#pragma unroll
        for (int q = 0; q < 4; q++) v[q] += a[q];
    }
    reduce_n<M, T, 4>(v);
    if (slane<M>() == 0) {
#pragma unroll
        for (int q = 0; q < 4; q++) v[q] *= mu;
        st4(C.b + (int64_t)J * ld + 4 * g, v);
    }
}

// kept row i of a level followed by elimination (Sec. 3.2), 4 columns:
// b^c = r_i + sum over its eliminated neighbours f of w_if r_f / a_ff; x^c = 0
template <int M, class T>
__device__ __forceinline__ void elim_restrict_row4(int32_t i, int g, const MKLevel<T> &L, const MKLevel<T> &C,
                                                   int ld) {
    const int32_t e = L.rp[i + 1];
    const int st = sstride<M>();
    T v[4];
    zero4(v);
    for (int32_t j = L.rp[i] + slane<M>(); j < e; j += st) {
        const int32_t f = L.col[j];
        if (L.ecx[f] >= 0) continue;
        const T wj = L.w[j], d = L.ed[f];
        T rv[4];
        ld4(L.r + (int64_t)f * ld + 4 * g, rv);
#pragma unroll
        for (int q = 0; q < 4; q++) v[q] += wj * rv[q] / d;
    }
    reduce_n<M, T, 4>(v);
    if (slane<M>() == 0) {
        const int32_t c = L.ecx[i];
        T rv[4], z[4];
        ld4(L.r + (int64_t)i * ld + 4 * g, rv);
#pragma unroll
        for (int q = 0; q < 4; q++) v[q] += rv[q];
        zero4(z);
        st4(C.b + (int64_t)c * ld + 4 * g, v);
        st4(C.x + (int64_t)c * ld + 4 * g, z);
    }
}

// ---------------------------------------------------------------------------
// per-column reductions.  With the grid-stride item index q = tid + k * nthr
// and nthr a multiple of G, a thread always sees the same group g = tid % G.
// ---------------------------------------------------------------------------

struct MRShared {
    double red[32][kMaxCols];   // per-warp column partials
    double coef[5][kMaxCols];   // per-column sums / coefficients
};

// block sums of v (the 4 columns of this thread's group) into prow[0..ld)
__device__ __forceinline__ void block_cols(MRShared &S, double (&v)[4], int G, double *prow) {
    for (int o = 16; o >= G && o > 0; o >>= 1) {
#pragma unroll
        for (int q = 0; q < 4; q++) v[q] += __shfl_xor_sync(kFullMask, v[q], o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, ld = 4 * G;
    __syncthreads();
    if (lane < G) {
#pragma unroll
        for (int q = 0; q < 4; q++) S.red[warp][4 * lane + q] = v[q];
    }
    __syncthreads();
    const int nw = (int)(blockDim.x >> 5);
    for (int c = threadIdx.x; c < ld; c += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < nw; w++) t += S.red[w][c];
        prow[c] = t;
    }
}

// S.coef[k][c] = sum over the nb blocks of part[(b * 8 + slot0 + k) * ld + c], k < ns
// (one warp per (k, c); the same order in every block)
__device__ __forceinline__ void gather_cols(MRShared &S, const double *part, int nb, int slot0, int ns, int ld) {
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    for (int p = warp; p < ns * ld; p += nw) {
        const int k = p / ld, c = p % ld;
        double t = 0.0;
        for (int b = lane; b < nb; b += 32) t += part[((int64_t)b * 8 + slot0 + k) * ld + c];
        t = warp_allsum(t);
        if (lane == 0) S.coef[k][c] = t;
    }
    __syncthreads();
}

template <class T>
struct MRArgs {
    const Op *prog;
    int32_t begin, end;
    const MKLevel<T> *lv;
    MKLevel<double> L0;   // FP64 finest level, vectors n x ld
    T mu;
    int32_t ld, groups, lg;
    double *part;         // gridDim * 8 * ld partial sums
    unsigned int *bar;
    int32_t *err;
};

template <class T>
__device__ __forceinline__ void sweep_colour4(const MRArgs<T> &a, const MKLevel<T> &L, int c, int bid, int nb) {
    const int32_t t0 = L.cb[4 * c], t1 = L.cb[4 * c + 1], t2 = L.cb[4 * c + 2], t3 = L.cb[4 * c + 3];
    const int G = a.groups, lg = a.lg, ld = a.ld;
    const int64_t nthr = (int64_t)nb * blockDim.x, tid = spread_tid(bid, nb);
    for (int64_t q = (int64_t)t0 * G + tid; q < (int64_t)t1 * G; q += nthr)
        gs_row4<M_THR, T>((int32_t)(q >> lg), (int)(q & (G - 1)), L, ld);
    const int64_t nwarp = nthr >> 5, wid = tid >> 5;
    for (int64_t k = wid; k < (int64_t)(t2 - t1) * G; k += nwarp)
        gs_row4<M_WARP, T>(t1 + (int32_t)(k >> lg), (int)(k & (G - 1)), L, ld);
    for (int64_t k = bid; k < (int64_t)(t3 - t2) * G; k += nb)
        gs_row4<M_BLK, T>(t2 + (int32_t)(k >> lg), (int)(k & (G - 1)), L, ld);
}

template <class T, class U>
__device__ __forceinline__ void residual4(const MRArgs<U> &a, const MKLevel<T> &L, const T *b, const T *x, T *r,
                                          T *xs, T *rs, int bid, int nb) {
    const int G = a.groups, lg = a.lg, ld = a.ld;
    const int64_t nthr = (int64_t)nb * blockDim.x, tid = spread_tid(bid, nb);
    for (int64_t q = tid; q < (int64_t)L.n * G; q += nthr) {
        const int32_t i = (int32_t)(q >> lg);
        if (L.rp[i + 1] - L.rp[i] > kLongRow) continue;
        resid_row4<M_THR, T>(i, (int)(q & (G - 1)), L, b, x, r, xs, rs, ld);
    }
    const int64_t nwarp = nthr >> 5, wid = tid >> 5;
    for (int64_t k = wid; k < (int64_t)L.nw * G; k += nwarp)
        resid_row4<M_WARP, T>(L.wrows[k >> lg], (int)(k & (G - 1)), L, b, x, r, xs, rs, ld);
    for (int64_t k = bid; k < (int64_t)L.nb * G; k += nb)
        resid_row4<M_BLK, T>(L.brows[k >> lg], (int)(k & (G - 1)), L, b, x, r, xs, rs, ld);
}

// the elimination ops of the batched engine, kept out of line so that their
// registers do not weigh on the rest of the op switch
template <class T>
__device__ __noinline__ void exec_elim4(const MRArgs<T> &a, const Op &op, int bid, int nb) {
    const int64_t nthr = (int64_t)nb * blockDim.x, tid = spread_tid(bid, nb);
    const int G = a.groups, lg = a.lg, ld = a.ld;
    const MKLevel<T> &L = a.lv[op.level];
    const int64_t items = (int64_t)L.n * G;
    switch (op.type) {
        case OP_ELIM_RESTRICT: {
            // the eliminated rows have degree <= 4 (thread tier); warp/block-tier rows are kept rows
            const MKLevel<T> &C = a.lv[op.level + 1];
            for (int64_t q = tid; q < items; q += nthr) {
                const int32_t i = (int32_t)(q >> lg);
                if (L.ecx[i] < 0 || L.rp[i + 1] - L.rp[i] > kLongRow) continue;
                elim_restrict_row4<M_THR, T>(i, (int)(q & (G - 1)), L, C, ld);
            }
            const int64_t nwarp = nthr >> 5, wid = tid >> 5;
            for (int64_t k = wid; k < (int64_t)L.nw * G; k += nwarp) {
                const int32_t i = L.wrows[k >> lg];
                if (L.ecx[i] >= 0) elim_restrict_row4<M_WARP, T>(i, (int)(k & (G - 1)), L, C, ld);
            }
            for (int64_t k = bid; k < (int64_t)L.nb * G; k += nb) {
                const int32_t i = L.brows[k >> lg];
                if (L.ecx[i] >= 0) elim_restrict_row4<M_BLK, T>(i, (int)(k & (G - 1)), L, C, ld);
            }
            break;
        }
        case OP_ELIM_PROLONG: {
            const MKLevel<T> &C = a.lv[op.level + 1];
            for (int64_t q = tid; q < items; q += nthr) {
                const int64_t i = q >> lg;
                const int32_t c = L.ecx[i];
                if (c < 0) continue;
                const int gg = (int)(q & (G - 1));
                T xv[4], cv[4];
                ld4(L.x + i * ld + 4 * gg, xv);
                ld4(C.x + (int64_t)c * ld + 4 * gg, cv);
#pragma unroll
                for (int k = 0; k < 4; k++) xv[k] += cv[k];
                st4(L.x + i * ld + 4 * gg, xv);
            }
            break;
        }
        case OP_ELIM_BACK:
            // exact back-substitution x_f = (b_f + sum_c w_fc x_c) / a_ff per column
            for (int64_t q = tid; q < items; q += nthr) {
                const int64_t i = q >> lg;
                if (L.ecx[i] >= 0) continue;
                const int gg = (int)(q & (G - 1));
                T acc[4];
                ld4(L.b + i * ld + 4 * gg, acc);
                for (int32_t j = L.rp[i]; j < L.rp[i + 1]; j++) {
                    const T wj = L.w[j];
                    T xv[4];
                    ld4(L.x + (int64_t)L.col[j] * ld + 4 * gg, xv);
#pragma unroll
                    for (int k = 0; k < 4; k++) acc[k] += wj * xv[k];
                }
                const T d = L.ed[i];
#pragma unroll
                for (int k = 0; k < 4; k++) acc[k] = acc[k] / d;
                st4(L.x + i * ld + 4 * gg, acc);
            }
            break;
        default:
            break;
    }
}

template <class T>
__device__ void exec_op4(const MRArgs<T> &a, MRShared &S, const Op &op, int bid, int nb) {
    const int64_t nthr = (int64_t)nb * blockDim.x, tid = spread_tid(bid, nb);
    const int G = a.groups, lg = a.lg, ld = a.ld;
    const int g = (int)(tid & (G - 1));
    const MKLevel<T> &L = a.lv[op.level];
    const int64_t items = (int64_t)L.n * G;
    if (op.type >= OP_ELIM_RESTRICT) {
        exec_elim4<T>(a, op, bid, nb);
        return;
    }
    switch (op.type) {
        case OP_SWEEP:
            sweep_colour4<T>(a, L, op.a, bid, nb);
            break;
        case OP_SWEEP_RUN:
            for (int c = op.a; c < op.b; c++) {
                sweep_colour4<T>(a, L, c, 0, 1);
                __syncthreads();
            }
            break;
        case OP_RESID: {
            T *xs = op.a == 0 ? L.xs0 : (op.a == 1 ? L.xs1 : nullptr);
            T *rs = op.a == 0 ? L.rs0 : (op.a == 1 ? L.rs1 : nullptr);
            residual4<T, T>(a, L, L.b, L.x, L.r, xs, rs, bid, nb);
            break;
        }
        case OP_RESTRICT: {
            const MKLevel<T> &C = a.lv[op.level + 1];
            for (int64_t q = tid; q < (int64_t)C.n * G; q += nthr) {
                const int32_t J = (int32_t)(q >> lg);
                const int gg = (int)(q & (G - 1));
                T z[4];
                zero4(z);
                st4(C.x + (int64_t)J * ld + 4 * gg, z);
                if (L.mptr[J + 1] - L.mptr[J] > kLongRow) continue;
                restrict_row4<M_THR, T>(J, gg, L, C, a.mu, ld);
            }
            const int64_t nwarp = nthr >> 5, wid = tid >> 5;
            for (int64_t k = wid; k < (int64_t)L.nwagg * G; k += nwarp)
                restrict_row4<M_WARP, T>(L.wagg[k >> lg], (int)(k & (G - 1)), L, C, a.mu, ld);
            for (int64_t k = bid; k < (int64_t)L.nbagg * G; k += nb)
                restrict_row4<M_BLK, T>(L.bagg[k >> lg], (int)(k & (G - 1)), L, C, a.mu, ld);
            break;
        }
        case OP_ZERO: {
            T z[4];
            zero4(z);
            for (int64_t q = tid; q < items; q += nthr) st4(L.x + 4 * q, z);
            break;
        }
        case OP_COARSE:
            // x = M^-1 b per column, FP64 accumulation
            for (int64_t q = tid; q < items; q += nthr) {
                const int64_t i = q >> lg;
                const int gg = (int)(q & (G - 1));
                double acc[4] = {0.0, 0.0, 0.0, 0.0};
                const double *mrow = L.minv + i * L.n;
                for (int32_t j = 0; j < L.n; j++) {
                    T bv[4];
                    ld4(L.b + (int64_t)j * ld + 4 * gg, bv);
                    const double m = mrow[j];
#pragma unroll
                    for (int k = 0; k < 4; k++) acc[k] += m * (double)bv[k];
                }
                T o[4];
#pragma unroll
                for (int k = 0; k < 4; k++) o[k] = (T)acc[k];
                st4(L.x + i * ld + 4 * gg, o);
            }
            break;
        case OP_PROLONG: {
            const MKLevel<T> &C = a.lv[op.level + 1];
            for (int64_t q = tid; q < items; q += nthr) {
                const int64_t i = q >> lg;
                const int gg = (int)(q & (G - 1));
                T xv[4], cv[4];
                ld4(L.x + i * ld + 4 * gg, xv);
                ld4(C.x + (int64_t)L.pagg[i] * ld + 4 * gg, cv);
#pragma unroll
                for (int k = 0; k < 4; k++) xv[k] += cv[k];
                st4(L.x + i * ld + 4 * gg, xv);
            }
            break;
        }
        case OP_RECOMB_DOTS: {
            // per column: G00 = |r - r0|^2, G01, G11, h0 = (r, r - r0), h1 (Eq. (3.13))
            double v[5][4];
#pragma unroll
            for (int k = 0; k < 5; k++) v[k][0] = v[k][1] = v[k][2] = v[k][3] = 0.0;
            for (int64_t q = tid; q < items; q += nthr) {
                T r[4], r0[4];
                ld4(L.r + 4 * q, r);
                ld4(L.rs0 + 4 * q, r0);
                if (op.a == 2) {
                    T r1[4];
                    ld4(L.rs1 + 4 * q, r1);
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        const double ri = (double)r[c], d0 = ri - (double)r0[c], d1 = ri - (double)r1[c];
                        v[0][c] += d0 * d0;
                        v[1][c] += d0 * d1;
                        v[2][c] += d1 * d1;
                        v[3][c] += ri * d0;
                        v[4][c] += ri * d1;
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        const double ri = (double)r[c], d0 = ri - (double)r0[c];
                        v[0][c] += d0 * d0;
                        v[3][c] += ri * d0;
                    }
                }
            }
            for (int k = 0; k < 5; k++) block_cols(S, v[k], G, a.part + ((int64_t)bid * 8 + k) * ld);
            break;
        }
        case OP_RECOMB_APPLY: {
            gather_cols(S, a.part, nb, 0, 5, ld);
            for (int c = threadIdx.x; c < ld; c += blockDim.x) {
                const double G00 = S.coef[0][c], G01 = S.coef[1][c], G11 = S.coef[2][c];
                const double h0 = S.coef[3][c], h1 = S.coef[4][c];
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
                S.red[0][c] = a0;
                S.red[1][c] = a1;
            }
            __syncthreads();
            for (int64_t q = tid; q < items; q += nthr) {
                const int gg = (int)(q & (G - 1));
                T x[4], x0[4], x1[4];
                ld4(L.x + 4 * q, x);
                ld4(L.xs0 + 4 * q, x0);
                if (op.a == 2) ld4(L.xs1 + 4 * q, x1);
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const double xi = (double)x[c];
                    double y = xi + S.red[0][4 * gg + c] * ((double)x0[c] - xi);
                    if (op.a == 2) y += S.red[1][4 * gg + c] * ((double)x1[c] - xi);
                    x[c] = (T)y;
                }
                st4(L.x + 4 * q, x);
            }
            __syncthreads();
            break;
        }
        case OP_MEAN_PART: {
            double v[4] = {0.0, 0.0, 0.0, 0.0};
            for (int64_t q = tid; q < items; q += nthr) {
                T x[4];
                ld4(L.x + 4 * q, x);
#pragma unroll
                for (int c = 0; c < 4; c++) v[c] += (double)x[c];
            }
            block_cols(S, v, G, a.part + (int64_t)bid * 8 * ld);
            break;
        }
        case OP_MEAN_APPLY: {
            gather_cols(S, a.part, nb, 0, 1, ld);
            for (int64_t q = tid; q < items; q += nthr) {
                const int gg = (int)(q & (G - 1));
                T x[4];
                ld4(L.x + 4 * q, x);
#pragma unroll
                for (int c = 0; c < 4; c++) x[c] = (T)((double)x[c] - S.coef[0][4 * gg + c] / (double)L.n);
                st4(L.x + 4 * q, x);
            }
            __syncthreads();
            break;
        }
        case OP_IR_PREP: {
            T z[4];
            zero4(z);
            for (int64_t q = tid; q < items; q += nthr) {
                double r[4];
                ld4(a.L0.r + 4 * q, r);
                T bv[4];
#pragma unroll
                for (int c = 0; c < 4; c++) bv[c] = (T)r[c];
                st4(L.b + 4 * q, bv);
                st4(L.x + 4 * q, z);
            }
            break;
        }
        case OP_IR_UPDATE:
            for (int64_t q = tid; q < items; q += nthr) {
                double x[4];
                T e[4];
                ld4(a.L0.x + 4 * q, x);
                ld4(L.x + 4 * q, e);
#pragma unroll
                for (int c = 0; c < 4; c++) x[c] += (double)e[c];
                st4(a.L0.x + 4 * q, x);
            }
            break;
        case OP_MEAN64_PART: {
            double v[4] = {0.0, 0.0, 0.0, 0.0};
            for (int64_t q = tid; q < (int64_t)a.L0.n * G; q += nthr) {
                double x[4];
                ld4(a.L0.x + 4 * q, x);
#pragma unroll
                for (int c = 0; c < 4; c++) v[c] += x[c];
            }
            block_cols(S, v, G, a.part + (int64_t)bid * 8 * ld);
            break;
        }
        case OP_MEAN64_APPLY: {
            gather_cols(S, a.part, nb, 0, 1, ld);
            for (int64_t q = tid; q < (int64_t)a.L0.n * G; q += nthr) {
                const int gg = (int)(q & (G - 1));
                double x[4];
                ld4(a.L0.x + 4 * q, x);
#pragma unroll
                for (int c = 0; c < 4; c++) x[c] -= S.coef[0][4 * gg + c] / (double)a.L0.n;
                st4(a.L0.x + 4 * q, x);
            }
            __syncthreads();
            break;
        }
        case OP_RES64:
            residual4<double, T>(a, a.L0, a.L0.b, a.L0.x, a.L0.r, (double *)nullptr, (double *)nullptr, bid, nb);
            break;
        case OP_NORM64_FIN: {
            double v[4] = {0.0, 0.0, 0.0, 0.0};
            for (int64_t q = tid; q < (int64_t)a.L0.n * G; q += nthr) {
                double r[4];
                ld4(a.L0.r + 4 * q, r);
#pragma unroll
                for (int c = 0; c < 4; c++) v[c] += r[c] * r[c];
            }
            block_cols(S, v, G, a.part + ((int64_t)bid * 8 + 5) * ld);
            break;
        }
        default:
            break;
    }
    (void)g;
}

template <class T>
__global__ void __launch_bounds__(kEngThreads, 1) k_engine4(MRArgs<T> a) {
    __shared__ MRShared S;
    int32_t pc = a.begin;
    unsigned int epoch = 0;
    while (pc < a.end) {
        const Op op = a.prog[pc];
        if (op.sb) {
            int32_t q = pc;
            if (blockIdx.x == 0) {
                while (q < a.end && a.prog[q].sb) {
                    exec_op4<T>(a, S, a.prog[q], 0, 1);
                    __syncthreads();
                    q++;
                }
            } else {
                while (q < a.end && a.prog[q].sb) q++;
            }
            pc = q;
        } else {
            exec_op4<T>(a, S, op, blockIdx.x, gridDim.x);
            pc++;
        }
        if (!grid_sync(a.bar, a.err, epoch)) return;
    }
}

// out[c] = sum over blocks of the slot-5 partials (||r64||^2 per column)
__global__ void k_norm4(const double *part, int nb, int ld, double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    for (int c = warp; c < ld; c += nw) {
        double t = 0.0;
        for (int b = lane; b < nb; b += 32) t += part[((int64_t)b * 8 + 5) * ld + c];
        t = warp_allsum(t);
        if (lane == 0) out[c] = t;
    }
}

// dst[i * ld + c] = src[perm[i] * lds + c] for c < R, 0 for R <= c < ld
__global__ void k_gather4(int32_t n, int32_t ld, int32_t R, const int32_t *__restrict__ perm,
                          const double *__restrict__ src, int64_t lds, double *__restrict__ dst) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * ld) return;
    const int64_t i = q / ld;
    const int c = (int)(q % ld);
    dst[q] = c < R ? src[(int64_t)perm[i] * lds + c] : 0.0;
}

// b[i * ld + c] -= mean[c] (columns past the batch have mean 0)
__global__ void k_sub_colmean(int32_t n, int32_t ld, const double *__restrict__ mean, double *__restrict__ b) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * ld) return;
    b[q] -= mean[q % ld];
}

__global__ void k_scatter4(int32_t n, int32_t ld, int32_t R, const int32_t *__restrict__ perm,
                           const double *__restrict__ src, int64_t lds, double *__restrict__ dst) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * ld) return;
    const int64_t i = q / ld;
    const int c = (int)(q % ld);
    if (c < R) dst[(int64_t)perm[i] * lds + c] = src[q];
}

// per-column sum, sum of |.| and sum of squares of an n x ld FP64 block
__global__ void __launch_bounds__(1024) k_colstats(int32_t n, int G, const double *__restrict__ v,
                                                   double *__restrict__ part) {
    __shared__ MRShared S;
    const int ld = 4 * G;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x, tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double s[3][4] = {};
    for (int64_t q = tid; q < (int64_t)n * G; q += nthr) {
        double x[4];
        ld4(v + 4 * q, x);
#pragma unroll
        for (int c = 0; c < 4; c++) {
            s[0][c] += x[c];
            s[1][c] += fabs(x[c]);
            s[2][c] += x[c] * x[c];
        }
    }
    for (int k = 0; k < 3; k++) block_cols(S, s[k], G, part + ((int64_t)blockIdx.x * 8 + k) * ld);
}

__global__ void __launch_bounds__(1024) k_colstats_fin(const double *part, int nb, int ld, double *out) {
    __shared__ MRShared S;
    gather_cols(S, part, nb, 0, 3, ld);
    for (int p = threadIdx.x; p < 3 * ld; p += blockDim.x) out[p] = S.coef[p / ld][p % ld];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static int groups_for(int R) {
    int G = 1;
    while (4 * G < R) G <<= 1;
    return G;
}

template <class T>
static void alloc_vecs4(lamg_ctx *h, std::vector<LevelVecs<T>> &vv, int ld) {
    vv.resize(h->L);
    for (int l = 0; l < h->L; l++) {
        const size_t n = (size_t)h->lv[l].n * ld;
        vv[l].x.alloc(n);
        vv[l].b.alloc(n);
        vv[l].r.alloc(n);
        if ((l >= 1 || h->opt.recomb_finest) && l + 1 < h->L) {
            vv[l].xs0.alloc(n); vv[l].xs1.alloc(n);
            vv[l].rs0.alloc(n); vv[l].rs1.alloc(n);
        }
    }
}

static void batch_prepare(lamg_ctx *h, int groups) {
    if (h->mr && h->mr->groups == groups) return;
    h->mr.reset();
    std::unique_ptr<BatchState> M(new BatchState);
    M->groups = groups;
    M->ld = 4 * groups;
    const int ld = M->ld;
    alloc_vecs4<double>(h, M->v64, ld);
    alloc_vecs4<float>(h, M->v32, ld);
    M->r64.alloc((size_t)h->lv[0].n * ld);
    M->out.alloc(4 * (size_t)ld);
    std::vector<MKLevel<double>> d64(h->L);
    std::vector<MKLevel<float>> d32(h->L);
    for (int l = 0; l < h->L; l++) {
        d64[l] = describe<double>(h, l, M->v64[l], h->lv[l].w64.get());
        d32[l] = describe<float>(h, l, M->v32[l], h->lv[l].w32.get());
    }
    M->lv64.alloc(sizeof(MKLevel<double>) * h->L);
    M->lv32.alloc(sizeof(MKLevel<float>) * h->L);
    LAMG_CUDA(cudaMemcpy(M->lv64.get(), d64.data(), sizeof(MKLevel<double>) * h->L, cudaMemcpyHostToDevice));
    LAMG_CUDA(cudaMemcpy(M->lv32.get(), d32.data(), sizeof(MKLevel<float>) * h->L, cudaMemcpyHostToDevice));
    int dev = 0, sms = 0, p64 = 0, p32 = 0;
    LAMG_CUDA(cudaGetDevice(&dev));
    LAMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LAMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p64, k_engine4<double>, kEngThreads, 0));
    LAMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p32, k_engine4<float>, kEngThreads, 0));
    LAMG_REQUIRE(std::min(p64, p32) >= 1, LAMG_ERR_CUDA, "batched cycle engine cannot be resident");
    M->grid = sms;
    M->part.alloc((size_t)M->grid * 8 * ld);
    M->bar.alloc(2);
    M->err.alloc(1);
    LAMG_CUDA(cudaMemset(M->bar.get(), 0, 2 * sizeof(unsigned int)));
    LAMG_CUDA(cudaMemset(M->err.get(), 0, sizeof(int32_t)));
    h->mr = std::move(M);
}

// kind 0: FP64 step, 1: FP32-IR step, 3: FP64 residual norms only
static void batch_run(lamg_ctx *h, int kind, int adaptive, cudaStream_t s) {
    BatchState &M = *h->mr;
    const int slot = (kind == 3 ? 2 : kind) * 2 + (adaptive ? 1 : 0);
    if (!M.prog[slot].get()) {
        std::vector<int32_t> prog;
        build_program(h, kind, adaptive, prog, M.groups);
        M.prog[slot].alloc(prog.size());
        LAMG_CUDA(cudaMemcpy(M.prog[slot].get(), prog.data(), sizeof(int32_t) * prog.size(), cudaMemcpyHostToDevice));
        M.len[slot] = (int32_t)(prog.size() / 5);
    }
    int lg = 0;
    while ((1 << lg) < M.groups) lg++;
    MKLevel<double> L0 = describe<double>(h, 0, M.v64[0], h->lv[0].w64.get());
    L0.r = M.r64.get();
    const double mu = adaptive ? h->opt.mu_adaptive : h->opt.mu_flat;
    LAMG_CUDA(cudaMemsetAsync(M.bar.get(), 0, 2 * sizeof(unsigned int), s));  // the barrier counts from 0
    const bool timed = h->prof_on && kind != 3;
    if (timed) {   // CUDA events around the engine launch (lamg_profile)
        if (h->prof_ev.size() < 2) {
            for (int k = 0; k < 2; k++) {
                cudaEvent_t e;
                LAMG_CUDA(cudaEventCreate(&e));
                h->prof_ev.push_back(e);
            }
        }
        LAMG_CUDA(cudaEventRecord(h->prof_ev[0], s));
    }
    if (kind == 1) {
        MRArgs<float> a{(const Op *)M.prog[slot].get(), 0, M.len[slot], (const MKLevel<float> *)M.lv32.get(), L0,
                        (float)mu, M.ld, M.groups, lg, M.part.get(), M.bar.get(), M.err.get()};
        void *args[] = {&a};
        LAMG_CUDA(cudaLaunchCooperativeKernel((void *)k_engine4<float>, dim3(M.grid), dim3(kEngThreads), args, 0, s));
    } else {
        MRArgs<double> a{(const Op *)M.prog[slot].get(), 0, M.len[slot], (const MKLevel<double> *)M.lv64.get(), L0,
                         mu, M.ld, M.groups, lg, M.part.get(), M.bar.get(), M.err.get()};
        void *args[] = {&a};
        LAMG_CUDA(cudaLaunchCooperativeKernel((void *)k_engine4<double>, dim3(M.grid), dim3(kEngThreads), args, 0, s));
    }
    note_launch();
    if (timed) {
        LAMG_CUDA(cudaEventRecord(h->prof_ev[1], s));
        // the launch's algorithmic bytes: its cycles on ld columns plus the FP64
        // residual of every column
        const SolveLevel &V = h->lv[0];
        const int64_t res64 = V.nnz * 12 + (int64_t)(V.n + 1) * 4 + (int64_t)V.n * 24 * M.ld;
        M.prof_bytes = kind == 1 ? std::max(1, h->opt.ir_inner) * cycle_bytes(h, 4, M.ld) + res64 +
                                       (int64_t)V.n * 32 * M.ld
                                 : cycle_bytes(h, 8, M.ld) + res64;
        M.prof_pending = 1;
    }
    k_norm4<<<1, 1024, 0, s>>>(M.part.get(), M.grid, M.ld, M.out.get());
    LAMG_CHECK_LAUNCH();
}

// copies the per-column ||r||^2 and the error word; true if the engine timed out
static bool batch_read(lamg_ctx *h, std::vector<double> &out, cudaStream_t s) {
    BatchState &M = *h->mr;
    int32_t e = 0;
    out.resize(M.ld);
    LAMG_CUDA(cudaMemcpyAsync(out.data(), M.out.get(), sizeof(double) * M.ld, cudaMemcpyDeviceToHost, s));
    LAMG_CUDA(cudaMemcpyAsync(&e, M.err.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LAMG_CUDA(cudaStreamSynchronize(s));
    if (M.prof_pending) {
        float ms = 0.f;
        LAMG_CUDA(cudaEventElapsedTime(&ms, h->prof_ev[0], h->prof_ev[1]));
        h->prof_ms += ms;
        h->prof_count++;
        h->prof_bytes = M.prof_bytes;
        M.prof_pending = 0;
    }
    if (e) {
        LAMG_CUDA(cudaMemsetAsync(M.err.get(), 0, sizeof(int32_t), s));
        LAMG_CUDA(cudaMemsetAsync(M.bar.get(), 0, 2 * sizeof(unsigned int), s));
        LAMG_CUDA(cudaStreamSynchronize(s));
    }
    return e != 0;
}

// columns per engine run: the tuned value, else the largest
static int batch_chunk(const lamg_ctx *h) {
    const int c = h->batch_cols;
    return (c >= 4 && c <= kMaxCols) ? c : kMaxCols;
}

void set_batch_cols(lamg_ctx *h, int32_t cols) {
    LAMG_REQUIRE(cols == 0 || (cols >= 4 && cols <= kMaxCols && (cols & (cols - 1)) == 0), LAMG_ERR_ARG,
                 "batch columns must be 0 (default) or a power of two in [4, 128]");
    h->batch_cols = cols;
}

// Autotuner of the column chunk (columns per engine run) of batched solves:
// times one refinement step of `nrhs` columns for each candidate chunk of
// 16, 32, 64 and 128 columns (right-hand side and iterate zero: a step does
// the same work for any values), keeps the fastest in the handle.
void autotune_batched(lamg_ctx *h, int32_t nrhs, lamg_precision p, cudaStream_t s, int32_t *chosen,
                      double *ms_out) {
    LAMG_REQUIRE(h->ngraphs == 1, LAMG_ERR_ARG, "lamg_autotune_batched: needs a single-graph handle");
    prepare_solve(h);
    const int32_t n = h->lv[0].n;
    const int kind = p == LAMG_FP64 ? 0 : 1;
    const int cand[4] = {16, 32, 64, 128};
    cudaEvent_t e0, e1;
    LAMG_CUDA(cudaEventCreate(&e0));
    LAMG_CUDA(cudaEventCreate(&e1));
    double best = 1e300;
    int best_c = kMaxCols;
    std::vector<double> rn2;
    for (int k = 0; k < 4; k++) {
        const int cw = cand[k];
        float ms = 0.f;
        for (int rep = 0; rep < 2; rep++) {   // first pass builds programs and buffers
            LAMG_CUDA(cudaEventRecord(e0, s));
            for (int32_t c0 = 0; c0 < nrhs; c0 += cw) {
                const int R = std::min(cw, nrhs - c0);
                batch_prepare(h, groups_for(R));
                BatchState &M = *h->mr;
                const size_t tot = (size_t)n * M.ld;
                LAMG_CUDA(cudaMemsetAsync(M.v64[0].x.get(), 0, sizeof(double) * tot, s));
                LAMG_CUDA(cudaMemsetAsync(M.v64[0].b.get(), 0, sizeof(double) * tot, s));
                LAMG_CUDA(cudaMemsetAsync(M.r64.get(), 0, sizeof(double) * tot, s));
                batch_run(h, kind, h->opt.adaptive, s);
                if (batch_read(h, rn2, s)) throw Error{LAMG_ERR_TIMEOUT, "cycle engine: grid barrier timed out"};
            }
            LAMG_CUDA(cudaEventRecord(e1, s));
            LAMG_CUDA(cudaEventSynchronize(e1));
            LAMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        }
        if (ms_out) ms_out[k] = ms;
        if (ms < best) { best = ms; best_c = cw; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->batch_cols = best_c;
    if (chosen) *chosen = best_c;
}

void solve_batched_device(lamg_ctx *h, int32_t nrhs, const double *B, double *X, int64_t ld, double tol,
                          lamg_precision p, cudaStream_t s, lamg_stats *st) {
    const auto t0 = std::chrono::steady_clock::now();
    LAMG_REQUIRE(h->ngraphs == 1, LAMG_ERR_ARG,
                 "lamg_solve_batched: several right-hand sides need a single-graph handle");
    prepare_solve(h);
    const int32_t n = h->lv[0].n;
    const int32_t *perm = h->lv[0].perm.get();
    const int adaptive = h->opt.adaptive;
    const int kind = p == LAMG_FP64 ? 0 : 1;
    const int per_step = p == LAMG_FP64 ? 1 : std::max(1, h->opt.ir_inner);
    std::vector<lamg_stats> stats(nrhs);
    bool all_ok = true;
    const int chunk = batch_chunk(h);
    for (int32_t c0 = 0; c0 < nrhs; c0 += chunk) {
        const int R = std::min(chunk, nrhs - c0);
        batch_prepare(h, groups_for(R));
        BatchState &M = *h->mr;
        const int ldi = M.ld;
        const int64_t tot = (int64_t)n * ldi;
        double *xb = M.v64[0].x.get(), *bb = M.v64[0].b.get();
        k_gather4<<<ceil_div(tot, 256), 256, 0, s>>>(n, ldi, R, perm, B + c0, ld, bb);
        LAMG_CHECK_LAUNCH();
        k_gather4<<<ceil_div(tot, 256), 256, 0, s>>>(n, ldi, R, perm, X + c0, ld, xb);
        LAMG_CHECK_LAUNCH();
        // zero-sum check and ||b|| per column (Sec. 1: b must be compatible)
        std::vector<double> cs(3 * (size_t)ldi);
        auto colstats = [&]() {
            k_colstats<<<M.grid, 1024, 0, s>>>(n, M.groups, bb, M.part.get());
            LAMG_CHECK_LAUNCH();
            k_colstats_fin<<<1, 1024, 0, s>>>(M.part.get(), M.grid, ldi, M.out.get());
            LAMG_CHECK_LAUNCH();
            LAMG_CUDA(cudaMemcpyAsync(cs.data(), M.out.get(), sizeof(double) * 3 * ldi, cudaMemcpyDeviceToHost, s));
            LAMG_CUDA(cudaStreamSynchronize(s));
        };
        colstats();
        if (h->opt.project_rhs) {  // solve for each column minus its mean
            std::vector<double> mean(ldi, 0.0);
            for (int c = 0; c < R; c++) mean[c] = cs[c] / (double)n;
            LAMG_CUDA(cudaMemcpyAsync(M.out.get(), mean.data(), sizeof(double) * ldi, cudaMemcpyHostToDevice, s));
            k_sub_colmean<<<ceil_div(tot, 256), 256, 0, s>>>(n, ldi, M.out.get(), bb);
            LAMG_CHECK_LAUNCH();
            colstats();
        }
        std::vector<double> bn(R);
        for (int c = 0; c < R; c++) {
            const double sum = cs[c], asum = cs[ldi + c];
            LAMG_REQUIRE(std::fabs(sum) <= 1e-10 * (asum > 0 ? asum : 1.0), LAMG_ERR_RHS_NOT_ZERO_SUM,
                         "right-hand side column " + std::to_string(c0 + c) + " is not zero-sum");
            bn[c] = std::sqrt(cs[2 * ldi + c]);
        }
        std::vector<double> rn2;
        batch_run(h, 3, adaptive, s);
        if (batch_read(h, rn2, s)) throw Error{LAMG_ERR_TIMEOUT, "cycle engine: grid barrier timed out"};
        std::vector<double> r0(R), rn(R);
        std::vector<int32_t> done_cycles(R, -1), done_steps(R, -1);
        auto converged = [&](int c) { return rn[c] <= tol * bn[c]; };
        int steps = 0, cycles = 0;
        bool pending = false;
        for (int c = 0; c < R; c++) {
            r0[c] = rn[c] = std::sqrt(rn2[c]);
            if (converged(c)) { done_cycles[c] = 0; done_steps[c] = 0; }
            else pending = true;
        }
        while (pending && cycles < h->opt.max_cycles) {
            batch_run(h, kind, adaptive, s);
            if (batch_read(h, rn2, s)) throw Error{LAMG_ERR_TIMEOUT, "cycle engine: grid barrier timed out"};
            steps++;
            cycles += per_step;
            pending = false;
            bool nan = false;
            for (int c = 0; c < R; c++) {
                rn[c] = std::sqrt(rn2[c]);
                if (!(rn[c] == rn[c])) nan = true;
                if (done_cycles[c] < 0 && converged(c)) { done_cycles[c] = cycles; done_steps[c] = steps; }
                if (done_cycles[c] < 0) pending = true;
            }
            if (nan) break;
        }
        k_scatter4<<<ceil_div(tot, 256), 256, 0, s>>>(n, ldi, R, perm, xb, ld, X + c0);
        LAMG_CHECK_LAUNCH();
        LAMG_CUDA(cudaStreamSynchronize(s));
        const double tsolve = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int c = 0; c < R; c++) {
            lamg_stats &S = stats[c0 + c];
            S = h->last;
            S.levels = h->L;
            const bool ok = done_cycles[c] >= 0 && rn[c] == rn[c];
            S.cycles = ok ? done_cycles[c] : cycles;
            S.outer_steps = ok ? done_steps[c] : steps;
            S.rel_res = bn[c] > 0 ? rn[c] / bn[c] : 0.0;
            S.acf = (cycles > 0 && r0[c] > 0 && rn[c] > 0) ? std::pow(rn[c] / r0[c], 1.0 / cycles) : 0.0;
            S.t_setup_s = h->t_setup_s;
            S.t_solve_s = tsolve;
            S.status = ok ? LAMG_OK : LAMG_ERR_NOT_CONVERGED;
            all_ok = all_ok && ok;
        }
    }
    if (st) std::copy(stats.begin(), stats.end(), st);
    if (!all_ok) throw Error{LAMG_ERR_NOT_CONVERGED, "max_cycles reached before tol in some column"};
}

}  // namespace lamg
