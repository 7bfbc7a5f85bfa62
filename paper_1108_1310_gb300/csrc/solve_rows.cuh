// solve_rows.cuh -- per-row device routines of the solve phase, shared by the
// cycle engine: Gauss-Seidel row update (Eq. (2.3)), residual row, restriction
// row (Eq. (3.9)).  Each is templated on the row tier (one thread, one warp,
// or the whole block) and on the value type; the summation order inside a row
// is free here (the solve is checked against the oracle within tolerance).
#pragma once

#include "lamg_internal.cuh"

namespace lamg {

enum { M_THR = 0, M_WARP = 1, M_BLK = 2 };
constexpr unsigned kFullMask = 0xffffffffu;

template <int M> __device__ __forceinline__ int slane() {
    return M == M_THR ? 0 : (M == M_WARP ? (int)(threadIdx.x & 31) : (int)threadIdx.x);
}
template <int M> __device__ __forceinline__ int sstride() {
    return M == M_THR ? 1 : (M == M_WARP ? 32 : (int)blockDim.x);
}

template <class T>
__device__ __forceinline__ T warp_allsum(T v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
    return v;
}

// block sum of two values, result in every thread of the block (the cross-warp
// step in warp 0 only: FP64 adds are expensive on this GPU)
template <class T>
__device__ __forceinline__ void block_allsum2(T &a, T &b) {
    __shared__ T sa[32], sb[32], res[2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    a = warp_allsum(a);
    b = warp_allsum(b);
    __syncthreads();
    if (lane == 0) { sa[warp] = a; sb[warp] = b; }
    __syncthreads();
    if (warp == 0) {
        T ta = lane < nw ? sa[lane] : T(0), tb = lane < nw ? sb[lane] : T(0);
        ta = warp_allsum(ta);
        tb = warp_allsum(tb);
        if (lane == 0) { res[0] = ta; res[1] = tb; }
    }
    __syncthreads();
    a = res[0];
    b = res[1];
    __syncthreads();
}

template <int M, class T>
__device__ __forceinline__ void reduce2(T &a, T &b) {
    if (M == M_WARP) { a = warp_allsum(a); b = warp_allsum(b); }
    if (M == M_BLK) block_allsum2(a, b);
}

// Row dot products with 8 independent gathers in flight per thread.
// acc += sum_j w_j * x[col_j]   and   d += sum_j w_j   over j = s + lane + k*stride
template <int M, class T>
__device__ __forceinline__ void row_dot(int32_t s, int32_t e, const int32_t *__restrict__ col,
                                        const T *__restrict__ w, const T *__restrict__ x, T &acc, T &d) {
    const int st = sstride<M>();
    int32_t j = s + slane<M>();
    for (; j + 7 * st < e; j += 8 * st) {
        int32_t c[8];
        T wv[8], xv[8];
#pragma unroll
        for (int k = 0; k < 8; k++) c[k] = col[j + k * st];
#pragma unroll
        for (int k = 0; k < 8; k++) wv[k] = w[j + k * st];
#pragma unroll
        for (int k = 0; k < 8; k++) xv[k] = x[c[k]];
#pragma unroll
        for (int k = 0; k < 8; k++) { acc += wv[k] * xv[k]; d += wv[k]; }
    }
    for (; j + 1 * st < e; j += 2 * st) {
        const int32_t c0 = col[j], c1 = col[j + st];
        const T w0 = w[j], w1 = w[j + st];
        const T x0 = x[c0], x1 = x[c1];
        acc += w0 * x0 + w1 * x1;
        d += w0 + w1;
    }
    for (; j < e; j += st) {
        const T wj = w[j];
        acc += wj * x[col[j]];
        d += wj;
    }
}

// x_i = (b_i + sum_v w_iv x_v) / sum_v w_iv; a row without entries (an isolated
// node of a union of graphs) is left unchanged
template <int M, class T>
__device__ __forceinline__ void gs_row(int32_t i, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                       const T *__restrict__ w, const T *__restrict__ b, T *__restrict__ x) {
    T acc = T(0), d = T(0);
    const int32_t s = rp[i], e = rp[i + 1];
    row_dot<M, T>(s, e, col, w, x, acc, d);
    reduce2<M>(acc, d);
    if (slane<M>() == 0 && e > s) x[i] = (b[i] + acc) / d;
}

// r_i = b_i - (A x)_i = b_i + sum_v w_iv (x_v - x_i)   (differences: no cancellation)
template <int M, class T>
__device__ __forceinline__ void resid_row(int32_t i, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                          const T *__restrict__ w, const T *__restrict__ b, const T *__restrict__ x,
                                          T *__restrict__ r) {
    const int32_t e = rp[i + 1];
    const int st = sstride<M>();
    const T xi = x[i];
    T acc = T(0), dummy = T(0);
    int32_t j = rp[i] + slane<M>();
    for (; j + 7 * st < e; j += 8 * st) {
        int32_t c[8];
        T wv[8], xv[8];
#pragma unroll
        for (int k = 0; k < 8; k++) c[k] = col[j + k * st];
#pragma unroll
        for (int k = 0; k < 8; k++) wv[k] = w[j + k * st];
#pragma unroll
        for (int k = 0; k < 8; k++) xv[k] = x[c[k]];
#pragma unroll
        for (int k = 0; k < 8; k++) acc += wv[k] * (xv[k] - xi);
    }
    for (; j < e; j += st) acc += w[j] * (x[col[j]] - xi);
    reduce2<M>(acc, dummy);
    if (slane<M>() == 0) r[i] = b[i] + acc;
}

// b^c_J = mu * sum_{i in T_J} r_i
template <int M, class T>
__device__ __forceinline__ void restrict_row(int32_t J, const int32_t *__restrict__ mptr,
                                             const int32_t *__restrict__ mlist, const T *__restrict__ r, T mu,
                                             T *__restrict__ bc) {
    T acc = T(0), dummy = T(0);
    const int st = sstride<M>();
    int32_t j = mptr[J] + slane<M>();
    const int32_t e = mptr[J + 1];
    for (; j + 3 * st < e; j += 4 * st) {
        const int32_t m0 = mlist[j], m1 = mlist[j + st], m2 = mlist[j + 2 * st], m3 = mlist[j + 3 * st];
        acc += (r[m0] + r[m1]) + (r[m2] + r[m3]);
    }
    for (; j < e; j += st) acc += r[mlist[j]];
    reduce2<M>(acc, dummy);
    if (slane<M>() == 0) bc[J] = mu * acc;
}

}  // namespace lamg
