// solve.cu -- the LAMG solve phase on the GPU (Sec. 4.2 and Fig. 4.2 of
// Livne & Brandt, arXiv 1108.1310): multicolour Gauss-Seidel (Eq. (2.3)),
// residual and caliber-1 restriction (Eqs. (2.5), (3.9)), prolongation
// (Eq. (2.6)), iterate recombination (Eq. (3.13)), the dense coarsest solve,
// mean subtraction, and FP32 cycles inside FP64 iterative refinement.
//
// Layout: every level's rows are permuted so that each colour is one
// contiguous range, rows with more than kLongRow entries at the end of their
// colour (warp per row), the rest one thread per row.  Vectors live in this
// order; the user's natural-order vectors are gathered/scattered at the ends.
// One cycle is a fixed launch sequence (the fractional cycle index is
// resolved per cycle), so it is captured once into a CUDA graph.
#include <chrono>
#include <cmath>
#include <cstring>

#include "lamg_internal.cuh"

namespace lamg {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRedBlocks = 608;     // 152 SMs x 4 blocks for reductions
constexpr int kRedThreads = 256;
constexpr int64_t kTailWork32 = 65536;  // entries of a colour run the single-block sweep takes (FP32)
constexpr int64_t kTailWork64 = 8192;   // same for FP64

// scratch layout (doubles)
enum {
    SC_PART = 0,                     // kRedBlocks * 8 partial sums
    SC_ALPHA = kRedBlocks * 8,       // recombination coefficients per level (2 each)
    SC_NORM = SC_ALPHA + 2 * 128,    // result slots
    SC_TOTAL = SC_NORM + 16
};

// ---------------------------------------------------------------------------
// Layout construction
// ---------------------------------------------------------------------------

// solve row tiers: one thread (<= kLongRow entries), one warp (<= kHugeSolve), one block
__host__ __device__ __forceinline__ int solve_tier(int64_t len) {
    return len <= kLongRow ? 0 : (len <= kHugeSolve ? 1 : 2);
}

__global__ void k_perm_keys(const int32_t *__restrict__ rp, const int32_t *__restrict__ colour,
                            int32_t n, uint32_t *__restrict__ key, int32_t *__restrict__ val) {
    int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    key[u] = (uint32_t)colour[u] * 3u + (uint32_t)solve_tier(rp[u + 1] - rp[u]);
    val[u] = u;
}

__global__ void k_invert(const int32_t *__restrict__ perm, int32_t n, int32_t *__restrict__ iperm) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) iperm[perm[i]] = i;
}

__global__ void k_key_hist(const uint32_t *__restrict__ key, int32_t n, int32_t *__restrict__ cnt) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&cnt[key[i]], 1);
}

__global__ void k_pdeg(const int32_t *__restrict__ rp, const int32_t *__restrict__ perm, int32_t n,
                       int32_t *__restrict__ deg) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) deg[i] = rp[perm[i] + 1] - rp[perm[i]];
    if (i == n) deg[n] = 0;
}

// entry-parallel copy of the CSR into permuted order
__global__ void k_permute_entries(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                  const double *__restrict__ w, const int32_t *__restrict__ iperm,
                                  const int32_t *__restrict__ prp, int32_t *__restrict__ pcol,
                                  double *__restrict__ pw64, float *__restrict__ pw32) {
    // one warp per natural row
    int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (wg >= n) return;
    int32_t u = (int32_t)wg;
    int32_t s = rp[u], e = rp[u + 1];
    int32_t d = prp[iperm[u]];
    for (int32_t j = s + lane; j < e; j += 32) {
        pcol[d + (j - s)] = iperm[col[j]];
        double x = w[j];
        pw64[d + (j - s)] = x;
        pw32[d + (j - s)] = (float)x;
    }
}

__global__ void k_tier_rows(const int32_t *__restrict__ ptr, int32_t n, int tier, uint8_t *__restrict__ f) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) f[i] = solve_tier(ptr[i + 1] - ptr[i]) == tier ? 1 : 0;
}

__global__ void k_pagg(const int32_t *__restrict__ perm, const int32_t *__restrict__ agg,
                       const int32_t *__restrict__ ciperm, int32_t n, uint32_t *__restrict__ key,
                       int32_t *__restrict__ pagg, int32_t *__restrict__ val) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t J = ciperm[agg[perm[i]]];
    pagg[i] = J;
    key[i] = (uint32_t)J;
    val[i] = i;
}

// Dense coarsest operator: M = A + (1/n) 1 1^T (SPD for a connected
// Laplacian; its inverse maps a zero-sum b to the zero-mean solution).  The
// inverse is formed by Gauss-Jordan elimination of [M | I] without pivoting
// (valid for SPD M), one all-SM launch per pivot, double-buffered so that
// every launch reads the previous step only.
__global__ void k_dense_assemble(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                 const double *__restrict__ w, double *__restrict__ G) {
    // G is n x 2n, row-major: [M | I]
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * 2 * n) return;
    const int32_t i = (int32_t)(q / (2 * n)), j = (int32_t)(q % (2 * n));
    double v;
    if (j >= n) {
        v = (j - n == i) ? 1.0 : 0.0;
    } else {
        v = 1.0 / (double)n;
        if (i == j) {
            double d = 0.0;
            for (int32_t e = rp[i]; e < rp[i + 1]; e++) d += w[e];
            v += d;
        } else {
            for (int32_t e = rp[i]; e < rp[i + 1]; e++)
                if (col[e] == j) v -= w[e];
        }
    }
    G[q] = v;
}

__global__ void k_gauss_jordan_step(int32_t n, int32_t k, const double *__restrict__ G, double *__restrict__ H,
                                    int32_t *err) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t W = 2 * (int64_t)n;
    if (q >= (int64_t)n * W) return;
    const int32_t i = (int32_t)(q / W);
    const int64_t j = q % W;
    const double piv = G[(int64_t)k * W + k];
    if (!(piv > 0.0)) {
        if (q == 0) *err = 1;
        H[q] = G[q];
        return;
    }
    const double pk = G[(int64_t)k * W + j] / piv;
    H[q] = (i == k) ? pk : G[q] - G[(int64_t)i * W + k] * pk;
}

__global__ void k_dense_extract(int32_t n, const double *__restrict__ G, double *__restrict__ Minv) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * n) return;
    const int32_t i = (int32_t)(q / n), j = (int32_t)(q % n);
    Minv[q] = G[(int64_t)i * 2 * n + n + j];
}

void build_solve_layout(lamg_ctx *h, cudaStream_t s) {
    const int L = h->L;
    h->lv.clear();
    h->lv.resize(L);
    std::vector<DBuf<int32_t>> iperm(L);
    for (int l = 0; l < L; l++) {
        SetupLevel &S = h->sl[l];
        SolveLevel &V = h->lv[l];
        const int32_t n = S.n;
        V.n = n;
        V.nnz = S.nnz;
        V.perm.alloc(n);
        iperm[l].alloc(n);
        const int nbins = 3 * S.ncolours;
        Tmp<uint32_t> key(n, s), ktmp(n, s);
        Tmp<int32_t> vtmp(n, s), cnt(nbins + 1, s), off(nbins + 1, s);
        k_perm_keys<<<ceil_div(n, 256), 256, 0, s>>>(S.rp.get(), S.colour.get(), n, key.get(), V.perm.get());
        LAMG_CHECK_LAUNCH();
        int nb = 0;
        while ((1ll << nb) < nbins) nb++;
        radix_sort_pairs<uint32_t, int32_t>(key.get(), V.perm.get(), ktmp.get(), vtmp.get(), n, nb, s);
        k_invert<<<ceil_div(n, 256), 256, 0, s>>>(V.perm.get(), n, iperm[l].get());
        LAMG_CHECK_LAUNCH();
        LAMG_CUDA(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t) * (nbins + 1), s));
        k_key_hist<<<ceil_div(n, 256), 256, 0, s>>>(key.get(), n, cnt.get());
        LAMG_CHECK_LAUNCH();
        exclusive_scan_i32(cnt.get(), off.get(), nbins + 1, s);
        std::vector<int32_t> hoff(nbins + 1);
        LAMG_CUDA(cudaMemcpyAsync(hoff.data(), off.get(), sizeof(int32_t) * (nbins + 1), cudaMemcpyDeviceToHost, s));
        LAMG_CUDA(cudaStreamSynchronize(s));
        V.cb.assign(4 * S.ncolours, 0);
        for (int c = 0; c < S.ncolours; c++)
            for (int t = 0; t < 4; t++) V.cb[4 * c + t] = hoff[3 * c + t];
        V.cb_dev.alloc(V.cb.size());
        LAMG_CUDA(cudaMemcpyAsync(V.cb_dev.get(), V.cb.data(), sizeof(int32_t) * V.cb.size(), cudaMemcpyHostToDevice, s));
        // permuted CSR
        Tmp<int32_t> deg(n + 1, s);
        V.rp.alloc(n + 1);
        V.col.alloc(S.nnz);
        V.w64.alloc(S.nnz);
        V.w32.alloc(S.nnz);
        k_pdeg<<<ceil_div(n + 1, 256), 256, 0, s>>>(S.rp.get(), V.perm.get(), n, deg.get());
        LAMG_CHECK_LAUNCH();
        exclusive_scan_i32(deg.get(), V.rp.get(), n + 1, s);
        if (S.nnz) {
            k_permute_entries<<<ceil_div((int64_t)n * 32, 256), 256, 0, s>>>(
                n, S.rp.get(), S.col.get(), S.w.get(), iperm[l].get(), V.rp.get(), V.col.get(),
                V.w64.get(), V.w32.get());
            LAMG_CHECK_LAUNCH();
        }
        // sweep plan: runs of colours without block-tier rows and few entries go
        // to one single-block launch (limits differ: FP64 throughput per SM is low)
        {
            std::vector<int32_t> hrp(n + 1);
            LAMG_CUDA(cudaMemcpyAsync(hrp.data(), V.rp.get(), sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, s));
            LAMG_CUDA(cudaStreamSynchronize(s));
            for (int p = 0; p < 2; p++) {
                const int64_t lim = p == 0 ? kTailWork64 : kTailWork32;
                auto small = [&](int c) {
                    return V.cb[4 * c + 3] == V.cb[4 * c + 2] &&
                           (int64_t)hrp[V.cb[4 * c + 3]] - hrp[V.cb[4 * c]] <= lim;
                };
                V.seg[p].clear();
                for (int c = 0; c < S.ncolours;) {
                    if (small(c)) {
                        int c1 = c;
                        while (c1 < S.ncolours && small(c1)) c1++;
                        V.seg[p].insert(V.seg[p].end(), {c, c1, 1});
                        c = c1;
                    } else {
                        V.seg[p].insert(V.seg[p].end(), {c, c + 1, 0});
                        c++;
                    }
                }
            }
        }
        Tmp<uint8_t> f(n, s);
        V.wrows.alloc(n);
        V.brows.alloc(n);
        k_tier_rows<<<ceil_div(n, 256), 256, 0, s>>>(V.rp.get(), n, 1, f.get());
        LAMG_CHECK_LAUNCH();
        V.nw = (int32_t)compact_indices(f.get(), V.wrows.get(), n, s);
        k_tier_rows<<<ceil_div(n, 256), 256, 0, s>>>(V.rp.get(), n, 2, f.get());
        LAMG_CHECK_LAUNCH();
        V.nb = (int32_t)compact_indices(f.get(), V.brows.get(), n, s);
    }
    for (int l = 0; l + 1 < L; l++) {
        SetupLevel &S = h->sl[l];
        SolveLevel &V = h->lv[l];
        const int32_t n = S.n, nc = S.nc;
        V.pagg.alloc(n);
        V.mptr.alloc(nc + 1);
        V.mlist.alloc(n);
        Tmp<uint32_t> key(n, s), ktmp(n, s);
        Tmp<int32_t> vtmp(n, s), cnt(nc + 1, s);
        k_pagg<<<ceil_div(n, 256), 256, 0, s>>>(V.perm.get(), S.agg.get(), iperm[l + 1].get(), n, key.get(),
                                                V.pagg.get(), V.mlist.get());
        LAMG_CHECK_LAUNCH();
        int nb = 0;
        while ((1ll << nb) < nc) nb++;
        radix_sort_pairs<uint32_t, int32_t>(key.get(), V.mlist.get(), ktmp.get(), vtmp.get(), n, nb, s);
        LAMG_CUDA(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t) * (nc + 1), s));
        k_key_hist<<<ceil_div(n, 256), 256, 0, s>>>(key.get(), n, cnt.get());
        LAMG_CHECK_LAUNCH();
        exclusive_scan_i32(cnt.get(), V.mptr.get(), nc + 1, s);
        Tmp<uint8_t> f(nc, s);
        V.wagg.alloc(nc);
        V.bagg.alloc(nc);
        k_tier_rows<<<ceil_div(nc, 256), 256, 0, s>>>(V.mptr.get(), nc, 1, f.get());
        LAMG_CHECK_LAUNCH();
        V.nwagg = (int32_t)compact_indices(f.get(), V.wagg.get(), nc, s);
        k_tier_rows<<<ceil_div(nc, 256), 256, 0, s>>>(V.mptr.get(), nc, 2, f.get());
        LAMG_CHECK_LAUNCH();
        V.nbagg = (int32_t)compact_indices(f.get(), V.bagg.get(), nc, s);
    }
    // coarsest level: dense inverse when small enough
    SolveLevel &C = h->lv[L - 1];
    if (C.n <= h->opt.dense_max) {
        const int32_t n = C.n;
        C.dense = 1;
        C.minv.alloc((size_t)n * n);
        Tmp<double> G((size_t)n * 2 * n, s), H((size_t)n * 2 * n, s);
        Tmp<int32_t> err(1, s);
        LAMG_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int32_t), s));
        const int64_t tot = (int64_t)n * 2 * n;
        k_dense_assemble<<<ceil_div(tot, 256), 256, 0, s>>>(n, C.rp.get(), C.col.get(), C.w64.get(), G.get());
        LAMG_CHECK_LAUNCH();
        double *a = G.get(), *bb = H.get();
        for (int32_t k = 0; k < n; k++) {
            k_gauss_jordan_step<<<ceil_div(tot, 256), 256, 0, s>>>(n, k, a, bb, err.get());
            LAMG_CHECK_LAUNCH();
            std::swap(a, bb);
        }
        k_dense_extract<<<ceil_div((int64_t)n * n, 256), 256, 0, s>>>(n, a, C.minv.get());
        LAMG_CHECK_LAUNCH();
        LAMG_REQUIRE(read_scalar(err.get(), s) == 0, LAMG_ERR_ARG,
                     "coarsest operator is not positive definite (disconnected graph?)");
    }
    LAMG_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------
// Cycle kernels (T = double or float)
// ---------------------------------------------------------------------------

// Tier helpers of the solve (any summation order is allowed here).
enum { M_THR = 0, M_WARP = 1, M_BLK = 2 };
template <int M> __device__ __forceinline__ int slane() {
    return M == M_THR ? 0 : (M == M_WARP ? (int)(threadIdx.x & 31) : (int)threadIdx.x);
}
template <int M> __device__ __forceinline__ int sstride() { return M == M_THR ? 1 : (M == M_WARP ? 32 : kBlk); }

template <class T>
__device__ __forceinline__ T warp_allsum(T v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// block sum of two values, result in every thread (blockDim = kBlk)
template <class T>
__device__ __forceinline__ void block_allsum2(T &a, T &b) {
    __shared__ T sa[32], sb[32];
    a = warp_allsum(a);
    b = warp_allsum(b);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) { sa[threadIdx.x >> 5] = a; sb[threadIdx.x >> 5] = b; }
    __syncthreads();
    a = T(0);
    b = T(0);
#pragma unroll 8
    for (int k = 0; k < kBlk / 32; k++) { a += sa[k]; b += sb[k]; }
}

template <int M, class T>
__device__ __forceinline__ void reduce2(T &a, T &b) {
    if (M == M_WARP) { a = warp_allsum(a); b = warp_allsum(b); }
    if (M == M_BLK) block_allsum2(a, b);
}

// Gauss-Seidel update of row i (Eq. (2.3)): x_i = (b_i + sum w x_v) / sum w.
template <int M, class T>
__device__ __forceinline__ void gs_row(int32_t i, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                       const T *__restrict__ w, const T *__restrict__ b, T *__restrict__ x) {
    const int32_t s = rp[i], e = rp[i + 1];
    T acc = T(0), d = T(0);
    for (int32_t j = s + slane<M>(); j < e; j += sstride<M>()) {
        const T wj = w[j];
        acc += wj * x[col[j]];
        d += wj;
    }
    reduce2<M>(acc, d);
    if (slane<M>() == 0) x[i] = (b[i] + acc) / d;
    if (M == M_BLK) __syncthreads();
}

// r_i = b_i - (A x)_i = b_i + sum_v w (x_v - x_i)
template <int M, class T>
__device__ __forceinline__ void resid_row(int32_t i, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                          const T *__restrict__ w, const T *__restrict__ b, const T *__restrict__ x,
                                          T *__restrict__ r) {
    const int32_t s = rp[i], e = rp[i + 1];
    const T xi = x[i];
    T acc = T(0), dummy = T(0);
    for (int32_t j = s + slane<M>(); j < e; j += sstride<M>()) acc += w[j] * (x[col[j]] - xi);
    reduce2<M>(acc, dummy);
    if (slane<M>() == 0) r[i] = b[i] + acc;
    if (M == M_BLK) __syncthreads();
}

// one colour's rows of a tier: THR/WARP/BLK over the contiguous range [row0, row0 + nrows)
template <int M, class T>
__global__ void __launch_bounds__(M == M_BLK ? kBlk : 256)
k_sweep(int32_t row0, int32_t nrows, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
        const T *__restrict__ w, const T *__restrict__ b, T *__restrict__ x) {
    int64_t k;
    if (M == M_THR) k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    else if (M == M_WARP) k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    else k = blockIdx.x;
    if (k >= nrows) return;
    gs_row<M, T>(row0 + (int32_t)k, rp, col, w, b, x);
}

// Colours c0 .. c1-1 of one sweep in a single block, colour by colour.
template <class T>
__global__ void __launch_bounds__(kBlk) k_sweep_tail(int32_t c0, int32_t c1, const int32_t *__restrict__ cb,
                                                    const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                                    const T *__restrict__ w, const T *__restrict__ b,
                                                    T *__restrict__ x) {
    const int warp = threadIdx.x >> 5;
    for (int32_t c = c0; c < c1; c++) {
        const int32_t t0 = cb[4 * c], t1 = cb[4 * c + 1], t2 = cb[4 * c + 2], t3 = cb[4 * c + 3];
        for (int32_t i = t0 + threadIdx.x; i < t1; i += kBlk) gs_row<M_THR, T>(i, rp, col, w, b, x);
        for (int32_t i = t1 + warp; i < t2; i += kBlk / 32) gs_row<M_WARP, T>(i, rp, col, w, b, x);
        for (int32_t i = t2; i < t3; i++) gs_row<M_BLK, T>(i, rp, col, w, b, x);
        __syncthreads();
    }
}

// residual: THR over all rows (skips the warp/block tiers), WARP/BLK over row lists
template <int M, class T>
__global__ void __launch_bounds__(M == M_BLK ? kBlk : 256)
k_resid(int32_t n, const int32_t *__restrict__ list, int32_t nlist, const int32_t *__restrict__ rp,
        const int32_t *__restrict__ col, const T *__restrict__ w, const T *__restrict__ b, const T *__restrict__ x,
        T *__restrict__ r) {
    int32_t i;
    if (M == M_THR) {
        const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (k >= n) return;
        i = (int32_t)k;
        if (rp[i + 1] - rp[i] > kLongRow) return;
    } else if (M == M_WARP) {
        const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        if (k >= nlist) return;
        i = list[k];
    } else {
        if (blockIdx.x >= nlist) return;
        i = list[blockIdx.x];
    }
    resid_row<M, T>(i, rp, col, w, b, x, r);
}

// b^c_J = mu * sum_{i in T_J} r_i ; x^c_J = 0   (Eq. (3.9))
template <int M, class T>
__global__ void __launch_bounds__(M == M_BLK ? kBlk : 256)
k_restrict(int32_t nc, const int32_t *__restrict__ list, int32_t nlist, const int32_t *__restrict__ mptr,
           const int32_t *__restrict__ mlist, const T *__restrict__ r, T mu, T *__restrict__ bc,
           T *__restrict__ xc) {
    int32_t J;
    if (M == M_THR) {
        const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (k >= nc) return;
        J = (int32_t)k;
        xc[J] = T(0);
        if (mptr[J + 1] - mptr[J] > kLongRow) return;
    } else if (M == M_WARP) {
        const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        if (k >= nlist) return;
        J = list[k];
    } else {
        if (blockIdx.x >= nlist) return;
        J = list[blockIdx.x];
    }
    T acc = T(0), dummy = T(0);
    for (int32_t j = mptr[J] + slane<M>(); j < mptr[J + 1]; j += sstride<M>()) acc += r[mlist[j]];
    reduce2<M>(acc, dummy);
    if (slane<M>() == 0) bc[J] = mu * acc;
}

// x_i += x^c_{agg(i)}   (Eq. (2.6))
template <class T>
__global__ void __launch_bounds__(256) k_prolong(int32_t n, const int32_t *__restrict__ pagg,
                                                 const T *__restrict__ xc, T *__restrict__ x) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += xc[pagg[i]];
}

template <class T>
__global__ void k_copy2(int32_t n, const T *__restrict__ a, T *__restrict__ a2, const T *__restrict__ c,
                        T *__restrict__ c2) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { a2[i] = a[i]; c2[i] = c[i]; }
}

template <class T>
__global__ void k_zero(int32_t n, T *__restrict__ a) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = T(0);
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[32];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    }
    return t;  // valid in thread 0
}

// Recombination dots (Eq. (3.13)): with d_i = r - r_i: G00, G01, G11, h0, h1.
template <class T>
__global__ void k_recomb_dots(int32_t n, const T *__restrict__ r, const T *__restrict__ r0,
                              const T *__restrict__ r1, int theta, double *__restrict__ part) {
    double g00 = 0, g01 = 0, g11 = 0, h0 = 0, h1 = 0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double ri = (double)r[i];
        const double d0 = ri - (double)r0[i];
        g00 += d0 * d0;
        h0 += ri * d0;
        if (theta == 2) {
            const double d1 = ri - (double)r1[i];
            g01 += d0 * d1;
            g11 += d1 * d1;
            h1 += ri * d1;
        }
    }
    double v[5] = {g00, g01, g11, h0, h1};
    for (int k = 0; k < 5; k++) {
        double t = block_sum(v[k]);
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * 8 + k] = t;
    }
}

__global__ void k_recomb_solve(const double *__restrict__ part, int nblocks, int theta,
                               double *__restrict__ alpha) {
    double s[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < 5; k++) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += part[(int64_t)b * 8 + k];
        v = block_sum(v);
        if (threadIdx.x == 0) s[k] = v;
    }
    if (threadIdx.x != 0) return;
    const double G00 = s[0], G01 = s[1], G11 = s[2], h0 = s[3], h1 = s[4];
    double a0 = 0.0, a1 = 0.0;
    if (theta == 1) {
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
    alpha[0] = a0;
    alpha[1] = a1;
}

template <class T>
__global__ void k_recomb_apply(int32_t n, T *__restrict__ x, const T *__restrict__ x0,
                               const T *__restrict__ x1, int theta, const double *__restrict__ alpha) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double xi = (double)x[i];
    double y = xi + alpha[0] * ((double)x0[i] - xi);
    if (theta == 2) y += alpha[1] * ((double)x1[i] - xi);
    x[i] = (T)y;
}

// Coarsest solve: x = M^-1 b in FP64 (warp per row), M^-1 b is zero-mean for zero-sum b.
template <class T>
__global__ void k_coarse_gemv(int32_t n, const double *__restrict__ minv, const T *__restrict__ b,
                              T *__restrict__ x) {
    const int32_t wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wg >= n) return;
    double acc = 0.0;
    for (int32_t j = lane; j < n; j += 32) acc += minv[(int64_t)wg * n + j] * (double)b[j];
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if (lane == 0) x[wg] = (T)acc;
}

// Sum (deterministic block partials) for the mean and norms.
template <class T>
__global__ void k_partial_sum(int32_t n, const T *__restrict__ a, double *__restrict__ part) {
    double v = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v += (double)a[i];
    v = block_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

template <class T>
__global__ void k_partial_sumsq(int32_t n, const T *__restrict__ a, double *__restrict__ part) {
    double v = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double t = (double)a[i];
        v += t * t;
    }
    v = block_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

template <class T>
__global__ void k_partial_abssum(int32_t n, const T *__restrict__ a, double *__restrict__ part) {
    double v = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v += fabs((double)a[i]);
    v = block_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

__global__ void k_finish_sum(const double *__restrict__ part, int nb, double *__restrict__ out) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[b];
    v = block_sum(v);
    if (threadIdx.x == 0) *out = v;
}

template <class T>
__global__ void k_sub_mean(int32_t n, T *__restrict__ x, const double *__restrict__ sum) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = (T)((double)x[i] - *sum / (double)n);
}

// FP64 refinement helpers
__global__ void k_d2f(int32_t n, const double *__restrict__ a, float *__restrict__ o) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) o[i] = (float)a[i];
}

__global__ void k_add_f2d(int32_t n, double *__restrict__ x, const float *__restrict__ e) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += (double)e[i];
}

// natural <-> permuted order for level-1 vectors
__global__ void k_gather_perm(int32_t n, const int32_t *__restrict__ perm, const double *__restrict__ src,
                              double *__restrict__ dst) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[perm[i]];
}

__global__ void k_scatter_perm(int32_t n, const int32_t *__restrict__ perm, const double *__restrict__ src,
                               double *__restrict__ dst) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[perm[i]] = src[i];
}

// ---------------------------------------------------------------------------
// Cycle issue (host recursion over a fixed schedule)
// ---------------------------------------------------------------------------

template <class T> struct Prec;
template <> struct Prec<double> {
    static const double *w(const SolveLevel &V) { return V.w64.get(); }
    static std::vector<LevelVecs<double>> &vecs(lamg_ctx *h) { return h->v64; }
};
template <> struct Prec<float> {
    static const float *w(const SolveLevel &V) { return V.w32.get(); }
    static std::vector<LevelVecs<float>> &vecs(lamg_ctx *h) { return h->v32; }
};

template <class T>
static void ensure_vecs(lamg_ctx *h) {
    auto &vv = Prec<T>::vecs(h);
    if (!vv.empty()) return;
    vv.resize(h->L);
    for (int l = 0; l < h->L; l++) {
        const int32_t n = h->lv[l].n;
        vv[l].x.alloc(n);
        vv[l].b.alloc(n);
        vv[l].r.alloc(n);
        if (l >= 1 && l + 1 < h->L) {
            vv[l].xs0.alloc(n); vv[l].xs1.alloc(n);
            vv[l].rs0.alloc(n); vv[l].rs1.alloc(n);
        }
    }
    if (!h->scratch.get()) h->scratch.alloc(SC_TOTAL);
}

struct IssueCtx {
    lamg_ctx *h;
    int adaptive;
    double mu;
    cudaStream_t s;
    std::vector<int32_t> visits;
    bool profile;
    int prof_idx;
};

template <class T>
static void sweep(IssueCtx &c, int l, const T *b, T *x) {
    const SolveLevel &V = c.h->lv[l];
    const T *w = Prec<T>::w(V);
    const bool prof = c.profile && l == 0;
    if (prof) LAMG_CUDA(cudaEventRecordWithFlags(c.h->prof_ev[2 * c.prof_idx], c.s, cudaEventRecordExternal));
    const std::vector<int32_t> &seg = V.seg[sizeof(T) == 8 ? 0 : 1];
    for (size_t q = 0; q < seg.size(); q += 3) {
        const int k = seg[q];
        if (seg[q + 2]) {
            k_sweep_tail<T><<<1, kBlk, 0, c.s>>>(seg[q], seg[q + 1], V.cb_dev.get(), V.rp.get(), V.col.get(), w, b, x);
            LAMG_CHECK_LAUNCH();
            continue;
        }
        const int32_t t0 = V.cb[4 * k], t1 = V.cb[4 * k + 1], t2 = V.cb[4 * k + 2], t3 = V.cb[4 * k + 3];
        if (t1 > t0) {
            k_sweep<M_THR, T><<<ceil_div(t1 - t0, 256), 256, 0, c.s>>>(t0, t1 - t0, V.rp.get(), V.col.get(), w, b, x);
            LAMG_CHECK_LAUNCH();
        }
        if (t2 > t1) {
            k_sweep<M_WARP, T><<<ceil_div((int64_t)(t2 - t1) * 32, 256), 256, 0, c.s>>>(t1, t2 - t1, V.rp.get(),
                                                                                       V.col.get(), w, b, x);
            LAMG_CHECK_LAUNCH();
        }
        if (t3 > t2) {
            k_sweep<M_BLK, T><<<t3 - t2, kBlk, 0, c.s>>>(t2, t3 - t2, V.rp.get(), V.col.get(), w, b, x);
            LAMG_CHECK_LAUNCH();
        }
    }
    if (prof) {
        LAMG_CUDA(cudaEventRecordWithFlags(c.h->prof_ev[2 * c.prof_idx + 1], c.s, cudaEventRecordExternal));
        c.prof_idx++;
    }
}

template <class T>
static void residual(IssueCtx &c, int l, const T *b, const T *x, T *r) {
    const SolveLevel &V = c.h->lv[l];
    const T *w = Prec<T>::w(V);
    k_resid<M_THR, T><<<ceil_div(V.n, 256), 256, 0, c.s>>>(V.n, nullptr, 0, V.rp.get(), V.col.get(), w, b, x, r);
    LAMG_CHECK_LAUNCH();
    if (V.nw) {
        k_resid<M_WARP, T><<<ceil_div((int64_t)V.nw * 32, 256), 256, 0, c.s>>>(0, V.wrows.get(), V.nw, V.rp.get(),
                                                                              V.col.get(), w, b, x, r);
        LAMG_CHECK_LAUNCH();
    }
    if (V.nb) {
        k_resid<M_BLK, T><<<V.nb, kBlk, 0, c.s>>>(0, V.brows.get(), V.nb, V.rp.get(), V.col.get(), w, b, x, r);
        LAMG_CHECK_LAUNCH();
    }
}

template <class T>
static void restrict_to(IssueCtx &c, int l, const T *r, T *bc, T *xc) {
    const SolveLevel &F = c.h->lv[l];
    const int32_t nc = c.h->lv[l + 1].n;
    const T mu = (T)c.mu;
    k_restrict<M_THR, T><<<ceil_div(nc, 256), 256, 0, c.s>>>(nc, nullptr, 0, F.mptr.get(), F.mlist.get(), r, mu, bc,
                                                            xc);
    LAMG_CHECK_LAUNCH();
    if (F.nwagg) {
        k_restrict<M_WARP, T><<<ceil_div((int64_t)F.nwagg * 32, 256), 256, 0, c.s>>>(
            0, F.wagg.get(), F.nwagg, F.mptr.get(), F.mlist.get(), r, mu, bc, xc);
        LAMG_CHECK_LAUNCH();
    }
    if (F.nbagg) {
        k_restrict<M_BLK, T><<<F.nbagg, kBlk, 0, c.s>>>(0, F.bagg.get(), F.nbagg, F.mptr.get(), F.mlist.get(), r, mu,
                                                        bc, xc);
        LAMG_CHECK_LAUNCH();
    }
}

template <class T>
static void coarsest_solve(IssueCtx &c, int l, const T *b, T *x) {
    const SolveLevel &V = c.h->lv[l];
    if (V.dense) {
        k_coarse_gemv<T><<<ceil_div((int64_t)V.n * 32, 256), 256, 0, c.s>>>(V.n, V.minv.get(), b, x);
        LAMG_CHECK_LAUNCH();
        return;
    }
    k_zero<T><<<ceil_div(V.n, 256), 256, 0, c.s>>>(V.n, x);
    LAMG_CHECK_LAUNCH();
    for (int k = 0; k < c.h->opt.coarse_sweeps; k++) sweep<T>(c, l, b, x);
}

// One visit to level l with theta two-level steps (Fig. 4.2); see the oracle
// for the schedule: the k-th coarse correction of level l (k counted from 0
// within the cycle) runs ceil((k+1) g) - ceil(k g) visits, g = gamma^l.
template <class T>
static void visit(IssueCtx &c, int l, int theta) {
    lamg_ctx *h = c.h;
    const SolveLevel &F = h->lv[l], &C = h->lv[l + 1];
    auto &vv = Prec<T>::vecs(h);
    LevelVecs<T> &vf = vv[l], &vc = vv[l + 1];
    const bool recomb = c.adaptive && l >= 1;
    const lamg_options &o = h->opt;
    for (int i = 0; i < theta; i++) {
        for (int k = 0; k < o.nu1; k++) sweep<T>(c, l, vf.b.get(), vf.x.get());
        residual<T>(c, l, vf.b.get(), vf.x.get(), vf.r.get());
        if (recomb) {
            T *xs = i == 0 ? vf.xs0.get() : vf.xs1.get();
            T *rs = i == 0 ? vf.rs0.get() : vf.rs1.get();
            k_copy2<T><<<ceil_div(F.n, 256), 256, 0, c.s>>>(F.n, vf.x.get(), xs, vf.r.get(), rs);
            LAMG_CHECK_LAUNCH();
        }
        restrict_to<T>(c, l, vf.r.get(), vc.b.get(), vc.x.get());
        if (l + 1 == h->L - 1) {
            coarsest_solve<T>(c, l + 1, vc.b.get(), vc.x.get());
        } else {
            const int32_t k = c.visits[l]++;
            const double g = h->sl[l].gamma_l;
            int th = (int)(std::ceil((double)(k + 1) * g) - std::ceil((double)k * g));
            th = th < 1 ? 1 : (th > 2 ? 2 : th);
            visit<T>(c, l + 1, th);
        }
        k_prolong<T><<<ceil_div(F.n, 256), 256, 0, c.s>>>(F.n, F.pagg.get(), vc.x.get(), vf.x.get());
        LAMG_CHECK_LAUNCH();
        for (int k = 0; k < o.nu2; k++) sweep<T>(c, l, vf.b.get(), vf.x.get());
    }
    if (recomb) {
        residual<T>(c, l, vf.b.get(), vf.x.get(), vf.r.get());
        double *part = h->scratch.get() + SC_PART;
        double *alpha = h->scratch.get() + SC_ALPHA + 2 * l;
        k_recomb_dots<T><<<kRedBlocks, kRedThreads, 0, c.s>>>(F.n, vf.r.get(), vf.rs0.get(), vf.rs1.get(), theta,
                                                              part);
        LAMG_CHECK_LAUNCH();
        k_recomb_solve<<<1, 256, 0, c.s>>>(part, kRedBlocks, theta, alpha);
        LAMG_CHECK_LAUNCH();
        k_recomb_apply<T><<<ceil_div(F.n, 256), 256, 0, c.s>>>(F.n, vf.x.get(), vf.xs0.get(), vf.xs1.get(), theta,
                                                              alpha);
        LAMG_CHECK_LAUNCH();
    }
}

template <class T>
static void subtract_mean(IssueCtx &c, int32_t n, T *x) {
    double *part = c.h->scratch.get() + SC_PART;
    double *out = c.h->scratch.get() + SC_NORM + 1;
    k_partial_sum<T><<<kRedBlocks, kRedThreads, 0, c.s>>>(n, x, part);
    LAMG_CHECK_LAUNCH();
    k_finish_sum<<<1, 256, 0, c.s>>>(part, kRedBlocks, out);
    LAMG_CHECK_LAUNCH();
    k_sub_mean<T><<<ceil_div(n, 256), 256, 0, c.s>>>(n, x, out);
    LAMG_CHECK_LAUNCH();
}

// One cycle on level-1 vectors vv[0].x / vv[0].b, then the mean subtraction M.
template <class T>
static void issue_cycle(IssueCtx &c) {
    lamg_ctx *h = c.h;
    auto &vv = Prec<T>::vecs(h);
    c.visits.assign(h->L, 0);
    if (h->L == 1) {
        coarsest_solve<T>(c, 0, vv[0].b.get(), vv[0].x.get());
    } else {
        visit<T>(c, 0, 1);
    }
    subtract_mean<T>(c, h->lv[0].n, vv[0].x.get());
}

// ||b - A x||^2 in FP64 at level 1 into scratch[SC_NORM] and the pinned slot.
static void issue_resnorm64(IssueCtx &c, const double *b, const double *x, double *r) {
    lamg_ctx *h = c.h;
    residual<double>(c, 0, b, x, r);
    double *part = h->scratch.get() + SC_PART;
    k_partial_sumsq<double><<<kRedBlocks, kRedThreads, 0, c.s>>>(h->lv[0].n, r, part);
    LAMG_CHECK_LAUNCH();
    k_finish_sum<<<1, 256, 0, c.s>>>(part, kRedBlocks, h->scratch.get() + SC_NORM);
    LAMG_CHECK_LAUNCH();
    LAMG_CUDA(cudaMemcpyAsync(h->host_pinned, h->scratch.get() + SC_NORM, sizeof(double), cudaMemcpyDeviceToHost, c.s));
}

// ---------------------------------------------------------------------------
// Graph capture of one step: FP64 = cycle + residual norm; FP32-IR = convert,
// ir_inner FP32 cycles, update, projection, FP64 residual norm.
// ---------------------------------------------------------------------------

static void issue_step(lamg_ctx *h, lamg_precision p, int adaptive, bool profile, cudaStream_t s) {
    IssueCtx c{h, adaptive, adaptive ? 1.0 : h->opt.mu_flat, s, {}, profile, 0};
    const int32_t n = h->lv[0].n;
    if (p == LAMG_FP64) {
        issue_cycle<double>(c);
        issue_resnorm64(c, h->v64[0].b.get(), h->v64[0].x.get(), h->r64.get());
    } else {
        k_d2f<<<ceil_div(n, 256), 256, 0, s>>>(n, h->r64.get(), h->v32[0].b.get());
        LAMG_CHECK_LAUNCH();
        k_zero<float><<<ceil_div(n, 256), 256, 0, s>>>(n, h->v32[0].x.get());
        LAMG_CHECK_LAUNCH();
        for (int k = 0; k < std::max(1, h->opt.ir_inner); k++) issue_cycle<float>(c);
        k_add_f2d<<<ceil_div(n, 256), 256, 0, s>>>(n, h->v64[0].x.get(), h->v32[0].x.get());
        LAMG_CHECK_LAUNCH();
        subtract_mean<double>(c, n, h->v64[0].x.get());
        issue_resnorm64(c, h->v64[0].b.get(), h->v64[0].x.get(), h->r64.get());
    }
}

static int events_per_step(lamg_ctx *h, lamg_precision p) {
    if (h->L == 1) return 0;
    const int per_cycle = h->opt.nu1 + h->opt.nu2;
    return p == LAMG_FP64 ? per_cycle : per_cycle * std::max(1, h->opt.ir_inner);
}

static cudaGraphExec_t get_graph(lamg_ctx *h, lamg_precision p, int adaptive) {
    const bool prof = h->prof_on != 0;
    cudaGraphExec_t *slot;
    int32_t *slot_ad;
    if (p == LAMG_FP64) { slot = prof ? &h->g64p : &h->g64; slot_ad = prof ? &h->g64p_adaptive : &h->g64_adaptive; }
    else { slot = prof ? &h->g32p : &h->g32; slot_ad = prof ? &h->g32p_adaptive : &h->g32_adaptive; }
    if (*slot && *slot_ad == adaptive) return *slot;
    if (*slot) { cudaGraphExecDestroy(*slot); *slot = nullptr; }
    if (prof) {
        const int ne = 2 * events_per_step(h, p);
        while ((int)h->prof_ev.size() < ne) {
            cudaEvent_t e;
            LAMG_CUDA(cudaEventCreate(&e));
            h->prof_ev.push_back(e);
        }
    }
    cudaStream_t cs = h->cap_stream;
    cudaGraph_t g;
    LAMG_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    begin_capture_count();
    try {
        issue_step(h, p, adaptive, prof, cs);
    } catch (...) {
        end_capture_count();
        cudaStreamEndCapture(cs, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    const int64_t kernels = end_capture_count();
    LAMG_CUDA(cudaStreamEndCapture(cs, &g));
    cudaGraphExec_t ge;
    cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    LAMG_CUDA(e);
    *slot = ge;
    *slot_ad = adaptive;
    (p == LAMG_FP64 ? (prof ? h->g64p_kernels : h->g64_kernels) : (prof ? h->g32p_kernels : h->g32_kernels)) = kernels;
    return ge;
}

static void prepare(lamg_ctx *h, lamg_precision p) {
    ensure_vecs<double>(h);
    if (p == LAMG_FP32_IR) ensure_vecs<float>(h);
    if (!h->r64.get()) h->r64.alloc(h->lv[0].n);
    if (!h->host_pinned) LAMG_CUDA(cudaMallocHost((void **)&h->host_pinned, 16 * sizeof(double)));
    if (!h->cap_stream) LAMG_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
}

static void accumulate_profile(lamg_ctx *h, lamg_precision p) {
    if (!h->prof_on) return;
    const int ne = events_per_step(h, p);
    for (int k = 0; k < ne; k++) {
        float ms = 0.f;
        LAMG_CUDA(cudaEventElapsedTime(&ms, h->prof_ev[2 * k], h->prof_ev[2 * k + 1]));
        h->prof_ms += ms;
        h->prof_count++;
    }
    const int64_t wb = p == LAMG_FP64 ? 8 : 4;
    const SolveLevel &V = h->lv[0];
    // one finest-level sweep: entries (col + w), row pointers, b, x read + write
    h->prof_bytes = V.nnz * (4 + wb) + (int64_t)(V.n + 1) * 4 + (int64_t)V.n * wb * 3;
}

// sum, ||b||_1 and ||b||_2 of the FP64 right-hand side (zero-sum check, Sec. 1).
static void rhs_norms(lamg_ctx *h, const double *b, cudaStream_t s, double &sum, double &asum, double &nrm) {
    const int32_t n = h->lv[0].n;
    double *part = h->scratch.get() + SC_PART;
    double *out = h->scratch.get() + SC_NORM + 4;
    k_partial_sum<double><<<kRedBlocks, kRedThreads, 0, s>>>(n, b, part);
    LAMG_CHECK_LAUNCH();
    k_finish_sum<<<1, 256, 0, s>>>(part, kRedBlocks, out);
    LAMG_CHECK_LAUNCH();
    k_partial_abssum<double><<<kRedBlocks, kRedThreads, 0, s>>>(n, b, part);
    LAMG_CHECK_LAUNCH();
    k_finish_sum<<<1, 256, 0, s>>>(part, kRedBlocks, out + 1);
    LAMG_CHECK_LAUNCH();
    k_partial_sumsq<double><<<kRedBlocks, kRedThreads, 0, s>>>(n, b, part);
    LAMG_CHECK_LAUNCH();
    k_finish_sum<<<1, 256, 0, s>>>(part, kRedBlocks, out + 2);
    LAMG_CHECK_LAUNCH();
    double hv[3];
    LAMG_CUDA(cudaMemcpyAsync(hv, out, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    LAMG_CUDA(cudaStreamSynchronize(s));
    sum = hv[0];
    asum = hv[1];
    nrm = std::sqrt(hv[2]);
}

void solve_device(lamg_ctx *h, const double *b, double *x, double tol, lamg_precision p, cudaStream_t s,
                  lamg_stats *st) {
    auto t0 = std::chrono::steady_clock::now();
    prepare(h, p);
    const int32_t n = h->lv[0].n;
    const SolveLevel &V0 = h->lv[0];
    double *xb = h->v64[0].x.get(), *bb = h->v64[0].b.get();
    k_gather_perm<<<ceil_div(n, 256), 256, 0, s>>>(n, V0.perm.get(), b, bb);
    LAMG_CHECK_LAUNCH();
    k_gather_perm<<<ceil_div(n, 256), 256, 0, s>>>(n, V0.perm.get(), x, xb);
    LAMG_CHECK_LAUNCH();
    double sb, ab, bn;
    rhs_norms(h, bb, s, sb, ab, bn);
    LAMG_REQUIRE(std::fabs(sb) <= 1e-10 * (ab > 0 ? ab : 1.0), LAMG_ERR_RHS_NOT_ZERO_SUM,
                 "right-hand side is not zero-sum");
    // initial residual
    IssueCtx c{h, h->opt.adaptive, 1.0, s, {}, false, 0};
    issue_resnorm64(c, bb, xb, h->r64.get());
    LAMG_CUDA(cudaStreamSynchronize(s));
    double r0 = std::sqrt(*h->host_pinned), rn = r0;
    const int adaptive = h->opt.adaptive;
    cudaGraphExec_t ge = nullptr;
    int steps = 0, cycles = 0;
    const int per_step = p == LAMG_FP64 ? 1 : std::max(1, h->opt.ir_inner);
    while (rn > tol * bn && cycles < h->opt.max_cycles) {
        if (!ge) ge = get_graph(h, p, adaptive);
        LAMG_CUDA(cudaGraphLaunch(ge, s));
        note_graph_launch(p == LAMG_FP64 ? (h->prof_on ? h->g64p_kernels : h->g64_kernels)
                                         : (h->prof_on ? h->g32p_kernels : h->g32_kernels));
        LAMG_CUDA(cudaStreamSynchronize(s));
        accumulate_profile(h, p);
        rn = std::sqrt(*h->host_pinned);
        steps++;
        cycles += per_step;
        if (!(rn == rn)) break;  // NaN: stop
    }
    k_scatter_perm<<<ceil_div(n, 256), 256, 0, s>>>(n, V0.perm.get(), xb, x);
    LAMG_CHECK_LAUNCH();
    LAMG_CUDA(cudaStreamSynchronize(s));
    auto t1 = std::chrono::steady_clock::now();
    lamg_stats &L = h->last;
    L.levels = h->L;
    L.cycles = cycles;
    L.outer_steps = steps;
    L.rel_res = bn > 0 ? rn / bn : 0.0;
    L.acf = (cycles > 0 && r0 > 0 && rn > 0) ? std::pow(rn / r0, 1.0 / cycles) : 0.0;
    L.t_setup_s = h->t_setup_s;
    L.t_solve_s = std::chrono::duration<double>(t1 - t0).count();
    L.status = (rn <= tol * bn) ? LAMG_OK : LAMG_ERR_NOT_CONVERGED;
    if (st) *st = L;
    LAMG_REQUIRE(rn == rn, LAMG_ERR_NOT_CONVERGED, "solve produced NaN");
    if (L.status != LAMG_OK) throw Error{LAMG_ERR_NOT_CONVERGED, "max_cycles reached before tol"};
}

void cycle_device(lamg_ctx *h, const double *b, double *x, int32_t adaptive, cudaStream_t s) {
    prepare(h, LAMG_FP64);
    const int32_t n = h->lv[0].n;
    const SolveLevel &V0 = h->lv[0];
    k_gather_perm<<<ceil_div(n, 256), 256, 0, s>>>(n, V0.perm.get(), b, h->v64[0].b.get());
    LAMG_CHECK_LAUNCH();
    k_gather_perm<<<ceil_div(n, 256), 256, 0, s>>>(n, V0.perm.get(), x, h->v64[0].x.get());
    LAMG_CHECK_LAUNCH();
    IssueCtx c{h, adaptive, adaptive ? 1.0 : h->opt.mu_flat, s, {}, false, 0};
    issue_cycle<double>(c);
    k_scatter_perm<<<ceil_div(n, 256), 256, 0, s>>>(n, V0.perm.get(), h->v64[0].x.get(), x);
    LAMG_CHECK_LAUNCH();
    LAMG_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------
// Adjoint: lambda = A^+ (g - mean g), dw_e = -(lambda_u - lambda_v)(x_u - x_v)
// ---------------------------------------------------------------------------

__global__ void k_edge_grad(int64_t m, const int32_t *__restrict__ eu, const int32_t *__restrict__ ev,
                            const double *__restrict__ lam, const double *__restrict__ x, void *dw, int32_t dw32) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int32_t u = eu[e], v = ev[e];
    const double g = -(lam[u] - lam[v]) * (x[u] - x[v]);
    if (dw32) ((float *)dw)[e] = (float)g; else ((double *)dw)[e] = g;
}

__global__ void k_center(int32_t n, const double *__restrict__ g, double *__restrict__ out,
                         const double *__restrict__ sum) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = g[i] - *sum / (double)n;
}

void adjoint_device(lamg_ctx *h, const double *x, const double *g, double *lambda, const int32_t *eu,
                    const int32_t *ev, int64_t m, void *dw, int32_t dw32, double tol, lamg_precision p,
                    cudaStream_t s, lamg_stats *st) {
    prepare(h, p);
    const int32_t n = h->lv[0].n;
    Tmp<double> gz(n, s);
    double *part = h->scratch.get() + SC_PART;
    double *out = h->scratch.get() + SC_NORM + 8;
    k_partial_sum<double><<<kRedBlocks, kRedThreads, 0, s>>>(n, g, part);
    LAMG_CHECK_LAUNCH();
    k_finish_sum<<<1, 256, 0, s>>>(part, kRedBlocks, out);
    LAMG_CHECK_LAUNCH();
    k_center<<<ceil_div(n, 256), 256, 0, s>>>(n, g, gz.get(), out);
    LAMG_CHECK_LAUNCH();
    LAMG_CUDA(cudaMemsetAsync(lambda, 0, sizeof(double) * n, s));
    LAMG_CHECK_LAUNCH();
    solve_device(h, gz.get(), lambda, tol, p, s, st);
    if (dw && m > 0) {
        k_edge_grad<<<ceil_div(m, 256), 256, 0, s>>>(m, eu, ev, lambda, x, dw, dw32);
        LAMG_CHECK_LAUNCH();
    }
    LAMG_CUDA(cudaStreamSynchronize(s));
}

void solve_batched_device(lamg_ctx *h, int32_t nrhs, const double *B, double *X, int64_t ld, double tol,
                          lamg_precision p, cudaStream_t s, lamg_stats *st) {
    throw Error{LAMG_ERR_ARG, "lamg_solve_batched: not built yet"};
}

void release_solve(lamg_ctx *h) {
    if (h->g64) cudaGraphExecDestroy(h->g64);
    if (h->g32) cudaGraphExecDestroy(h->g32);
    if (h->g64p) cudaGraphExecDestroy(h->g64p);
    if (h->g32p) cudaGraphExecDestroy(h->g32p);
    h->g64 = h->g32 = h->g64p = h->g32p = nullptr;
    for (auto e : h->prof_ev) cudaEventDestroy(e);
    h->prof_ev.clear();
    if (h->host_pinned) cudaFreeHost(h->host_pinned);
    h->host_pinned = nullptr;
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
}

}  // namespace lamg
