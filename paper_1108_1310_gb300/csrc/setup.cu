// setup.cu -- the LAMG setup phase on the GPU (Sec. 4.1 of Livne & Brandt,
// arXiv 1108.1310): colouring, test-vector relaxation (Sec. 3.3.1), affinity
// (Eq. (3.5)) and energy ratio (Eq. (3.12)) per edge, hubs (Sec. 3.4.1),
// aggregation stages (Sec. 3.4.2), Galerkin coarse operator (Eq. (2.5)).
//
// Every floating-point value that feeds an integer decision is computed in
// FP64 with a fixed operation order (this translation unit is compiled with
// -fmad=false, so no multiply-add is contracted).  A row (or segment) of
// `len` terms is summed
//  * len <= 32   by one thread, left to right from +0.0;
//  * len <= 512  by one warp: lane j sums terms j, j+32, ... left to right,
//    then p_j += p_{j+h} for h = 16, 8, 4, 2, 1 (shfl_down); lane 0's value;
//  * len  > 512  by a 1024-thread block: thread j sums j, j+1024, ...; each
//    warp reduces its 32 partials by the same halving tree, then warp 0
//    reduces the 32 warp results by it again.
// Kernels are therefore templated on the row tier M (thread / warp / block).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "lamg_internal.cuh"

namespace lamg {

constexpr unsigned kFull = 0xffffffffu;
enum { ST_U = 0, ST_S = 1, ST_A = 2, ST_D = 3 };
enum { M_THR = 0, M_WARP = 1, M_BLK = 2 };

// ---------------------------------------------------------------------------
// splitmix64 (Steele, Lea & Flood 2014): first output of the generator seeded
// with `key`.  Used as a counter-based generator: value(key + counter).
// ---------------------------------------------------------------------------

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t key) {
    uint64_t z = key + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static uint64_t colour_key(uint64_t seed, int level) {
    return splitmix64(splitmix64(seed) ^ (0x100000000ULL * (uint64_t)(2 * level + 1)));
}
static uint64_t tv_key(uint64_t seed, int level) {
    return splitmix64(splitmix64(seed) ^ (0x100000000ULL * (uint64_t)(2 * level + 2)));
}
// elimination sweep order: the colour key's form with the top bit set
static uint64_t elim_key(uint64_t seed, int level) {
    return splitmix64(splitmix64(seed) ^ (0x100000000ULL * (uint64_t)(2 * level + 1)) ^ (1ULL << 63));
}
// aggregation scan order (agg_rule 2): the TV key's form with the top bit set
static uint64_t agg_key(uint64_t seed, int level) {
    return splitmix64(splitmix64(seed) ^ (0x100000000ULL * (uint64_t)(2 * level + 2)) ^ (1ULL << 63));
}

// ---------------------------------------------------------------------------
// Tier helpers
// ---------------------------------------------------------------------------

__host__ __device__ __forceinline__ int row_tier(int64_t len) {
    return len <= kLongRow ? 0 : (len <= kHugeRow ? 1 : 2);
}

template <int M> __device__ __forceinline__ int tlane() {
    return M == M_THR ? 0 : (M == M_WARP ? (int)(threadIdx.x & 31) : (int)threadIdx.x);
}
template <int M> __device__ __forceinline__ int tstride() { return M == M_THR ? 1 : (M == M_WARP ? 32 : kBlk); }

__device__ __forceinline__ double warp_tree(double p) {
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) p = p + __shfl_down_sync(kFull, p, h);
    return __shfl_sync(kFull, p, 0);
}

// Canonical reduction of the tier's partial sums; result in every thread.
template <int M>
__device__ __forceinline__ double canon_reduce(double p) {
    if (M == M_THR) return p;
    p = warp_tree(p);
    if (M == M_WARP) return p;
    __shared__ double red[33];
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = p;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = warp_tree(red[threadIdx.x]);
        if (threadIdx.x == 0) red[32] = v;
    }
    __syncthreads();
    return red[32];
}

template <int M>
__device__ __forceinline__ int32_t reduce_sum_i32(int32_t v) {
    if (M == M_THR) return v;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (M == M_WARP) return v;
    __shared__ int32_t red[33];
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        int32_t t = red[threadIdx.x];
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
        if (threadIdx.x == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

template <int M>
__device__ __forceinline__ double reduce_max(double v) {
    if (M == M_THR) return v;
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    if (M == M_WARP) return v;
    __shared__ double red[33];
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = red[threadIdx.x];
        for (int o = 16; o; o >>= 1) t = fmax(t, __shfl_xor_sync(kFull, t, o));
        if (threadIdx.x == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

template <int M>
__device__ __forceinline__ bool reduce_any(bool v) {
    if (M == M_THR) return v;
    if (M == M_WARP) return __any_sync(kFull, v);
    return __syncthreads_or(v) != 0;
}

template <int M>
__device__ __forceinline__ bool reduce_all(bool v) {
    if (M == M_THR) return v;
    if (M == M_WARP) return __all_sync(kFull, v);
    return __syncthreads_and(v) != 0;
}

template <int M>
__device__ __forceinline__ unsigned long long reduce_or64(unsigned long long v) {
    if (M == M_THR) return v;
    for (int o = 16; o; o >>= 1) v |= __shfl_xor_sync(kFull, v, o);
    if (M == M_WARP) return v;
    __shared__ unsigned long long red[33];
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned long long t = red[threadIdx.x];
        for (int o = 16; o; o >>= 1) t |= __shfl_xor_sync(kFull, t, o);
        if (threadIdx.x == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// best = largest score, ties -> smaller neighbour; v < 0 means none
__device__ __forceinline__ void best_merge(double &bs, int32_t &bv, double os, int32_t ov) {
    if (ov >= 0 && (bv < 0 || os > bs || (os == bs && ov < bv))) { bs = os; bv = ov; }
}

template <int M>
__device__ __forceinline__ int32_t reduce_best(double bs, int32_t bv) {
    if (M == M_THR) return bv;
    for (int o = 16; o; o >>= 1) {
        const double os = __shfl_xor_sync(kFull, bs, o);
        const int32_t ov = __shfl_xor_sync(kFull, bv, o);
        best_merge(bs, bv, os, ov);
    }
    if (M == M_WARP) return bv;
    __shared__ double rs[32];
    __shared__ int32_t rv[33];
    __syncthreads();
    if ((threadIdx.x & 31) == 0) { rs[threadIdx.x >> 5] = bs; rv[threadIdx.x >> 5] = bv; }
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = rs[threadIdx.x];
        int32_t v = rv[threadIdx.x];
        for (int o = 16; o; o >>= 1) {
            const double os = __shfl_xor_sync(kFull, s, o);
            const int32_t ov = __shfl_xor_sync(kFull, v, o);
            best_merge(s, v, os, ov);
        }
        if (threadIdx.x == 0) rv[32] = v;
    }
    __syncthreads();
    return rv[32];
}

// the preferred (score, index) pair of the tier, in every thread
template <int M>
__device__ __forceinline__ void reduce_best_pair(double &bs, int32_t &bv) {
    if (M == M_THR) return;
    for (int o = 16; o; o >>= 1) {
        const double os = __shfl_xor_sync(kFull, bs, o);
        const int32_t ov = __shfl_xor_sync(kFull, bv, o);
        best_merge(bs, bv, os, ov);
    }
    if (M == M_WARP) return;
    __shared__ double rs[33];
    __shared__ int32_t rv[33];
    __syncthreads();
    if ((threadIdx.x & 31) == 0) { rs[threadIdx.x >> 5] = bs; rv[threadIdx.x >> 5] = bv; }
    __syncthreads();
    if (threadIdx.x < 32) {
        double ss = rs[threadIdx.x];
        int32_t v = rv[threadIdx.x];
        for (int o = 16; o; o >>= 1) {
            const double os = __shfl_xor_sync(kFull, ss, o);
            const int32_t ov = __shfl_xor_sync(kFull, v, o);
            best_merge(ss, v, os, ov);
        }
        if (threadIdx.x == 0) { rs[32] = ss; rv[32] = v; }
    }
    __syncthreads();
    bs = rs[32];
    bv = rv[32];
}

// Row addressing.  THR: thread i takes list[i] (or i when list is NULL) of n
// rows; kernels skip rows above the thread tier.  WARP / BLK: one warp /
// block per list entry.
template <int M>
__device__ __forceinline__ bool get_row(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                                        int32_t &row) {
    if (M == M_THR) {
        const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (i >= n) return false;
        row = list ? list[i] : (int32_t)i;
        return true;
    }
    if (M == M_WARP) {
        const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        if (w >= nlist) return false;
        row = list[w];
        return true;
    }
    if (blockIdx.x >= nlist) return false;
    row = list[blockIdx.x];
    return true;
}

// Launch the three tiers of a per-row kernel: THR over all n rows (or a
// list), WARP over the warp-tier list, BLK over the block-tier list.
#define LAUNCH3(KERNEL, N, TLIST, WL, NW, BL, NB, S, ...)                                  \
    do {                                                                                    \
        if ((N) > 0) {                                                                      \
            KERNEL<M_THR><<<ceil_div((N), 256), 256, 0, (S)>>>((N), (TLIST), 0, __VA_ARGS__); \
            LAMG_CHECK_LAUNCH();                                                            \
        }                                                                                   \
        if ((NW) > 0) {                                                                     \
            KERNEL<M_WARP><<<ceil_div((int64_t)(NW) * 32, 256), 256, 0, (S)>>>(0, (WL), (NW), __VA_ARGS__); \
            LAMG_CHECK_LAUNCH();                                                            \
        }                                                                                   \
        if ((NB) > 0) {                                                                     \
            KERNEL<M_BLK><<<(NB), kBlk, 0, (S)>>>(0, (BL), (NB), __VA_ARGS__);             \
            LAMG_CHECK_LAUNCH();                                                            \
        }                                                                                   \
    } while (0)

// Rows of one level split by tier.
struct Tiers {
    Tmp<int32_t> w, b;
    int32_t nw = 0, nb = 0;
    Tiers(int32_t n, cudaStream_t s) : w(n, s), b(n, s) {}
};

// ---------------------------------------------------------------------------
// Input conversion and validation (Eq. (1.2), Sec. 1)
// ---------------------------------------------------------------------------

__global__ void k_rp64_to_32(const int64_t *__restrict__ in, int32_t *__restrict__ out, int64_t n1) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n1) out[i] = (int32_t)in[i];
}

__global__ void k_w_to_64(const void *__restrict__ in, int32_t is32, double *__restrict__ out,
                          int64_t nnz) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nnz) out[i] = is32 ? (double)((const float *)in)[i] : ((const double *)in)[i];
}

enum { VF_ARG = 1, VF_WEIGHT = 2, VF_SYM = 4 };

// signed_w = 0: weights positive and finite; 1 (negative_weights): nonzero and
// finite, and each row with entries has a positive sum (Gauss-Seidel divides by it)
__global__ void k_validate_rows(int64_t n, const int64_t *__restrict__ rp,
                                const int32_t *__restrict__ col, const double *__restrict__ w,
                                int32_t signed_w, int32_t *flags) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    int64_t s = rp[u], e = rp[u + 1];
    int f = 0;
    if (e < s) f |= VF_ARG;
    double sum = 0.0;
    for (int64_t i = s; i < e && !(f & VF_ARG); i++) {
        int32_t v = col[i];
        if (v < 0 || v >= n || v == u) f |= VF_ARG;
        if (i > s && v <= col[i - 1]) f |= VF_ARG;
        double x = w[i];
        if (!isfinite(x) || (signed_w ? !(x != 0.0) : !(x > 0.0))) f |= VF_WEIGHT;
        sum += x;
    }
    if (signed_w && e > s && !(f & VF_ARG) && !(sum > 0.0)) f |= VF_WEIGHT;
    if (f) atomicOr(flags, f);
}

// row of entry i: the last u with rp[u] <= i (binary search)
__device__ __forceinline__ int64_t row_of(const int64_t *__restrict__ rp, int64_t n, int64_t i) {
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (rp[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// entry-parallel symmetry check
__global__ void k_validate_sym(int64_t n, int64_t nnz, const int64_t *__restrict__ rp,
                               const int32_t *__restrict__ col, const double *__restrict__ w,
                               int32_t *flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nnz) return;
    const int64_t u = row_of(rp, n, i);
    const int32_t v = col[i];
    int64_t a = rp[v], b = rp[v + 1] - 1, f = -1;
    while (a <= b) {
        int64_t mid = (a + b) >> 1;
        int32_t c = col[mid];
        if (c == u) { f = mid; break; }
        if (c < u) a = mid + 1; else b = mid - 1;
    }
    if (f < 0 || __double_as_longlong(w[f]) != __double_as_longlong(w[i])) atomicOr(flags, VF_SYM);
}

__device__ __forceinline__ int32_t uf_find(int32_t *parent, int32_t x) {
    // path halving; concurrent writes only ever point a node at one of its ancestors
    while (true) {
        int32_t p = parent[x];
        if (p == x) return x;
        int32_t gp = parent[p];
        if (gp != p) parent[x] = gp;
        x = gp;
    }
}

__global__ void k_uf_init(int32_t *parent, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) parent[i] = (int32_t)i;
}

// entry-parallel union of the endpoints of every entry (u < v)
__global__ void k_uf_union(int64_t n, int64_t nnz, const int64_t *__restrict__ rp,
                           const int32_t *__restrict__ col, int32_t *parent) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nnz) return;
    int32_t a = (int32_t)row_of(rp, n, i), b = col[i];
    if (b <= a) return;
    // hook the larger root under the smaller; retry until both share a root
    for (int it = 0; it < (1 << 20); it++) {
        int32_t ra = uf_find(parent, a), rb = uf_find(parent, b);
        if (ra == rb) break;
        int32_t hi2 = ra > rb ? ra : rb, lo2 = ra > rb ? rb : ra;
        if (atomicCAS(&parent[hi2], hi2, lo2) == hi2) break;
        a = ra; b = rb;
    }
}

__global__ void k_uf_roots(int32_t *parent, int64_t n, unsigned long long *roots) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c = 0;
    if (i < n) c = (uf_find(parent, (int32_t)i) == i) ? 1ull : 0ull;
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(roots, c);
}

// graph of node u in a union: the g with gptr[g] <= u < gptr[g+1]
__device__ __forceinline__ int32_t graph_of(const int64_t *__restrict__ gptr, int32_t G, int64_t u) {
    int32_t lo = 0, hi = G - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (gptr[mid] <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// every entry must stay inside its row's graph
__global__ void k_graph_cross(int64_t n, int64_t nnz, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                              const int64_t *__restrict__ gptr, int32_t G, int32_t *flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nnz) return;
    const int64_t u = row_of(rp, n, i);
    if (graph_of(gptr, G, u) != graph_of(gptr, G, col[i])) atomicOr(flags, VF_ARG);
}

__global__ void k_graph_ids(int64_t n, const int64_t *__restrict__ gptr, int32_t G, int32_t *__restrict__ gid) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n) gid[u] = graph_of(gptr, G, u);
}

void graph_ids(int64_t n, const int64_t *gptr_dev, int32_t G, int32_t *gid, cudaStream_t s) {
    k_graph_ids<<<ceil_div(n, 256), 256, 0, s>>>(n, gptr_dev, G, gid);
    LAMG_CHECK_LAUNCH();
}

void validate_graph(int64_t n, const int64_t *row_ptr, const int32_t *col, const void *w,
                    int32_t w_is_fp32, cudaStream_t s, int32_t ngraphs, const int64_t *gptr, int32_t signed_w) {
    int64_t rp_n[2];
    LAMG_CUDA(cudaMemcpyAsync(&rp_n[0], row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LAMG_CUDA(cudaMemcpyAsync(&rp_n[1], row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LAMG_CUDA(cudaStreamSynchronize(s));
    LAMG_REQUIRE(rp_n[0] == 0 && rp_n[1] >= 0 && rp_n[1] < ((int64_t)1 << 31), LAMG_ERR_ARG,
                 "row_ptr[0] must be 0 and row_ptr[n] < 2^31");
    int64_t nnz = rp_n[1];
    LAMG_REQUIRE(nnz == 0 || (col && w), LAMG_ERR_ARG, "NULL col or w");
    Tmp<double> w64(nnz, s);
    if (nnz) {
        k_w_to_64<<<ceil_div(nnz, 256), 256, 0, s>>>(w, w_is_fp32, w64.get(), nnz);
        LAMG_CHECK_LAUNCH();
    }
    Tmp<int32_t> flags(1, s);
    LAMG_CUDA(cudaMemsetAsync(flags.get(), 0, sizeof(int32_t), s));
    k_validate_rows<<<ceil_div(n, 256), 256, 0, s>>>(n, row_ptr, col, w64.get(), signed_w, flags.get());
    LAMG_CHECK_LAUNCH();
    int32_t f = read_scalar(flags.get(), s);
    LAMG_REQUIRE(!(f & VF_ARG), LAMG_ERR_ARG,
                 "malformed CSR: columns must be in range, strictly increasing, no self loops");
    LAMG_REQUIRE(!(f & VF_WEIGHT), LAMG_ERR_BAD_WEIGHT,
                 signed_w ? "weights must be nonzero and finite, with positive row sums"
                          : "weights must be positive and finite");
    if (nnz) {
        k_validate_sym<<<ceil_div(nnz, 256), 256, 0, s>>>(n, nnz, row_ptr, col, w64.get(), flags.get());
        LAMG_CHECK_LAUNCH();
    }
    f = read_scalar(flags.get(), s);
    LAMG_REQUIRE(!(f & VF_SYM), LAMG_ERR_NOT_SYMMETRIC, "CSR is not symmetric (w_uv != w_vu)");
    Tmp<int32_t> parent(n, s);
    Tmp<unsigned long long> roots(1, s);
    LAMG_CUDA(cudaMemsetAsync(roots.get(), 0, sizeof(unsigned long long), s));
    k_uf_init<<<ceil_div(n, 256), 256, 0, s>>>(parent.get(), n);
    LAMG_CHECK_LAUNCH();
    if (nnz) {
        k_uf_union<<<ceil_div(nnz, 256), 256, 0, s>>>(n, nnz, row_ptr, col, parent.get());
        LAMG_CHECK_LAUNCH();
    }
    k_uf_roots<<<ceil_div(n, 256), 256, 0, s>>>(parent.get(), n, roots.get());
    LAMG_CHECK_LAUNCH();
    if (ngraphs > 1 && nnz) {
        // a union: no entry may join two graphs; then #components == #graphs iff each is connected
        Tmp<int64_t> gp(ngraphs + 1, s);
        LAMG_CUDA(cudaMemcpyAsync(gp.get(), gptr, sizeof(int64_t) * (ngraphs + 1), cudaMemcpyHostToDevice, s));
        k_graph_cross<<<ceil_div(nnz, 256), 256, 0, s>>>(n, nnz, row_ptr, col, gp.get(), ngraphs, flags.get());
        LAMG_CHECK_LAUNCH();
        LAMG_REQUIRE(!(read_scalar(flags.get(), s) & VF_ARG), LAMG_ERR_ARG, "an edge joins two graphs of the union");
    }
    unsigned long long r = read_scalar(roots.get(), s);
    if (ngraphs > 1)
        LAMG_REQUIRE(r == (unsigned long long)ngraphs, LAMG_ERR_DISCONNECTED, "a graph of the union is not connected");
    else
        LAMG_REQUIRE(r == 1, LAMG_ERR_DISCONNECTED, "graph is not connected");
}

// ---------------------------------------------------------------------------
// Per-node statistics: a_uu, max|w|, hub test (Sec. 3.4.1 footnote)
// ---------------------------------------------------------------------------

template <int M>
__global__ void __launch_bounds__(M == M_BLK ? kBlk : 256) k_node_stats(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                             const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                             const double *__restrict__ w, double hub_factor,
                             double *__restrict__ diag, double *__restrict__ adiag, double *__restrict__ maxw,
                             uint8_t *__restrict__ hub) {
    int32_t u;
    if (!get_row<M>(n, list, nlist, u)) return;
    const int32_t s = rp[u], e = rp[u + 1], deg = e - s;
    if (M == M_THR && deg > kLongRow) return;
    double d = 0.0, m = 0.0, s1 = 0.0, s2 = 0.0;
    for (int32_t i = s + tlane<M>(); i < e; i += tstride<M>()) {
        const double wi = w[i];
        const int32_t v = col[i];
        const double a = fabs(wi);
        d = d + wi;
        m = fmax(m, a);
        s1 = s1 + a;
        s2 = s2 + a * (double)(rp[v + 1] - rp[v]);
    }
    d = canon_reduce<M>(d);
    s1 = canon_reduce<M>(s1);
    s2 = canon_reduce<M>(s2);
    m = reduce_max<M>(m);
    if (tlane<M>() != 0) return;
    diag[u] = d;
    adiag[u] = s1;   // sum of |w_uv|: the energy-ratio test's diagonal (equals d for positive weights)
    maxw[u] = m;
    const double lhs = (double)deg * s1;
    const double rhs = hub_factor * s2;
    hub[u] = (deg > 0 && lhs >= rhs) ? 1 : 0;
}

// Initial aggregation state (Sec. 3.4.2): nodes without strong edges form the
// dummy aggregate (D), hubs are seeds (S), the rest undecided (U).
template <int M>
__global__ void __launch_bounds__(M == M_BLK ? kBlk : 256) k_node_state(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                             const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                             const double *__restrict__ w, const double *__restrict__ maxw,
                             double weak_tol, const uint8_t *__restrict__ hub,
                             int32_t *__restrict__ state) {
    int32_t u;
    if (!get_row<M>(n, list, nlist, u)) return;
    const int32_t s = rp[u], e = rp[u + 1];
    if (M == M_THR && e - s > kLongRow) return;
    bool strong = false;
    const double mu = maxw[u];
    for (int32_t i = s + tlane<M>(); i < e; i += tstride<M>()) {
        const double mw = fmax(mu, maxw[col[i]]);
        if (fabs(w[i]) >= weak_tol * mw) strong = true;
    }
    strong = reduce_any<M>(strong);
    if (tlane<M>() != 0) return;
    state[u] = !strong ? ST_D : (hub[u] ? ST_S : ST_U);
}

// ---------------------------------------------------------------------------
// Jones-Plassmann colouring
// ---------------------------------------------------------------------------

// Priority: largest degree first, then the hash, ties to the lower index.
__device__ __forceinline__ bool beats(int32_t du, uint64_t pu, int32_t u, int32_t dv, uint64_t pv, int32_t v) {
    if (du != dv) return du > dv;
    return pu > pv || (pu == pv && u < v);
}

// smallest colour >= base0 not used by any neighbour, searched in windows of 64
template <int M>
__device__ __forceinline__ int32_t jp_free_colour(int32_t u, const int32_t *__restrict__ rp,
                                                  const int32_t *__restrict__ col,
                                                  const int32_t *__restrict__ colour, int32_t base0 = 0) {
    for (int32_t base = base0;; base += 64) {
        unsigned long long mask = 0ull;
        for (int32_t i = rp[u] + tlane<M>(); i < rp[u + 1]; i += tstride<M>()) {
            const int32_t c = colour[col[i]];
            if (c >= base && c < base + 64) mask |= 1ull << (c - base);
        }
        mask = reduce_or64<M>(mask);
        if (mask != ~0ull) return base + __ffsll((long long)~mask) - 1;
    }
}

// Same result for a block-tier row in one pass: the neighbours' colours below
// kFreeBits are marked in a shared bitmap, then the first clear bit is found;
// only when all of them are taken does the windowed search continue above.
constexpr int kFreeBits = 8192;
__device__ __forceinline__ int32_t jp_free_colour_blk(int32_t u, const int32_t *__restrict__ rp,
                                                      const int32_t *__restrict__ col,
                                                      const int32_t *__restrict__ colour) {
    __shared__ unsigned int bits[kFreeBits / 32];
    __shared__ int32_t first;
    for (int k = threadIdx.x; k < kFreeBits / 32; k += blockDim.x) bits[k] = 0u;
    if (threadIdx.x == 0) first = kFreeBits;
    __syncthreads();
    for (int32_t i = rp[u] + threadIdx.x; i < rp[u + 1]; i += blockDim.x) {
        const int32_t c = colour[col[i]];
        if (c >= 0 && c < kFreeBits) atomicOr(&bits[c >> 5], 1u << (c & 31));
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kFreeBits / 32; k += blockDim.x)
        if (bits[k] != ~0u) atomicMin(&first, k * 32 + __ffs(~bits[k]) - 1);
    __syncthreads();
    const int32_t f = first;
    __syncthreads();
    if (f < kFreeBits) return f;
    for (int32_t base = kFreeBits;; base += 64) {
        unsigned long long mask = 0ull;
        for (int32_t i = rp[u] + threadIdx.x; i < rp[u + 1]; i += blockDim.x) {
            const int32_t c = colour[col[i]];
            if (c >= base && c < base + 64) mask |= 1ull << (c - base);
        }
        mask = reduce_or64<M_BLK>(mask);
        if (mask != ~0ull) return base + __ffsll((long long)~mask) - 1;
    }
}


constexpr long long kCoopMaxSpins = 1ll << 21;  // one to two seconds of polling

// Counting grid barrier of the cooperative setup kernels: bar[0] counts the
// arrivals of the whole launch (zeroed before it); barrier e completes at
// e * gridDim.x.  Thread 0 arrives with a release reduction after the block's
// __syncthreads and polls with acquire loads; the closing __syncthreads passes
// the acquire on to the block.  Bounded spin: on expiry (or when another block
// gave up) the error word is set and every block returns.
__device__ __forceinline__ bool coop_sync(unsigned int *bar, int32_t *err, unsigned int &epoch) {
    __shared__ int bad;
    __syncthreads();
    if (threadIdx.x == 0) {
        bad = 0;
        const unsigned int target = (++epoch) * gridDim.x;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        long long spins = 0;
        while (true) {
            unsigned int v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if (v >= target) break;
            if ((++spins & 255) == 0) {
                if (*(volatile int32_t *)err) { bad = 1; break; }
                if (spins > kCoopMaxSpins) { atomicExch(err, 1); bad = 1; break; }
            }
        }
    }
    __syncthreads();
    return bad == 0;
}

// ---- Jones-Plassmann by wait counts.  wait[u] = number of neighbours that
// beat u (higher priority).  Round r colours every node whose count is zero
// -- exactly the uncoloured nodes that beat all their uncoloured neighbours,
// i.e. the JP selection of that round -- with the smallest colour unused by
// its (already coloured) higher-priority neighbours; then each such node
// decrements the counts of the neighbours it beats, and a count reaching zero
// puts that neighbour in the next round's frontier.  Every edge is examined a
// constant number of times instead of once per round.  Frontiers are kept per
// row tier (lst: [parity][tier], cnt: [parity][tier]); their order (atomic
// appends) changes no decision.  out[0] = rounds.
// hashed = 0 (colour_rule 1): the priority is the degree, then the lower index
__global__ void k_jp_prio(int32_t n, const int32_t *__restrict__ rp, uint64_t key, int32_t hashed,
                          int32_t *__restrict__ deg, uint64_t *__restrict__ hsh) {
    const int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    deg[u] = rp[u + 1] - rp[u];
    hsh[u] = hashed ? splitmix64(key + (uint64_t)u) : 0ull;
}

template <int M>
__global__ void __launch_bounds__(M == M_BLK ? kBlk : 256) k_jp_wait(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                                                                    const int32_t *__restrict__ rp,
                                                                    const int32_t *__restrict__ col,
                                                                    const int32_t *__restrict__ deg,
                                                                    const uint64_t *__restrict__ hsh,
                                                                    int32_t *__restrict__ wait) {
    int32_t u;
    if (!get_row<M>(n, list, nlist, u)) return;
    if (M == M_THR && rp[u + 1] - rp[u] > kLongRow) return;
    const int32_t du = deg[u];
    const uint64_t pu = hsh[u];
    int32_t c = 0;
    for (int32_t i = rp[u] + tlane<M>(); i < rp[u + 1]; i += tstride<M>()) {
        const int32_t v = col[i];
        c += beats(deg[v], hsh[v], v, du, pu, u) ? 1 : 0;
    }
    c = reduce_sum_i32<M>(c);
    if (tlane<M>() == 0) wait[u] = c;
}

// frontier flags: rows of tier `tier` with no waiting count
__global__ void k_jp_ready(const int32_t *__restrict__ rp, int64_t n, int tier, const int32_t *__restrict__ wait,
                           uint8_t *__restrict__ f) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    f[u] = (wait[u] == 0 && row_tier(rp[u + 1] - rp[u]) == tier) ? 1 : 0;
}

// decrement the counts of the neighbours that u beats; append those that reach zero
// Append the ready lanes' nodes v to the next frontier, list row_tier(deg[v]),
// with one atomic per warp and tier: a round releases tens of thousands of
// nodes on the finest levels of a grid, and one atomic per node on the three
// list counters serialised there.  All 32 lanes of the warp call it together.
// The order inside a list changes no decision (a frontier's nodes are
// pairwise non-adjacent, and each one's colour depends on earlier rounds only).
__device__ __forceinline__ void jp_append_warp(bool ready, int32_t v, int t, int32_t *nlst, int64_t cap,
                                               int32_t *nxt) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
#pragma unroll
    for (int tier = 0; tier < 3; tier++) {
        const bool mine = ready && t == tier;
        const unsigned m = __ballot_sync(0xffffffffu, mine);
        if (m == 0u) continue;
        const int leader = __ffs(m) - 1;
        int32_t base = 0;
        if (lane == leader) base = atomicAdd(&nxt[tier], __popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (mine) nlst[(int64_t)tier * cap + base + __popc(m & below)] = v;
    }
}

// Release neighbour col[i] of u (its wait count drops by one when u beats it);
// true when that made it ready, with its list tier.
__device__ __forceinline__ bool jp_release_one(int32_t u, int32_t du, uint64_t pu, int32_t i,
                                               const int32_t *__restrict__ col, const int32_t *__restrict__ deg,
                                               const uint64_t *__restrict__ hsh, int32_t *__restrict__ wait,
                                               int32_t &v, int &t) {
    v = col[i];
    if (!beats(du, pu, u, deg[v], hsh[v], v)) return false;
    if (atomicSub(&wait[v], 1) != 1) return false;
    t = row_tier(deg[v]);
    return true;
}

// Thread tier: lane l releases the neighbours of u (u < 0: no row).  Called by
// all 32 lanes of a warp; the loop runs to the warp's longest row.
__device__ __forceinline__ void jp_release_thr(int32_t u, const int32_t *__restrict__ rp,
                                               const int32_t *__restrict__ col, const int32_t *__restrict__ deg,
                                               const uint64_t *__restrict__ hsh, int32_t *__restrict__ wait,
                                               int32_t *nlst, int64_t cap, int32_t *nxt) {
    int32_t s = 0, len = 0, du = 0;
    uint64_t pu = 0;
    if (u >= 0) {
        s = rp[u];
        len = rp[u + 1] - s;
        du = deg[u];
        pu = hsh[u];
    }
    const int32_t mlen = __reduce_max_sync(0xffffffffu, len);
    for (int32_t k = 0; k < mlen; k++) {
        int32_t v = 0;
        int t = 0;
        const bool ready = k < len && jp_release_one(u, du, pu, s + k, col, deg, hsh, wait, v, t);
        jp_append_warp(ready, v, t, nlst, cap, nxt);
    }
}

// Warp or block tier: the row's entries in strides of 32 (warp) or kBlk
// (block) lanes; every warp of the row loops the same number of times.
template <int M>
__device__ __forceinline__ void jp_release(int32_t u, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                           const int32_t *__restrict__ deg, const uint64_t *__restrict__ hsh,
                                           int32_t *__restrict__ wait, int32_t *nlst, int64_t cap, int32_t *nxt) {
    static_assert(M != M_THR, "thread-tier rows go through jp_release_thr");
    const int32_t du = deg[u];
    const uint64_t pu = hsh[u];
    const int32_t s = rp[u], e = rp[u + 1];
    const int32_t w0 = M == M_WARP ? 0 : (int32_t)(threadIdx.x & ~31u);
    for (int32_t i0 = s + w0; i0 < e; i0 += tstride<M>()) {
        const int32_t i = i0 + (int32_t)(threadIdx.x & 31);
        int32_t v = 0;
        int t = 0;
        const bool ready = i < e && jp_release_one(u, du, pu, i, col, deg, hsh, wait, v, t);
        jp_append_warp(ready, v, t, nlst, cap, nxt);
    }
}

// A round's hub rows (block tier) are few and long (a median of about 1,000
// entries at the middle levels of a power-law graph).  With at most
// kSpreadHubs of them, their entries are dealt to every warp of the grid in
// pieces of 32, instead of one block per hub:
//   colour phase:  each piece ORs its neighbours' colours below kFreeBits into
//                  the hub's bitmap in global memory (gbits, kept zeroed);
//   release phase: the hub's global warp j takes the first clear bit as the
//                  colour and clears the bitmap, while all warps release the
//                  hub's neighbours piece by piece.
// The colours are the same as with one block per hub: the colour is the
// smallest one free among the neighbours, and the release order changes no
// decision.  More hubs in one round take the per-block path.
constexpr int kSpreadHubs = 32;
constexpr int kFreeWords = kFreeBits / 32;

// the piece p of the frontier's c2 <= 32 hub rows: hub index j, row u and this
// lane's entry e (valid when e < rp[u + 1]); hub data are held one per lane
struct HubPieces {
    int32_t myu, myn, incl, total;
};
__device__ __forceinline__ HubPieces hub_pieces(int32_t c2, const int32_t *L2, const int32_t *__restrict__ rp) {
    const int lane = threadIdx.x & 31;
    HubPieces h;
    h.myu = lane < c2 ? L2[lane] : 0;
    h.myn = lane < c2 ? (rp[h.myu + 1] - rp[h.myu] + 31) >> 5 : 0;
    int32_t v = h.myn;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    h.incl = v;
    h.total = __shfl_sync(0xffffffffu, v, 31);
    return h;
}
__device__ __forceinline__ void hub_piece(const HubPieces &h, int64_t p, int32_t c2, const int32_t *__restrict__ rp,
                                          int &j, int32_t &u, int32_t &e) {
    const int lane = threadIdx.x & 31;
    j = __popc(__ballot_sync(0xffffffffu, lane < c2 && h.incl <= p));
    u = __shfl_sync(0xffffffffu, h.myu, j);
    const int32_t start = __shfl_sync(0xffffffffu, h.incl - h.myn, j);
    e = rp[u] + (int32_t)(p - start) * 32 + lane;
}

__global__ void __launch_bounds__(kBlk) k_jp_dag(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                                const int32_t *__restrict__ deg, const uint64_t *__restrict__ hsh,
                                                int32_t *__restrict__ wait, int32_t *__restrict__ colour, int32_t *lst,
                                                int64_t cap, int32_t *cnt, int32_t *out, unsigned int *bar,
                                                int32_t *err, unsigned int *gbits) {
    const int64_t nthr = (int64_t)gridDim.x * kBlk;
    // chunks of 32 items, consecutive chunks on consecutive blocks (spread over every SM)
    const int64_t tid = ((int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32 + (threadIdx.x & 31);
    const int64_t nwarp = nthr >> 5, wid = tid >> 5;
    const int lane = threadIdx.x & 31;
    unsigned int epoch = 0;
    for (int32_t r = 0;; r++) {
        const volatile int32_t *cur = cnt + (r & 1) * 3;
        int32_t *nxt = cnt + ((r + 1) & 1) * 3;
        const int32_t c0 = cur[0], c1 = cur[1], c2 = cur[2];
        if (c0 + c1 + c2 == 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = r;
            return;
        }
        const int32_t *L0 = lst + (int64_t)(r & 1) * 3 * cap, *L1 = L0 + cap, *L2 = L1 + cap;
        int32_t *N = lst + (int64_t)((r + 1) & 1) * 3 * cap;
        const bool spread = c2 <= kSpreadHubs;
        // colour the frontier: its higher-priority neighbours are all coloured
        for (int64_t i = tid; i < c0; i += nthr) {
            const int32_t u = L0[i];
            colour[u] = jp_free_colour<M_THR>(u, rp, col, colour);
        }
        for (int64_t i = wid; i < c1; i += nwarp) {
            const int32_t u = L1[i];
            const int32_t c = jp_free_colour<M_WARP>(u, rp, col, colour);
            if (lane == 0) colour[u] = c;
        }
        if (spread) {
            if (c2 > 0) {
                const HubPieces hp = hub_pieces(c2, L2, rp);
                for (int64_t p = wid; p < hp.total; p += nwarp) {
                    int j;
                    int32_t u, e;
                    hub_piece(hp, p, c2, rp, j, u, e);
                    if (e < rp[u + 1]) {
                        const int32_t c = colour[col[e]];
                        if (c >= 0 && c < kFreeBits) atomicOr(&gbits[j * kFreeWords + (c >> 5)], 1u << (c & 31));
                    }
                }
            }
        } else {
            for (int64_t i = blockIdx.x; i < c2; i += gridDim.x) {
                const int32_t u = L2[i];
                const int32_t c = jp_free_colour_blk(u, rp, col, colour);
                if (threadIdx.x == 0) colour[u] = c;
            }
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) { nxt[0] = 0; nxt[1] = 0; nxt[2] = 0; }
        if (!coop_sync(bar, err, epoch)) return;
        // release the neighbours they beat
        for (int64_t i0 = tid - lane; i0 < c0; i0 += nthr) {   // warp-uniform loop
            const int64_t i = i0 + lane;
            jp_release_thr(i < c0 ? L0[i] : -1, rp, col, deg, hsh, wait, N, cap, nxt);
        }
        for (int64_t i = wid; i < c1; i += nwarp) jp_release<M_WARP>(L1[i], rp, col, deg, hsh, wait, N, cap, nxt);
        if (spread) {
            if (c2 > 0) {
                if (wid < c2) {   // the colour of hub j = wid: first clear bit of its bitmap, which is cleared
                    const int32_t u = L2[wid];
                    unsigned int *bw = gbits + wid * kFreeWords;
                    int32_t first = kFreeBits;
                    for (int k = lane; k < kFreeWords; k += 32) {
                        const unsigned int m = bw[k];
                        if (m != ~0u && first == kFreeBits) first = k * 32 + __ffs(~m) - 1;
                        bw[k] = 0u;
                    }
#pragma unroll
                    for (int o = 16; o; o >>= 1) first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
                    if (first == kFreeBits) first = jp_free_colour<M_WARP>(u, rp, col, colour, kFreeBits);
                    if (lane == 0) colour[u] = first;
                }
                const HubPieces hp = hub_pieces(c2, L2, rp);
                for (int64_t p = wid; p < hp.total; p += nwarp) {
                    int j;
                    int32_t u, e;
                    hub_piece(hp, p, c2, rp, j, u, e);
                    int32_t v = 0;
                    int t = 0;
                    const bool ready = e < rp[u + 1] && jp_release_one(u, deg[u], hsh[u], e, col, deg, hsh, wait, v, t);
                    jp_append_warp(ready, v, t, N, cap, nxt);
                }
            }
        } else {
            for (int64_t i = blockIdx.x; i < c2; i += gridDim.x) jp_release<M_BLK>(L2[i], rp, col, deg, hsh, wait, N, cap, nxt);
        }
        if (!coop_sync(bar, err, epoch)) return;
    }
}

__global__ void k_fill_i32(int32_t *a, int64_t n, int32_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

__global__ void k_hist_u32(const uint32_t *__restrict__ a, int64_t n, int32_t *__restrict__ cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&cnt[a[i]], 1);
}

// flag rows of one tier (only uncoloured ones when `colour` is given)
__global__ void k_tier_flags(const int32_t *__restrict__ rp, int64_t n, int tier,
                             const int32_t *__restrict__ colour, uint8_t *__restrict__ f) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const bool ok = colour ? colour[u] < 0 : true;
    f[u] = (ok && row_tier(rp[u + 1] - rp[u]) == tier) ? 1 : 0;
}

// key = colour * 3 + tier, value = node
__global__ void k_order_keys(const int32_t *__restrict__ rp, const int32_t *__restrict__ colour, int32_t n,
                             uint32_t *__restrict__ key, int32_t *__restrict__ val) {
    int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    key[u] = (uint32_t)colour[u] * 3u + (uint32_t)row_tier(rp[u + 1] - rp[u]);
    val[u] = u;
}

static int bits_for(uint64_t maxval) {
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) b++;
    return b;
}

// Rows of tier `tier` (only uncoloured ones when colour != NULL), increasing id.
static int32_t tier_list(const int32_t *rp, int64_t n, int tier, const int32_t *colour, int32_t *out,
                         cudaStream_t s) {
    if (n <= 0) return 0;
    Tmp<uint8_t> f(n, s);
    k_tier_flags<<<ceil_div(n, 256), 256, 0, s>>>(rp, n, tier, colour, f.get());
    LAMG_CHECK_LAUNCH();
    return (int32_t)compact_indices(f.get(), out, n, s);
}

// ---------------------------------------------------------------------------
// Test vectors (Sec. 3.3.1): random[-1,1] then nu GS sweeps on A x = 0
// ---------------------------------------------------------------------------

__global__ void k_tv_init(double *__restrict__ X, int64_t count, uint64_t key) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint64_t z = splitmix64(key + (uint64_t)i);
    const double t = (double)(z >> 11) * 0x1.0p-53;
    X[i] = 2.0 * t - 1.0;
}

// x_uk = (canonical sum of w_uv x_vk) / a_uu for every TV k (b = 0); one pass
// over the row with K accumulators, each summed in its canonical order; each
// lane's running sum advances by a fused multiply-add, as in the oracle.
template <int M>
__device__ __forceinline__ void tv_update(int32_t u, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                          const double *__restrict__ w, const double *__restrict__ diag, int32_t K,
                                          double *__restrict__ X) {
    const int32_t s = rp[u], e = rp[u + 1];
    // an isolated node (a whole graph of a union, coarsened to one node) keeps its TVs;
    // such a row has no entries, so it is always in the thread tier
    if (M == M_THR && e == s) return;
    double acc[16];
#pragma unroll
    for (int k = 0; k < 16; k++) acc[k] = 0.0;
    // two entries per step (their loads overlap); each lane still adds its
    // entries in increasing order, so the canonical partial is unchanged
    const int32_t st = tstride<M>();
    int32_t j = s + tlane<M>();
    for (; j + st < e; j += 2 * st) {
        const double w0 = w[j], w1 = w[j + st];
        const double *x0 = X + (int64_t)col[j] * K, *x1 = X + (int64_t)col[j + st] * K;
#pragma unroll
        for (int k = 0; k < 16; k++)
            if (k < K) {
                const double a = x0[k], b = x1[k];
                acc[k] = fma(w0, a, acc[k]);
                acc[k] = fma(w1, b, acc[k]);
            }
    }
    if (j < e) {
        const double wj = w[j];
        const double *xv = X + (int64_t)col[j] * K;
#pragma unroll
        for (int k = 0; k < 16; k++)
            if (k < K) acc[k] = fma(wj, xv[k], acc[k]);
    }
    const double du = diag[u];
#pragma unroll
    for (int k = 0; k < 16; k++) {
        if (k < K) {
            const double t = canon_reduce<M>(acc[k]);
            if (tlane<M>() == 0) X[(int64_t)u * K + k] = t / du;
        }
    }
    if (M == M_WARP) __syncwarp();
    if (M == M_BLK) __syncthreads();
}

template <int M>
__global__ void __launch_bounds__(M == M_BLK ? kBlk : 256) k_tv_sweep(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                           const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                           const double *__restrict__ w, const double *__restrict__ diag,
                           int32_t K, double *__restrict__ X) {
    int32_t u;
    if (!get_row<M>(n, list, nlist, u)) return;
    tv_update<M>(u, rp, col, w, diag, K, X);
}

// Colours c0 .. c1-1 of a TV sweep in one block (colour/tier ranges in cb).
__global__ void __launch_bounds__(kBlk) k_tv_sweep_tail(int32_t c0, int32_t c1, const int32_t *__restrict__ cb,
                                                       const int32_t *__restrict__ order,
                                                       const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                                       const double *__restrict__ w, const double *__restrict__ diag,
                                                       int32_t K, double *__restrict__ X) {
    const int warp = threadIdx.x >> 5;
    for (int32_t c = c0; c < c1; c++) {
        const int32_t t0 = cb[4 * c], t1 = cb[4 * c + 1], t2 = cb[4 * c + 2], t3 = cb[4 * c + 3];
        for (int32_t i = t0 + threadIdx.x; i < t1; i += kBlk) tv_update<M_THR>(order[i], rp, col, w, diag, K, X);
        for (int32_t i = t1 + warp; i < t2; i += kBlk / 32) tv_update<M_WARP>(order[i], rp, col, w, diag, K, X);
        for (int32_t i = t2; i < t3; i++) tv_update<M_BLK>(order[i], rp, col, w, diag, K, X);
        __syncthreads();
    }
}

// ---- All colours of nu TV sweeps in one cooperative launch.  plan = triples
// (c0, c1, single): single runs (small colours) go to block 0 alone with
// __syncthreads between colours; other colours are spread over every block,
// with a bounded grid barrier after each.  The row updates and their order
// within a colour are those of the per-colour launches (bit-identical).
__global__ void __launch_bounds__(kBlk) k_tv_sweeps_coop(int32_t nsweeps, const int32_t *__restrict__ plan,
                                                         int32_t nplan, const int32_t *__restrict__ cb,
                                                         const int32_t *__restrict__ order,
                                                         const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                                         const double *__restrict__ w, const double *__restrict__ diag,
                                                         int32_t K, double *__restrict__ X, unsigned int *bar,
                                                         int32_t *err, double *__restrict__ gsum,
                                                         unsigned long long *__restrict__ ptime) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nthr = (int64_t)gridDim.x * kBlk;
    // chunks of 32 items, consecutive chunks on consecutive blocks (spread over every SM)
    const int64_t tid = ((int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32 + (threadIdx.x & 31);
    const int64_t nwarp = nthr >> 5, wid = tid >> 5;
    unsigned int epoch = 0;
    for (int32_t sw = 0; sw < nsweeps; sw++) {
        for (int32_t q = 0; q < nplan; q++) {
            unsigned long long t_start = 0;
            if (ptime && blockIdx.x == 0 && threadIdx.x == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
            const int32_t c0 = plan[3 * q], c1 = plan[3 * q + 1], single = plan[3 * q + 2];
            if (single) {
                if (blockIdx.x == 0) {
                    for (int32_t c = c0; c < c1; c++) {
                        const int32_t t0 = cb[4 * c], t1 = cb[4 * c + 1], t2 = cb[4 * c + 2], t3 = cb[4 * c + 3];
                        for (int32_t i = t0 + threadIdx.x; i < t1; i += kBlk) tv_update<M_THR>(order[i], rp, col, w, diag, K, X);
                        for (int32_t i = t1 + warp; i < t2; i += kBlk / 32) tv_update<M_WARP>(order[i], rp, col, w, diag, K, X);
                        for (int32_t i = t2; i < t3; i++) tv_update<M_BLK>(order[i], rp, col, w, diag, K, X);
                        __syncthreads();
                    }
                }
            } else {
                const int32_t t0 = cb[4 * c0], t1 = cb[4 * c0 + 1], t2 = cb[4 * c0 + 2], t3 = cb[4 * c0 + 3];
                for (int64_t i = t0 + tid; i < t1; i += nthr) tv_update<M_THR>(order[i], rp, col, w, diag, K, X);
                for (int64_t i = t1 + wid; i < t2; i += nwarp) tv_update<M_WARP>(order[i], rp, col, w, diag, K, X);
                // Block-tier rows (hubs): the 1024 lane partials of the canonical order
                // come in 32 groups of 32 lanes; each group is one warp's work item
                // anywhere on the GPU (its lane partials, then the group's tree), so a
                // hub's FP64 work spreads over many SMs.  After a barrier one warp per
                // row adds the 32 group sums by the same tree (R1 order, bit-identical).
                const int32_t nbr = t3 - t2;
                if (nbr > 0) {
                    for (int64_t it = wid; it < (int64_t)nbr * 32; it += nwarp) {
                        const int32_t r = (int32_t)(it >> 5), g = (int32_t)(it & 31);
                        const int32_t u = order[t2 + r];
                        double acc[16];
#pragma unroll
                        for (int k = 0; k < 16; k++) acc[k] = 0.0;
                        int32_t j = rp[u] + 32 * g + lane;
                        const int32_t je = rp[u + 1];
                        for (; j + kBlk < je; j += 2 * kBlk) {   // two entries per step, same order
                            const double w0 = w[j], w1 = w[j + kBlk];
                            const double *x0 = X + (int64_t)col[j] * K, *x1 = X + (int64_t)col[j + kBlk] * K;
#pragma unroll
                            for (int k = 0; k < 16; k++)
                                if (k < K) {
                                    const double a = x0[k], b = x1[k];
                                    acc[k] = fma(w0, a, acc[k]);
                                    acc[k] = fma(w1, b, acc[k]);
                                }
                        }
                        if (j < je) {
                            const double wj = w[j];
                            const double *xv = X + (int64_t)col[j] * K;
#pragma unroll
                            for (int k = 0; k < 16; k++)
                                if (k < K) acc[k] = fma(wj, xv[k], acc[k]);
                        }
#pragma unroll
                        for (int k = 0; k < 16; k++) {
                            if (k < K) {
                                const double t = warp_tree(acc[k]);
                                if (lane == 0) gsum[((int64_t)r * 32 + g) * K + k] = t;
                            }
                        }
                    }
                    if (!coop_sync(bar, err, epoch)) return;
                    for (int64_t r = wid; r < nbr; r += nwarp) {
                        const int32_t u = order[t2 + r];
                        const double du = diag[u];
                        for (int k = 0; k < K; k++) {
                            const double t = warp_tree(gsum[((int64_t)r * 32 + lane) * K + k]);
                            if (lane == 0) X[(int64_t)u * K + k] = t / du;
                        }
                    }
                }
            }
            if (!coop_sync(bar, err, epoch)) return;
            if (ptime && blockIdx.x == 0 && threadIdx.x == 0) {
                unsigned long long t_end;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
                ptime[q] += t_end - t_start;
            }
        }
    }
}

// Nodal energy E_u = 1/2 sum_v w_uv (x_u - x_v)^2 of TV k (Eq. (3.11a)).
template <int M>
__global__ void __launch_bounds__(M == M_BLK ? kBlk : 256) k_tv_energy(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                            const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                            const double *__restrict__ w, int32_t K, int32_t k,
                            const double *__restrict__ X, double *__restrict__ eu) {
    int32_t u;
    if (!get_row<M>(n, list, nlist, u)) return;
    const int32_t s = rp[u], e = rp[u + 1];
    if (M == M_THR && e - s > kLongRow) return;
    const double xu = X[(int64_t)u * K + k];
    double acc = 0.0;
    for (int32_t j = s + tlane<M>(); j < e; j += tstride<M>()) {
        const double d = xu - X[(int64_t)col[j] * K + k];
        acc = fma(w[j], d * d, acc);
    }
    acc = canon_reduce<M>(acc);
    if (tlane<M>() == 0) eu[u] = 0.5 * acc;
}

// Canonical sum of chunks of 512 terms, one warp per chunk.
__global__ void k_canon_chunks(const double *__restrict__ t, int64_t len, double *__restrict__ out) {
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t lo = c * 512;
    if (lo >= len) return;
    const int64_t cnt = (len - lo) < 512 ? (len - lo) : 512;
    if (cnt <= 32) {
        if (lane == 0) {
            double s = 0.0;
            for (int64_t i = 0; i < cnt; i++) s = s + t[lo + i];
            out[c] = s;
        }
        return;
    }
    double p = 0.0;
    for (int64_t i = lane; i < cnt; i += 32) p = p + t[lo + i];
    p = warp_tree(p);
    if (lane == 0) out[c] = p;
}

static double canon_sum_global(const double *t, int64_t len, cudaStream_t s) {
    Tmp<double> a((size_t)std::max<int64_t>(1, (len + 511) / 512), s);
    Tmp<double> b((size_t)std::max<int64_t>(1, (len + 511) / 512), s);
    const double *src = t;
    double *dst = a.get(), *other = b.get();
    while (true) {
        int64_t nch = (len + 511) / 512;
        if (nch < 1) nch = 1;
        k_canon_chunks<<<ceil_div(nch * 32, 256), 256, 0, s>>>(src, len, dst);
        LAMG_CHECK_LAUNCH();
        if (len <= 512) break;
        len = nch;
        src = dst;
        std::swap(dst, other);
    }
    return read_scalar(dst, s);
}

// ---------------------------------------------------------------------------
// Affinity and energy ratio (Eqs. (3.5), (3.12)); the reading of Eq. (3.12):
// q_us = max_k E_u(x^k; x^k_s) / min_y E_u(x^k; y), with
// Emin = 1/2 sum_v |w_uv| (y* - x_v)^2 and E_s = Emin + a+_uu (x_s - y*)^2 / 2,
// a+_uu = sum_v |w_uv| (the nodal energies use |w|: the same numbers for
// positive weights, and non-negative energies for signed ones).
// ---------------------------------------------------------------------------

template <int M>
__global__ void __launch_bounds__(M == M_BLK ? kBlk : 256) k_node_pre(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                           const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                           const double *__restrict__ w, const double *__restrict__ diag,
                           int32_t K, const double *__restrict__ X, double *__restrict__ XX,
                           double *__restrict__ ystar, double *__restrict__ emin) {
    int32_t u;
    if (!get_row<M>(n, list, nlist, u)) return;
    const int32_t s = rp[u], e = rp[u + 1];
    if (M == M_THR && e - s > kLongRow) return;
    const int lane = tlane<M>();
    if (lane == 0) {
        double xx = 0.0;
        for (int k = 0; k < K; k++) {
            const double x = X[(int64_t)u * K + k];
            xx = fma(x, x, xx);
        }
        XX[u] = xx;
    }
    const double du = diag[u];
    double acc[16], y[16];
#pragma unroll
    for (int k = 0; k < 16; k++) acc[k] = 0.0;
    for (int32_t j = s + lane; j < e; j += tstride<M>()) {
        const double wj = fabs(w[j]);
        const double *xv = X + (int64_t)col[j] * K;
#pragma unroll
        for (int k = 0; k < 16; k++)
            if (k < K) acc[k] = fma(wj, xv[k], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < 16; k++) {
        y[k] = 0.0;
        if (k < K) y[k] = canon_reduce<M>(acc[k]) / du;
        acc[k] = 0.0;
    }
    for (int32_t j = s + lane; j < e; j += tstride<M>()) {
        const double wj = fabs(w[j]);
        const double *xv = X + (int64_t)col[j] * K;
#pragma unroll
        for (int k = 0; k < 16; k++)
            if (k < K) {
                const double d = y[k] - xv[k];
                acc[k] = fma(wj, d * d, acc[k]);
            }
    }
#pragma unroll
    for (int k = 0; k < 16; k++) {
        if (k < K) {
            const double E = canon_reduce<M>(acc[k]);
            if (lane == 0) {
                ystar[(int64_t)u * K + k] = y[k];
                emin[(int64_t)u * K + k] = 0.5 * E;
            }
        }
    }
}

template <int M>
__global__ void __launch_bounds__(M == M_BLK ? kBlk : 256) k_entry_rows(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                             const int32_t *__restrict__ rp, int32_t *__restrict__ erow) {
    int32_t u;
    if (!get_row<M>(n, list, nlist, u)) return;
    const int32_t s = rp[u], e = rp[u + 1];
    if (M == M_THR && e - s > kLongRow) return;
    for (int32_t j = s + tlane<M>(); j < e; j += tstride<M>()) erow[j] = u;
}

__global__ void k_scores(int64_t nnz, const int32_t *__restrict__ erow, const int32_t *__restrict__ col,
                         const double *__restrict__ w, int32_t K, const double *__restrict__ X,
                         const double *__restrict__ XX, const double *__restrict__ ystar,
                         const double *__restrict__ emin, const double *__restrict__ diag,
                         const double *__restrict__ maxw, double q_max, double weak_tol,
                         double *__restrict__ aff_out, double *__restrict__ q_out,
                         double *__restrict__ score) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nnz) return;
    const int32_t u = erow[j], v = col[j];
    const double *xu = X + (int64_t)u * K, *xv = X + (int64_t)v * K;
    double dot = 0.0;
    for (int k = 0; k < K; k++) dot = fma(xu[k], xv[k], dot);
    const double num = dot * dot, den = XX[u] * XX[v];
    const double a = den > 0.0 ? num / den : 0.0;
    const double half_a = 0.5 * diag[u];
    double qq = 0.0;
    for (int k = 0; k < K; k++) {
        const double d = xv[k] - ystar[(int64_t)u * K + k];
        const double em = emin[(int64_t)u * K + k];
        const double es = em + half_a * (d * d);
        const double r = em > 0.0 ? es / em : (es == 0.0 ? 1.0 : INFINITY);
        if (r > qq) qq = r;
    }
    const double mw = fmax(maxw[u], maxw[v]);
    const bool strong = fabs(w[j]) >= weak_tol * mw;
    if (aff_out) aff_out[j] = a;
    if (q_out) q_out[j] = qq;
    score[j] = (strong && qq <= q_max) ? a : -1.0;
}

// ---------------------------------------------------------------------------
// Aggregation stages (Sec. 3.4.2, build reading; see the oracle)
// ---------------------------------------------------------------------------

template <int M>
__global__ void __launch_bounds__(M == M_BLK ? kBlk : 256) k_best(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                       const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                       const double *__restrict__ score, const int32_t *__restrict__ state,
                       int32_t *__restrict__ best) {
    int32_t u;
    if (!get_row<M>(n, list, nlist, u)) return;
    const int32_t s = rp[u], e = rp[u + 1];
    if (M == M_THR && e - s > kLongRow) return;
    if (state[u] != ST_U) {
        if (tlane<M>() == 0) best[u] = -1;
        return;
    }
    double bs = -1.0;
    int32_t bv = -1;
    for (int32_t j = s + tlane<M>(); j < e; j += tstride<M>()) {
        const int32_t v = col[j];
        const double sc = score[j];
        if (sc < 0.0 || state[v] == ST_A) continue;
        best_merge(bs, bv, sc, v);
    }
    bv = reduce_best<M>(bs, bv);
    if (tlane<M>() == 0) best[u] = bv;
}

__global__ void k_resolve(int32_t n, const int32_t *__restrict__ state, const int32_t *__restrict__ best,
                          int32_t *__restrict__ nstate, int32_t *__restrict__ nseed, int32_t *changed) {
    const int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    if (state[u] != ST_U) return;
    const int32_t v = best[u];
    if (v < 0) return;
    if (state[v] == ST_S) {
        nstate[u] = ST_A;
        nseed[u] = v;
        *changed = 1;
    } else if (state[v] == ST_U && best[v] == u) {
        const int32_t lo = u < v ? u : v, hi = u < v ? v : u;
        nstate[lo] = ST_S;
        nstate[hi] = ST_A;
        nseed[hi] = lo;
        *changed = 1;
    }
}

// ---------------------------------------------------------------------------
// The paper's aggregation scan (Sec. 3.4.2; agg_rule 1 and 2).  One stage visits
// the undecided nodes in the order of rank (0 first); a node u that is still
// undecided at its turn joins its best admissible neighbour that is a seed or
// undecided (the largest score, ties to the lower index; an undecided one
// becomes a seed).  Parallel rounds reproduce the sequential stage exactly.
//
// A node is active while it is undecided and has not had its turn.  u's choice
// is the first of its candidates, in its order of preference, that has not
// become an associate; whether a candidate is a seed or undecided does not
// change the choice, and a candidate becomes an associate only by its own turn.
// Candidates ranked after u's best seed candidate never matter (a seed stays a
// seed).  So u's decision is fixed once no active neighbour v of smaller rank
//   (a) is a candidate of u preferred to u's best seed candidate (v may still
//       become an associate), or
//   (b) has u as a candidate preferred to v's own best seed candidate (v may
//       still make u a seed).
// Nodes deciding in the same round cannot touch each other's candidates or
// themselves, so their decisions commute.  Every round decides at least the
// active node of smallest rank.
// ---------------------------------------------------------------------------

// (s1, v1) preferred to (s2, v2): larger score, ties to the lower index; v2 < 0 is none
__device__ __forceinline__ bool pref(double s1, int32_t v1, double s2, int32_t v2) {
    return v2 < 0 || s1 > s2 || (s1 == s2 && v1 < v2);
}

// rank of each node in the scan order: by decreasing splitmix64(key + u), ties to
// the lower index (keys ~hash sorted ascending by a stable sort of u = 0..n-1)
__global__ void k_scan_keys(int32_t n, uint64_t key, uint64_t *__restrict__ keys, int32_t *__restrict__ idx) {
    const int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    keys[u] = ~splitmix64(key + (uint64_t)u);
    idx[u] = u;
}
__global__ void k_scan_rank(int32_t n, const int32_t *__restrict__ order, int32_t *__restrict__ rank) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rank[order[i]] = i;
}
__global__ void k_iota(int32_t n, int32_t *__restrict__ a) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = i;
}
__global__ void k_scan_stage_init(int32_t n, const int32_t *__restrict__ state, uint8_t *__restrict__ done) {
    const int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n) done[u] = state[u] != ST_U ? 1 : 0;
}
// rev[j]: the entry (v -> u) of entry j = (u -> v); rows are sorted by column
__global__ void k_rev_entries(int64_t nnz, const int32_t *__restrict__ erow, const int32_t *__restrict__ rp,
                              const int32_t *__restrict__ col, int32_t *__restrict__ rev) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nnz) return;
    const int32_t u = erow[j], v = col[j];
    int32_t lo = rp[v], hi = rp[v + 1] - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (col[mid] < u) lo = mid + 1;
        else hi = mid;
    }
    // a symmetric graph has col[lo] == u; otherwise (an unchecked input) -1
    rev[j] = (lo < rp[v + 1] && col[lo] == u) ? lo : -1;
}

// per active node: its preferred seed candidate (score, index), or index -1
template <int M>
__global__ void __launch_bounds__(M == M_BLK ? kBlk : 256) k_scan_bests(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                             const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                             const double *__restrict__ score, const int32_t *__restrict__ state,
                             const uint8_t *__restrict__ done, double *__restrict__ bs_out,
                             int32_t *__restrict__ bv_out) {
    int32_t u;
    if (!get_row<M>(n, list, nlist, u)) return;
    const int32_t s = rp[u], e = rp[u + 1];
    if (M == M_THR && e - s > kLongRow) return;
    if (state[u] != ST_U || done[u]) return;   // read only for active nodes
    double bs = -1.0;
    int32_t bv = -1;
    for (int32_t j = s + tlane<M>(); j < e; j += tstride<M>()) {
        const int32_t v = col[j];
        const double sc = score[j];
        if (sc >= 0.0 && state[v] == ST_S) best_merge(bs, bv, sc, v);
    }
    reduce_best_pair<M>(bs, bv);
    if (tlane<M>() == 0) {
        bv_out[u] = bv;
        bs_out[u] = bs;
    }
}

// per active node u: whether it decides this round, and its decision:
// dec[u] = -2 (waits, or not active), -1 (no candidate), else the chosen node
template <int M>
__global__ void __launch_bounds__(M == M_BLK ? kBlk : 256) k_scan_decide(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                              const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                              const int32_t *__restrict__ rev, const double *__restrict__ score,
                              const int32_t *__restrict__ rank, const int32_t *__restrict__ state,
                              const uint8_t *__restrict__ done, const double *__restrict__ bs_seed,
                              const int32_t *__restrict__ bv_seed, int32_t *__restrict__ dec,
                              int32_t *__restrict__ waiting) {
    int32_t u;
    if (!get_row<M>(n, list, nlist, u)) return;
    const int32_t s = rp[u], e = rp[u + 1];
    if (M == M_THR && e - s > kLongRow) return;
    if (state[u] != ST_U || done[u]) {
        if (tlane<M>() == 0) dec[u] = -2;
        return;
    }
    const int32_t ru = rank[u];
    const double su = bs_seed[u];
    const int32_t vu = bv_seed[u];
    bool blocked = false;
    double bs = -1.0;
    int32_t bv = -1;
    for (int32_t j = s + tlane<M>(); j < e; j += tstride<M>()) {
        const int32_t v = col[j];
        const int32_t sv = state[v];
        const double sc = score[j];
        const bool cand = sc >= 0.0 && (sv == ST_U || sv == ST_S);
        if (sv == ST_U && !done[v] && rank[v] < ru) {
            if (cand && pref(sc, v, su, vu)) blocked = true;                      // (a)
            const int32_t rj = rev[j];
            if (rj < 0) blocked = true;   // no reverse entry: wait for v (exact, conservative)
            else if (score[rj] >= 0.0 && pref(score[rj], u, bs_seed[v], bv_seed[v])) blocked = true;  // (b)
        }
        if (cand) best_merge(bs, bv, sc, v);
    }
    blocked = reduce_any<M>(blocked);
    bv = reduce_best<M>(bs, bv);
    if (tlane<M>() == 0) {
        dec[u] = blocked ? -2 : bv;
        if (blocked) atomicAdd(waiting, 1);
    }
}

__global__ void k_scan_apply(int32_t n, const int32_t *__restrict__ dec, int32_t *__restrict__ state,
                             uint8_t *__restrict__ done, int32_t *__restrict__ seed, int32_t *changed) {
    const int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int32_t d = dec[u];
    if (d == -2) return;
    done[u] = 1;
    if (d < 0) return;
    state[d] = ST_S;
    state[u] = ST_A;
    seed[u] = d;
    *changed = 1;
}

__global__ void k_count_su(const int32_t *__restrict__ state, int32_t n, unsigned long long *out) {
    const int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c = 0;
    if (u < n) c = (state[u] == ST_S || state[u] == ST_U) ? 1ull : 0ull;
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

__global__ void k_seed_flags(const int32_t *__restrict__ state, int32_t n, int32_t *__restrict__ f) {
    const int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n) f[u] = (state[u] == ST_S || state[u] == ST_U) ? 1 : 0;
}

__global__ void k_number_seeds(const int32_t *__restrict__ state, const int32_t *__restrict__ pos,
                               int32_t n, int32_t *__restrict__ agg) {
    const int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n && (state[u] == ST_S || state[u] == ST_U)) agg[u] = pos[u];
}

__global__ void k_number_rest(const int32_t *__restrict__ state, const int32_t *__restrict__ seed,
                              int32_t n, int32_t ndummy_id, int32_t *__restrict__ agg) {
    const int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    if (state[u] == ST_A) agg[u] = agg[seed[u]];
    else if (state[u] == ST_D) agg[u] = ndummy_id;
}

// ---------------------------------------------------------------------------
// Galerkin P^T A P (Eq. (2.5)) with the canonical summation order: for U < V,
// the fine entries (u -> v), u in T_U, v in T_V, in increasing (u, v)
// (= stable sort of the CSR order by (U, V)), summed canonically.
// ---------------------------------------------------------------------------

__global__ void k_gal_flag(int64_t nnz, const int32_t *__restrict__ erow, const int32_t *__restrict__ col,
                           const int32_t *__restrict__ agg, uint8_t *__restrict__ f) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nnz) f[j] = agg[erow[j]] < agg[col[j]] ? 1 : 0;
}

__global__ void k_gal_keys(int64_t M, const int32_t *__restrict__ idx, const int32_t *__restrict__ erow,
                           const int32_t *__restrict__ col, const double *__restrict__ w,
                           const int32_t *__restrict__ agg, int64_t nc, uint64_t *__restrict__ key,
                           double *__restrict__ val) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int32_t j = idx[i];
    key[i] = (uint64_t)agg[erow[j]] * (uint64_t)nc + (uint64_t)agg[col[j]];
    val[i] = w[j];
}

__global__ void k_seg_heads(int64_t M, const uint64_t *__restrict__ key, uint8_t *__restrict__ f) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) f[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}

// segment p covers [start[p], start[p+1]) (the last one ends at M): an rp-like array
__global__ void k_seg_ptr(int64_t P, const int32_t *__restrict__ start, int64_t M, int32_t *__restrict__ sp) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) sp[p] = start[p];
    if (p == P) sp[P] = (int32_t)M;
}

template <int M>
__global__ void __launch_bounds__(M == M_BLK ? kBlk : 256) k_seg_sum(int32_t P, const int32_t *__restrict__ list, int32_t nlist,
                          const int32_t *__restrict__ sp, const double *__restrict__ val, double *__restrict__ W) {
    int32_t p;
    if (!get_row<M>(P, list, nlist, p)) return;
    const int32_t s = sp[p], e = sp[p + 1];
    if (M == M_THR && e - s > kLongRow) return;
    double acc = 0.0;
    for (int32_t j = s + tlane<M>(); j < e; j += tstride<M>()) acc = acc + val[j];
    acc = canon_reduce<M>(acc);
    if (tlane<M>() == 0) W[p] = acc;
}

__global__ void k_gal_dir(int64_t P, const int32_t *__restrict__ start, const uint64_t *__restrict__ key,
                          const double *__restrict__ W, uint64_t nc, uint64_t *__restrict__ key2,
                          double *__restrict__ val2) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const uint64_t k = key[start[p]];
    const uint64_t U = k / nc, V = k % nc;
    key2[2 * p] = U * nc + V;
    val2[2 * p] = W[p];
    key2[2 * p + 1] = V * nc + U;
    val2[2 * p + 1] = W[p];
}

__global__ void k_gal_csr(int64_t E, const uint64_t *__restrict__ key2, const double *__restrict__ val2,
                          uint64_t nc, int32_t *__restrict__ col, double *__restrict__ w,
                          int32_t *__restrict__ rowcnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= E) return;
    const uint64_t k = key2[i];
    col[i] = (int32_t)(k % nc);
    w[i] = val2[i];
    atomicAdd(&rowcnt[k / nc], 1);
}

// ---------------------------------------------------------------------------
// Low-degree elimination (Sec. 3.2).  F: one sweep through the nodes in
// decreasing priority splitmix64(key + u) (ties: lower index); an eligible node
// of degree 1..4 joins F and its neighbours become ineligible.  Equivalently, a
// candidate is in F iff none of its higher-priority candidate neighbours is;
// rounds decide every candidate whose higher-priority candidate neighbours are
// all decided (the states only move forward, so a stale read only delays a
// decision, and the result is the sweep's).
// ---------------------------------------------------------------------------

enum : int32_t { EL_UND = 0, EL_IN = 1, EL_OUT = 2, EL_NONE = 3 };

__global__ void k_elim_init(int32_t n, const int32_t *__restrict__ rp, uint64_t key, uint64_t *__restrict__ prio,
                            int32_t *__restrict__ state) {
    const int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int32_t d = rp[u + 1] - rp[u];
    state[u] = (d >= 1 && d <= 4) ? EL_UND : EL_NONE;
    prio[u] = splitmix64(key + (uint64_t)u);
}

__global__ void k_elim_round(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                             const uint64_t *__restrict__ prio, int32_t *state, int32_t *left) {
    const int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n || ((volatile int32_t *)state)[u] != EL_UND) return;
    const uint64_t pu = prio[u];
    bool wait = false, out = false;
    for (int32_t e = rp[u]; e < rp[u + 1]; e++) {   // at most 4 entries
        const int32_t v = col[e];
        const int32_t sv = ((volatile int32_t *)state)[v];
        if (sv != EL_UND && sv != EL_IN) continue;
        const uint64_t pv = prio[v];
        if (pv > pu || (pv == pu && v < u)) {
            if (sv == EL_IN) out = true;
            else wait = true;
        }
    }
    if (out) state[u] = EL_OUT;
    else if (!wait) state[u] = EL_IN;
    else atomicAdd(left, 1);
}

__global__ void k_elim_cflag(int32_t n, const int32_t *__restrict__ state, int32_t *__restrict__ f) {
    const int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n) f[u] = state[u] == EL_IN ? 0 : 1;
    if (u == n) f[n] = 0;
}

__global__ void k_elim_cidx(int32_t n, const int32_t *__restrict__ state, const int32_t *__restrict__ pos,
                            int32_t *__restrict__ cidx) {
    const int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n) cidx[u] = state[u] == EL_IN ? -1 : pos[u];
}

// Schur complement on C (Eq. (3.1)); A_FF is diagonal, so for c1 < c2
// W^c = w_{c1 c2} + sum over f in F adjacent to both of (w_{f c1} w_{f c2}) / a_ff.
// Terms: the direct C-C entries (c1 < c2) in CSR order, then every f's
// neighbour pairs in increasing f; a stable sort by (c1, c2) keeps, within one
// pair, the direct term first and the fill terms by increasing f, the order
// the canonical sum takes (bit-identical to the oracle).  The sums are then
// mirrored into the coarse CSR exactly as in the Galerkin step.
__global__ void k_elim_dflag(int64_t nnz, const int32_t *__restrict__ erow, const int32_t *__restrict__ col,
                             const int32_t *__restrict__ cidx, uint8_t *__restrict__ f) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nnz) return;
    const int32_t u = erow[j], v = col[j];
    f[j] = (cidx[u] >= 0 && cidx[v] >= 0 && u < v) ? 1 : 0;
}

__global__ void k_elim_npairs(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ cidx,
                              int32_t *__restrict__ cnt) {
    const int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n) {
        const int32_t d = rp[u + 1] - rp[u];
        cnt[u] = cidx[u] < 0 ? d * (d - 1) / 2 : 0;
    }
    if (u == n) cnt[n] = 0;
}

__global__ void k_elim_fill(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                            const double *__restrict__ w, const int32_t *__restrict__ cidx,
                            const double *__restrict__ diag, const int32_t *__restrict__ off, uint64_t nc,
                            uint64_t *__restrict__ key, double *__restrict__ val) {
    const int32_t f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n || cidx[f] >= 0) return;
    int64_t o = off[f];
    const int32_t s = rp[f], e = rp[f + 1];
    for (int32_t i = s; i < e; i++)
        for (int32_t j = i + 1; j < e; j++) {
            const uint64_t a = (uint64_t)cidx[col[i]], b = (uint64_t)cidx[col[j]];
            key[o] = a < b ? a * nc + b : b * nc + a;
            val[o] = __ddiv_rn(__dmul_rn(w[i], w[j]), diag[f]);
            o++;
        }
}

__global__ void k_elim_dkeys(int64_t M, const int32_t *__restrict__ idx, const int32_t *__restrict__ erow,
                             const int32_t *__restrict__ col, const double *__restrict__ w,
                             const int32_t *__restrict__ cidx, uint64_t nc, uint64_t *__restrict__ key,
                             double *__restrict__ val) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int32_t j = idx[i];
    key[i] = (uint64_t)cidx[erow[j]] * nc + (uint64_t)cidx[col[j]];
    val[i] = w[j];
}

// ---------------------------------------------------------------------------
// Driver
// ---------------------------------------------------------------------------

static void build_tiers(const int32_t *rp, int32_t n, Tiers &t, cudaStream_t s) {
    t.nw = tier_list(rp, n, 1, nullptr, t.w.get(), s);
    t.nb = tier_list(rp, n, 2, nullptr, t.b.get(), s);
}

// Grid of a cooperative setup kernel on the current device: one kBlk-thread
// block per SM (the kernels' launch bounds guarantee one fits).
static int coop_grid(const void *kernel, const char *what) {
    int dev = 0, sms = 0, per = 0;
    LAMG_CUDA(cudaGetDevice(&dev));
    LAMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LAMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kBlk, 0));
    LAMG_REQUIRE(per >= 1, LAMG_ERR_CUDA, std::string(what) + " cannot be resident");
    return sms;
}

// Lean Geometric Multigrid (Sec. 6): node u = (row u / nx, column u % nx) of an
// nx x nx periodic grid; red-black colours and 2x2 aggregates numbered row by row
__global__ void k_rb_colour(int32_t n, int32_t nx, int32_t *__restrict__ colour) {
    const int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n) colour[u] = ((u % nx) + (u / nx)) & 1;
}
__global__ void k_geo_agg(int32_t n, int32_t nx, int32_t *__restrict__ agg, int32_t *__restrict__ state) {
    const int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    agg[u] = (u / nx) / 2 * (nx / 2) + (u % nx) / 2;
    state[u] = 0;
}

// Lexicographic Gauss-Seidel as a colour-ordered sweep (relax_rule 1): colour[u] =
// 1 + the largest colour of a lower-index neighbour, the level sets of the lower-
// triangular dependency graph, found by peeling: wait[u] counts the lower-index
// neighbours not yet coloured; round r colours the frontier (wait 0) with r and
// releases their higher-index neighbours.  Colours do not depend on the order in
// which a round's frontier is listed.
__global__ void k_lex_wait(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                           int32_t *__restrict__ wait, uint8_t *__restrict__ ready) {
    const int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    int32_t c = 0;
    for (int32_t j = rp[u]; j < rp[u + 1]; j++) c += col[j] < u ? 1 : 0;
    wait[u] = c;
    ready[u] = c == 0 ? 1 : 0;
}
__global__ void k_lex_round(const int32_t *__restrict__ front, int32_t nf, int32_t r,
                            const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                            int32_t *__restrict__ wait, int32_t *__restrict__ colour,
                            int32_t *__restrict__ next, int32_t *__restrict__ nnext) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const int32_t u = front[i];
    colour[u] = r;
    for (int32_t j = rp[u]; j < rp[u + 1]; j++) {
        const int32_t v = col[j];
        if (v > u && atomicSub(&wait[v], 1) == 1) next[atomicAdd(nnext, 1)] = v;
    }
}

static void colour_lex(SetupLevel &L, cudaStream_t s) {
    const int32_t n = L.n;
    Tmp<int32_t> wait(n, s), fa(n, s), fb(n, s), cnt(1, s);
    Tmp<uint8_t> ready(n, s);
    k_lex_wait<<<ceil_div(n, 256), 256, 0, s>>>(n, L.rp.get(), L.col.get(), wait.get(), ready.get());
    LAMG_CHECK_LAUNCH();
    int32_t nf = (int32_t)compact_indices(ready.get(), fa.get(), n, s);
    int32_t *cur = fa.get(), *nxt = fb.get();
    int64_t done = 0;
    for (int32_t r = 0; nf > 0; r++) {
        done += nf;
        LAMG_REQUIRE(done <= n, LAMG_ERR_CUDA, "lexicographic colouring: frontier overran the level");
        LAMG_CUDA(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t), s));
        k_lex_round<<<ceil_div(nf, 256), 256, 0, s>>>(cur, nf, r, L.rp.get(), L.col.get(), wait.get(),
                                                       L.colour.get(), nxt, cnt.get());
        LAMG_CHECK_LAUNCH();
        nf = read_scalar(cnt.get(), s);
        std::swap(cur, nxt);
    }
    LAMG_REQUIRE(done == n, LAMG_ERR_CUDA, "lexicographic colouring: some nodes were never released");
}

// The JP colouring of a level that relaxes, and the (colour, tier, id) order of
// its nodes.  A level followed by elimination never relaxes (nu = 0, Sec. 4.2):
// it gets one colour, 0, and only the order.  rb_nx > 0: red-black colours of an
// rb_nx x rb_nx periodic grid instead of JP.
static void colour_level(lamg_ctx *h, SetupLevel &L, int level, const Tiers &T, int32_t rb_nx, cudaStream_t s,
                         bool relaxes = true) {
    const int32_t n = L.n;
    L.colour.alloc(n);
    k_fill_i32<<<ceil_div(n, 256), 256, 0, s>>>(L.colour.get(), n, relaxes ? -1 : 0);
    LAMG_CHECK_LAUNCH();
    int32_t batch_rounds = 0;
    const int32_t fin_rounds = 0;
    if (relaxes && rb_nx > 0) {
        k_rb_colour<<<ceil_div(n, 256), 256, 0, s>>>(n, rb_nx, L.colour.get());
        LAMG_CHECK_LAUNCH();
    } else if (relaxes && h->opt.relax_rule == 1) {
        colour_lex(L, s);
    } else if (relaxes) {
        const uint64_t key = colour_key(h->opt.seed, level);
        {
        // wait counts, the first frontier, then all rounds in one cooperative launch
        Tmp<int32_t> deg(n, s), wait(n, s);
        Tmp<uint64_t> hsh(n, s);
        k_jp_prio<<<ceil_div(n, 256), 256, 0, s>>>(n, L.rp.get(), key, h->opt.colour_rule == 0 ? 1 : 0, deg.get(),
                                                   hsh.get());
        LAMG_CHECK_LAUNCH();
        LAUNCH3(k_jp_wait, n, (const int32_t *)nullptr, T.w.get(), T.nw, T.b.get(), T.nb, s, L.rp.get(), L.col.get(),
                deg.get(), hsh.get(), wait.get());
        const int64_t cap = n;
        Tmp<int32_t> lst(6 * (size_t)cap, s), fcnt(6, s), out(1, s), err(1, s);
        Tmp<unsigned int> bar(2, s);
        int32_t c6[6] = {0, 0, 0, 0, 0, 0};
        {
            Tmp<uint8_t> f(n, s);
            for (int t = 0; t < 3; t++) {
                k_jp_ready<<<ceil_div(n, 256), 256, 0, s>>>(L.rp.get(), n, t, wait.get(), f.get());
                LAMG_CHECK_LAUNCH();
                c6[t] = (int32_t)compact_indices(f.get(), lst.get() + t * cap, n, s);
            }
        }
        LAMG_CUDA(cudaMemcpyAsync(fcnt.get(), c6, sizeof(c6), cudaMemcpyHostToDevice, s));
        LAMG_CUDA(cudaMemsetAsync(bar.get(), 0, 2 * sizeof(unsigned int), s));
        LAMG_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int32_t), s));
        Tmp<unsigned int> gbits((size_t)kSpreadHubs * kFreeWords, s);   // hub colour bitmaps, kept zeroed by the kernel
        LAMG_CUDA(cudaMemsetAsync(gbits.get(), 0, sizeof(unsigned int) * kSpreadHubs * kFreeWords, s));
        const int grid = coop_grid((const void *)k_jp_dag, "colouring kernel");
        {
            const int32_t *rpp = L.rp.get(), *colp = L.col.get(), *dp = deg.get();
            const uint64_t *hp = hsh.get();
            int32_t *wp = wait.get(), *colour = L.colour.get(), *lp = lst.get(), *cp = fcnt.get(), *op = out.get(),
                    *ep = err.get();
            int64_t capv = cap;
            unsigned int *bp = bar.get(), *gb = gbits.get();
            void *args[] = {&rpp, &colp, &dp, &hp, &wp, &colour, &lp, &capv, &cp, &op, &bp, &ep, &gb};
            LAMG_CUDA(cudaLaunchCooperativeKernel((void *)k_jp_dag, dim3(grid), dim3(kBlk), args, 0, s));
            note_launch();
        }
        LAMG_REQUIRE(read_scalar(err.get(), s) == 0, LAMG_ERR_TIMEOUT, "colouring: grid barrier timed out");
        batch_rounds = read_scalar(out.get(), s);
        }
    }
    L.jp_rounds = batch_rounds + fin_rounds;
    L.ncolours = reduce_max_i32(L.colour.get(), n, s) + 1;
    // nodes sorted by (colour, tier, id) and the ranges of each (colour, tier)
    const int nbins = 3 * L.ncolours;
    L.sorder.alloc(n);
    Tmp<uint32_t> keys(n, s), ktmp(n, s);
    Tmp<int32_t> vtmp(n, s), cnt(nbins + 1, s), off(nbins + 1, s);
    k_order_keys<<<ceil_div(n, 256), 256, 0, s>>>(L.rp.get(), L.colour.get(), n, keys.get(), L.sorder.get());
    LAMG_CHECK_LAUNCH();
    radix_sort_pairs<uint32_t, int32_t>(keys.get(), L.sorder.get(), ktmp.get(), vtmp.get(), n,
                                        bits_for((uint64_t)nbins - 1), s);
    LAMG_CUDA(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t) * (nbins + 1), s));
    k_hist_u32<<<ceil_div(n, 256), 256, 0, s>>>(keys.get(), n, cnt.get());
    LAMG_CHECK_LAUNCH();
    exclusive_scan_i32(cnt.get(), off.get(), nbins + 1, s);
    std::vector<int32_t> hoff(nbins + 1);
    LAMG_CUDA(cudaMemcpyAsync(hoff.data(), off.get(), sizeof(int32_t) * (nbins + 1), cudaMemcpyDeviceToHost, s));
    LAMG_CUDA(cudaStreamSynchronize(s));
    L.cb.assign(4 * L.ncolours, 0);
    for (int c = 0; c < L.ncolours; c++)
        for (int t = 0; t < 4; t++) L.cb[4 * c + t] = hoff[3 * c + t];
    L.cb_dev.alloc(L.cb.size());
    LAMG_CUDA(cudaMemcpyAsync(L.cb_dev.get(), L.cb.data(), sizeof(int32_t) * L.cb.size(), cudaMemcpyHostToDevice, s));
}

// Colours whose sweep is cheap enough for one block: no block-tier rows and
// (entries of the colour) * K <= kTailWork.  Consecutive such colours are
// swept by one single-block launch; the others by their own launches.
constexpr int64_t kTailWork = 16384;

__global__ void k_colour_entries(const int32_t *__restrict__ rp, const int32_t *__restrict__ colour, int32_t n,
                                 int32_t *__restrict__ ent) {
    const int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n) atomicAdd(&ent[colour[u]], rp[u + 1] - rp[u]);
}

// TVs and their sweeps; returns the largest per-TV energy ratio of the last
// sweep when the relaxation-speed test is enabled (else +inf).
static double relax_tvs(lamg_ctx *h, SetupLevel &L, int level, const Tiers &T, const double *diag, double *X,
                        cudaStream_t s) {
    const int32_t n = L.n, K = L.K;
    const lamg_options &o = h->opt;
    k_tv_init<<<ceil_div((int64_t)n * K, 256), 256, 0, s>>>(X, (int64_t)n * K, tv_key(o.seed, level));
    LAMG_CHECK_LAUNCH();
    const int32_t *ord = L.sorder.get();
    const bool test = o.relax_fast_ratio > 0.0 && o.nu_tv >= 2;
    Tmp<double> eu(test ? n : 0, s);
    double eprev[16], ecur[16];
    // per-colour entry counts -> which colours the single-block sweep takes
    std::vector<int32_t> ent(L.ncolours);
    {
        Tmp<int32_t> de(L.ncolours, s);
        LAMG_CUDA(cudaMemsetAsync(de.get(), 0, sizeof(int32_t) * L.ncolours, s));
        k_colour_entries<<<ceil_div(n, 256), 256, 0, s>>>(L.rp.get(), L.colour.get(), n, de.get());
        LAMG_CHECK_LAUNCH();
        LAMG_CUDA(cudaMemcpyAsync(ent.data(), de.get(), sizeof(int32_t) * L.ncolours, cudaMemcpyDeviceToHost, s));
        LAMG_CUDA(cudaStreamSynchronize(s));
    }
    auto small = [&](int c) {
        return L.cb[4 * c + 3] == L.cb[4 * c + 2] && (int64_t)ent[c] * K <= kTailWork;
    };
    if (!test && o.nu_tv > 0) {
        // every sweep in one cooperative launch (the energy test, when on, needs the host between sweeps)
        std::vector<int32_t> plan;
        for (int c = 0; c < L.ncolours;) {
            if (small(c)) {
                int c1 = c;
                while (c1 < L.ncolours && small(c1)) c1++;
                plan.insert(plan.end(), {c, c1, 1});
                c = c1;
            } else {
                plan.insert(plan.end(), {c, c + 1, 0});
                c++;
            }
        }
        int32_t maxbr = 0;
        for (size_t q = 0; q < plan.size(); q += 3)
            if (!plan[q + 2]) maxbr = std::max(maxbr, L.cb[4 * plan[q] + 3] - L.cb[4 * plan[q] + 2]);
        Tmp<double> gsum((size_t)maxbr * 32 * K, s);
        Tmp<int32_t> dplan(plan.size(), s);
        Tmp<unsigned int> bar(2, s);
        Tmp<int32_t> err(1, s);
        LAMG_CUDA(cudaMemcpyAsync(dplan.get(), plan.data(), sizeof(int32_t) * plan.size(), cudaMemcpyHostToDevice, s));
        LAMG_CUDA(cudaMemsetAsync(bar.get(), 0, 2 * sizeof(unsigned int), s));
        LAMG_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int32_t), s));
        const int grid = coop_grid((const void *)k_tv_sweeps_coop, "TV sweep kernel");
        int32_t nsw = o.nu_tv, npl = (int32_t)(plan.size() / 3);
        const int32_t *pp = dplan.get(), *cbp = L.cb_dev.get(), *rpp = L.rp.get(), *colp = L.col.get();
        const double *wp = L.w.get();
        unsigned int *barp = bar.get();
        int32_t *errp = err.get();
        int32_t Kv = K;
        double *gp = gsum.get();
        unsigned long long *tp = nullptr;   // per-phase clock (kernel support kept; off)
        void *args[] = {&nsw, &pp, &npl, &cbp, &ord, &rpp, &colp, &wp, &diag, &Kv, &X, &barp, &errp, &gp, &tp};
        LAMG_CUDA(cudaLaunchCooperativeKernel((void *)k_tv_sweeps_coop, dim3(grid), dim3(kBlk), args, 0, s));
        note_launch();
        LAMG_REQUIRE(read_scalar(err.get(), s) == 0, LAMG_ERR_TIMEOUT, "TV sweep: grid barrier timed out");
        return INFINITY;
    }
    for (int sw = 1; sw <= o.nu_tv; sw++) {
        for (int c = 0; c < L.ncolours;) {
            if (small(c)) {
                int c1 = c;
                while (c1 < L.ncolours && small(c1)) c1++;
                k_tv_sweep_tail<<<1, kBlk, 0, s>>>(c, c1, L.cb_dev.get(), ord, L.rp.get(), L.col.get(), L.w.get(),
                                                   diag, K, X);
                LAMG_CHECK_LAUNCH();
                c = c1;
                continue;
            }
            const int32_t t0 = L.cb[4 * c], t1 = L.cb[4 * c + 1], t2 = L.cb[4 * c + 2], t3 = L.cb[4 * c + 3];
            if (t1 > t0) {
                k_tv_sweep<M_THR><<<ceil_div(t1 - t0, 256), 256, 0, s>>>(t1 - t0, ord + t0, 0, L.rp.get(),
                                                                        L.col.get(), L.w.get(), diag, K, X);
                LAMG_CHECK_LAUNCH();
            }
            if (t2 > t1) {
                k_tv_sweep<M_WARP><<<ceil_div((int64_t)(t2 - t1) * 32, 256), 256, 0, s>>>(
                    0, ord + t1, t2 - t1, L.rp.get(), L.col.get(), L.w.get(), diag, K, X);
                LAMG_CHECK_LAUNCH();
            }
            if (t3 > t2) {
                k_tv_sweep<M_BLK><<<t3 - t2, kBlk, 0, s>>>(0, ord + t2, t3 - t2, L.rp.get(), L.col.get(),
                                                          L.w.get(), diag, K, X);
                LAMG_CHECK_LAUNCH();
            }
            c++;
        }
        if (test && sw >= o.nu_tv - 1) {
            for (int k = 0; k < K; k++) {
                LAUNCH3(k_tv_energy, n, (const int32_t *)nullptr, T.w.get(), T.nw, T.b.get(), T.nb, s, L.rp.get(),
                        L.col.get(), L.w.get(), K, k, X, eu.get());
                double E = canon_sum_global(eu.get(), n, s);
                if (sw == o.nu_tv - 1) eprev[k] = E; else ecur[k] = E;
            }
        }
    }
    if (!test) return INFINITY;
    double worst = 0.0;
    for (int k = 0; k < K; k++) {
        double r = eprev[k] > 0.0 ? ecur[k] / eprev[k] : 0.0;
        if (r > worst) worst = r;
    }
    return worst;
}

// Aggregation of one level; fills L.agg, L.state, L.nc, L.alpha, L.rounds, L.sel_round.
static void aggregate_level(lamg_ctx *h, SetupLevel &L, int level, const Tiers &T, const double *score,
                            const double *maxw, cudaStream_t s) {
    const int32_t n = L.n;
    const lamg_options &o = h->opt;
    Tmp<int32_t> state(n, s), seed(n, s), best(n, s), nstate(n, s), nseed(n, s), bseed(n, s);
    L.state.alloc(n);
    L.agg.alloc(n);
    LAUNCH3(k_node_state, n, (const int32_t *)nullptr, T.w.get(), T.nw, T.b.get(), T.nb, s, L.rp.get(), L.col.get(),
            L.w.get(), maxw, o.weak_tol, L.hub.get(), state.get());
    LAMG_CUDA(cudaMemsetAsync(seed.get(), 0xFF, sizeof(int32_t) * n, s));
    const int64_t nd = count_equal_i32(state.get(), n, ST_D, s);
    const double amax = 0.7 / o.gamma;
    double best_alpha = INFINITY;
    int best_round = 0, r;
    Tmp<int32_t> changed(1, s);
    Tmp<unsigned long long> cnt(1, s);
    const bool scan = o.agg_rule != 0;
    const int max_stages = scan ? std::min(o.max_rounds, 2) : o.max_rounds;
    Tmp<int32_t> rank(scan ? n : 0, s), bvs(scan ? n : 0, s), dec(scan ? n : 0, s), waiting(scan ? 1 : 0, s),
        rev(scan ? L.nnz : 0, s);
    Tmp<double> bss(scan ? n : 0, s);
    Tmp<uint8_t> done(scan ? n : 0, s);
    if (scan) {
        if (L.nnz > 0) {
            Tmp<int32_t> erow(L.nnz, s);
            LAUNCH3(k_entry_rows, n, (const int32_t *)nullptr, T.w.get(), T.nw, T.b.get(), T.nb, s, L.rp.get(),
                    erow.get());
            k_rev_entries<<<ceil_div(L.nnz, 256), 256, 0, s>>>(L.nnz, erow.get(), L.rp.get(), L.col.get(),
                                                                rev.get());
            LAMG_CHECK_LAUNCH();
        }
        if (o.agg_rule == 1) {   // the paper's index order
            k_iota<<<ceil_div(n, 256), 256, 0, s>>>(n, rank.get());
            LAMG_CHECK_LAUNCH();
        } else {                 // hashed priority order
            Tmp<uint64_t> keys(n, s), ktmp(n, s);
            Tmp<int32_t> order(n, s), vtmp(n, s);
            k_scan_keys<<<ceil_div(n, 256), 256, 0, s>>>(n, agg_key(o.seed, level), keys.get(), order.get());
            LAMG_CHECK_LAUNCH();
            radix_sort_pairs<uint64_t, int32_t>(keys.get(), order.get(), ktmp.get(), vtmp.get(), n, 64, s);
            k_scan_rank<<<ceil_div(n, 256), 256, 0, s>>>(n, order.get(), rank.get());
            LAMG_CHECK_LAUNCH();
        }
    }
    for (r = 1; r <= max_stages; r++) {
        if (scan) {
            LAMG_CUDA(cudaMemsetAsync(changed.get(), 0, sizeof(int32_t), s));
            k_scan_stage_init<<<ceil_div(n, 256), 256, 0, s>>>(n, state.get(), done.get());
            LAMG_CHECK_LAUNCH();
            for (int64_t round = 0;; round++) {
                // every round decides at least the active node of smallest rank
                LAMG_REQUIRE(round <= (int64_t)n, LAMG_ERR_CUDA, "aggregation scan: rounds did not converge");
                LAMG_CUDA(cudaMemsetAsync(waiting.get(), 0, sizeof(int32_t), s));
                LAUNCH3(k_scan_bests, n, (const int32_t *)nullptr, T.w.get(), T.nw, T.b.get(), T.nb, s, L.rp.get(),
                        L.col.get(), score, state.get(), done.get(), bss.get(), bvs.get());
                LAUNCH3(k_scan_decide, n, (const int32_t *)nullptr, T.w.get(), T.nw, T.b.get(), T.nb, s,
                        L.rp.get(), L.col.get(), rev.get(), score, rank.get(), state.get(), done.get(), bss.get(),
                        bvs.get(), dec.get(), waiting.get());
                k_scan_apply<<<ceil_div(n, 256), 256, 0, s>>>(n, dec.get(), state.get(), done.get(), seed.get(),
                                                              changed.get());
                LAMG_CHECK_LAUNCH();
                if (read_scalar(waiting.get(), s) == 0) break;
            }
        } else {
            LAUNCH3(k_best, n, (const int32_t *)nullptr, T.w.get(), T.nw, T.b.get(), T.nb, s, L.rp.get(),
                    L.col.get(), score, state.get(), best.get());
            LAMG_CUDA(cudaMemcpyAsync(nstate.get(), state.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
            LAMG_CUDA(cudaMemcpyAsync(nseed.get(), seed.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
            LAMG_CUDA(cudaMemsetAsync(changed.get(), 0, sizeof(int32_t), s));
            k_resolve<<<ceil_div(n, 256), 256, 0, s>>>(n, state.get(), best.get(), nstate.get(), nseed.get(),
                                                      changed.get());
            LAMG_CHECK_LAUNCH();
            LAMG_CUDA(cudaMemcpyAsync(state.get(), nstate.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
            LAMG_CUDA(cudaMemcpyAsync(seed.get(), nseed.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
        }
        LAMG_CUDA(cudaMemsetAsync(cnt.get(), 0, sizeof(unsigned long long), s));
        k_count_su<<<ceil_div(n, 256), 256, 0, s>>>(state.get(), n, cnt.get());
        LAMG_CHECK_LAUNCH();
        int32_t ch;
        unsigned long long su;
        LAMG_CUDA(cudaMemcpyAsync(&ch, changed.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LAMG_CUDA(cudaMemcpyAsync(&su, cnt.get(), sizeof(su), cudaMemcpyDeviceToHost, s));
        LAMG_CUDA(cudaStreamSynchronize(s));
        const int64_t nc = (int64_t)su + (nd > 0 ? 1 : 0);
        const double alpha = (double)nc / (double)n;
        if (fabs(alpha - amax) < fabs(best_alpha - amax)) {
            best_alpha = alpha;
            best_round = r;
            LAMG_CUDA(cudaMemcpyAsync(L.state.get(), state.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
            LAMG_CUDA(cudaMemcpyAsync(bseed.get(), seed.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
        }
        if (alpha <= amax || !ch) break;
    }
    L.rounds = r > max_stages ? max_stages : r;
    L.sel_round = best_round;
    L.alpha = best_alpha;
    // numbering: seeds (S and left-over U) by ascending index, dummy aggregate last
    Tmp<int32_t> f(n + 1, s), pos(n + 1, s);
    k_seed_flags<<<ceil_div(n, 256), 256, 0, s>>>(L.state.get(), n, f.get());
    LAMG_CHECK_LAUNCH();
    LAMG_CUDA(cudaMemsetAsync(f.get() + n, 0, sizeof(int32_t), s));
    exclusive_scan_i32(f.get(), pos.get(), n + 1, s);
    const int32_t nseeds = read_scalar(pos.get() + n, s);
    k_number_seeds<<<ceil_div(n, 256), 256, 0, s>>>(L.state.get(), pos.get(), n, L.agg.get());
    LAMG_CHECK_LAUNCH();
    k_number_rest<<<ceil_div(n, 256), 256, 0, s>>>(L.state.get(), bseed.get(), n, nseeds, L.agg.get());
    LAMG_CHECK_LAUNCH();
    L.nc = nseeds + (nd > 0 ? 1 : 0);
}

// F of level L; fills L.cidx and returns |F|
static int64_t select_elim(lamg_ctx *h, SetupLevel &L, int level, cudaStream_t s) {
    const int32_t n = L.n;
    Tmp<uint64_t> prio(n, s);
    Tmp<int32_t> state(n, s), left(1, s), f(n + 1, s), pos(n + 1, s);
    k_elim_init<<<ceil_div(n, 256), 256, 0, s>>>(n, L.rp.get(), elim_key(h->opt.seed, level), prio.get(), state.get());
    LAMG_CHECK_LAUNCH();
    for (int64_t round = 0;; round++) {
        // every round decides at least the highest-priority undecided candidate
        LAMG_REQUIRE(round <= (int64_t)n, LAMG_ERR_CUDA, "elimination: rounds did not converge");
        LAMG_CUDA(cudaMemsetAsync(left.get(), 0, sizeof(int32_t), s));
        k_elim_round<<<ceil_div(n, 256), 256, 0, s>>>(n, L.rp.get(), L.col.get(), prio.get(), state.get(), left.get());
        LAMG_CHECK_LAUNCH();
        if (read_scalar(left.get(), s) == 0) break;
    }
    k_elim_cflag<<<ceil_div(n + 1, 256), 256, 0, s>>>(n, state.get(), f.get());
    LAMG_CHECK_LAUNCH();
    exclusive_scan_i32(f.get(), pos.get(), n + 1, s);
    L.cidx.alloc(n);
    k_elim_cidx<<<ceil_div(n, 256), 256, 0, s>>>(n, state.get(), pos.get(), L.cidx.get());
    LAMG_CHECK_LAUNCH();
    const int32_t nc = read_scalar(pos.get() + n, s);
    return (int64_t)n - nc;
}

static void eliminate_level(SetupLevel &F, SetupLevel &C, const int32_t *erow, const double *diag, cudaStream_t s) {
    const int64_t nnz = F.nnz;
    const int32_t n = F.n;
    const uint64_t nc = (uint64_t)(F.n - F.nF);
    C.n = (int32_t)nc;
    // direct terms
    Tmp<uint8_t> f(nnz, s);
    Tmp<int32_t> idx(nnz, s);
    if (nnz) {
        k_elim_dflag<<<ceil_div(nnz, 256), 256, 0, s>>>(nnz, erow, F.col.get(), F.cidx.get(), f.get());
        LAMG_CHECK_LAUNCH();
    }
    const int64_t M1 = compact_indices(f.get(), idx.get(), nnz, s);
    // fill terms: d(d-1)/2 per eliminated node, d <= 4
    Tmp<int32_t> cnt(n + 1, s), off(n + 1, s);
    k_elim_npairs<<<ceil_div(n + 1, 256), 256, 0, s>>>(n, F.rp.get(), F.cidx.get(), cnt.get());
    LAMG_CHECK_LAUNCH();
    exclusive_scan_i32(cnt.get(), off.get(), n + 1, s);
    const int64_t M2 = read_scalar(off.get() + n, s);
    const int64_t M = M1 + M2;
    Tmp<uint64_t> key(M, s), ktmp(M, s);
    Tmp<double> val(M, s), vtmp(M, s);
    if (M1) {
        k_elim_dkeys<<<ceil_div(M1, 256), 256, 0, s>>>(M1, idx.get(), erow, F.col.get(), F.w.get(), F.cidx.get(),
                                                       nc, key.get(), val.get());
        LAMG_CHECK_LAUNCH();
    }
    if (M2) {
        k_elim_fill<<<ceil_div(n, 256), 256, 0, s>>>(n, F.rp.get(), F.col.get(), F.w.get(), F.cidx.get(), diag,
                                                     off.get(), nc, key.get() + M1, val.get() + M1);
        LAMG_CHECK_LAUNCH();
    }
    radix_sort_pairs<uint64_t, double>(key.get(), val.get(), ktmp.get(), vtmp.get(), M, bits_for(nc * nc - 1), s);
    Tmp<uint8_t> hf(M, s);
    Tmp<int32_t> start(M, s);
    if (M) {
        k_seg_heads<<<ceil_div(M, 256), 256, 0, s>>>(M, key.get(), hf.get());
        LAMG_CHECK_LAUNCH();
    }
    const int64_t P = compact_indices(hf.get(), start.get(), M, s);
    Tmp<double> W(P, s);
    if (P) {
        Tmp<int32_t> sp(P + 1, s);
        k_seg_ptr<<<ceil_div(P + 1, 256), 256, 0, s>>>(P, start.get(), M, sp.get());
        LAMG_CHECK_LAUNCH();
        Tiers ST((int32_t)P, s);
        build_tiers(sp.get(), (int32_t)P, ST, s);
        LAUNCH3(k_seg_sum, (int32_t)P, (const int32_t *)nullptr, ST.w.get(), ST.nw, ST.b.get(), ST.nb, s, sp.get(),
                val.get(), W.get());
    }
    const int64_t E = 2 * P;
    Tmp<uint64_t> key2(E, s), k2tmp(E, s);
    Tmp<double> val2(E, s), v2tmp(E, s);
    if (P) {
        k_gal_dir<<<ceil_div(P, 256), 256, 0, s>>>(P, start.get(), key.get(), W.get(), nc, key2.get(), val2.get());
        LAMG_CHECK_LAUNCH();
    }
    radix_sort_pairs<uint64_t, double>(key2.get(), val2.get(), k2tmp.get(), v2tmp.get(), E, bits_for(nc * nc - 1), s);
    C.nnz = E;
    C.rp.alloc(C.n + 1);
    C.col.alloc(E);
    C.w.alloc(E);
    Tmp<int32_t> rowcnt(C.n + 1, s);
    LAMG_CUDA(cudaMemsetAsync(rowcnt.get(), 0, sizeof(int32_t) * (C.n + 1), s));
    if (E) {
        k_gal_csr<<<ceil_div(E, 256), 256, 0, s>>>(E, key2.get(), val2.get(), nc, C.col.get(), C.w.get(), rowcnt.get());
        LAMG_CHECK_LAUNCH();
    }
    exclusive_scan_i32(rowcnt.get(), C.rp.get(), C.n + 1, s);
}

static void galerkin_level(SetupLevel &F, SetupLevel &C, const int32_t *erow, cudaStream_t s) {
    const int64_t nnz = F.nnz;
    const uint64_t nc = (uint64_t)F.nc;
    C.n = F.nc;
    Tmp<uint8_t> f(nnz, s);
    Tmp<int32_t> idx(nnz, s);
    if (nnz) {
        k_gal_flag<<<ceil_div(nnz, 256), 256, 0, s>>>(nnz, erow, F.col.get(), F.agg.get(), f.get());
        LAMG_CHECK_LAUNCH();
    }
    const int64_t M = compact_indices(f.get(), idx.get(), nnz, s);
    Tmp<uint64_t> key(M, s), ktmp(M, s);
    Tmp<double> val(M, s), vtmp(M, s);
    if (M) {
        k_gal_keys<<<ceil_div(M, 256), 256, 0, s>>>(M, idx.get(), erow, F.col.get(), F.w.get(),
                                                   F.agg.get(), (int64_t)nc, key.get(), val.get());
        LAMG_CHECK_LAUNCH();
    }
    radix_sort_pairs<uint64_t, double>(key.get(), val.get(), ktmp.get(), vtmp.get(), M,
                                       bits_for(nc * nc - 1), s);
    Tmp<uint8_t> hf(M, s);
    Tmp<int32_t> start(M, s);
    if (M) {
        k_seg_heads<<<ceil_div(M, 256), 256, 0, s>>>(M, key.get(), hf.get());
        LAMG_CHECK_LAUNCH();
    }
    const int64_t P = compact_indices(hf.get(), start.get(), M, s);
    Tmp<double> W(P, s);
    if (P) {
        Tmp<int32_t> sp(P + 1, s);
        k_seg_ptr<<<ceil_div(P + 1, 256), 256, 0, s>>>(P, start.get(), M, sp.get());
        LAMG_CHECK_LAUNCH();
        Tiers ST((int32_t)P, s);
        build_tiers(sp.get(), (int32_t)P, ST, s);
        LAUNCH3(k_seg_sum, (int32_t)P, (const int32_t *)nullptr, ST.w.get(), ST.nw, ST.b.get(), ST.nb, s, sp.get(),
                val.get(), W.get());
    }
    const int64_t E = 2 * P;
    Tmp<uint64_t> key2(E, s), k2tmp(E, s);
    Tmp<double> val2(E, s), v2tmp(E, s);
    if (P) {
        k_gal_dir<<<ceil_div(P, 256), 256, 0, s>>>(P, start.get(), key.get(), W.get(), nc, key2.get(),
                                                  val2.get());
        LAMG_CHECK_LAUNCH();
    }
    radix_sort_pairs<uint64_t, double>(key2.get(), val2.get(), k2tmp.get(), v2tmp.get(), E,
                                       bits_for(nc * nc - 1), s);
    C.nnz = E;
    C.rp.alloc(C.n + 1);
    C.col.alloc(E);
    C.w.alloc(E);
    Tmp<int32_t> rowcnt(C.n + 1, s);
    LAMG_CUDA(cudaMemsetAsync(rowcnt.get(), 0, sizeof(int32_t) * (C.n + 1), s));
    if (E) {
        k_gal_csr<<<ceil_div(E, 256), 256, 0, s>>>(E, key2.get(), val2.get(), nc, C.col.get(), C.w.get(),
                                                  rowcnt.get());
        LAMG_CHECK_LAUNCH();
    }
    exclusive_scan_i32(rowcnt.get(), C.rp.get(), C.n + 1, s);
}

// Cycle index per level (Eq. (4.1), build reading; see the oracle).
static void cycle_indices(lamg_ctx *h) {
    const double m1 = (double)h->sl[0].nnz / 2.0;
    for (int l = 0; l + 1 < h->L; l++) {
        if (h->sl[l].elim) { h->sl[l].gamma_l = 1.0; continue; }   // Sec. 4.2: gamma = 1 above an elimination
        if (h->opt.lgmg_nx > 0) {   // Sec. 6: a standard gamma-cycle
            h->sl[l].gamma_l = h->opt.gamma;
            continue;
        }
        const double ml = (double)h->sl[l].nnz / 2.0, mn = (double)h->sl[l + 1].nnz / 2.0;
        double g = mn > 0.0 ? 0.7 * ml / mn : 2.0;
        const double gmax = ml > 0.1 * m1 ? h->opt.gamma : h->opt.gamma_coarse_max;
        if (g > gmax) g = gmax;
        if (g < 1.0) g = 1.0;
        h->sl[l].gamma_l = g;
    }
    h->sl[h->L - 1].gamma_l = 0.0;
}

void build_hierarchy(lamg_ctx *h, int64_t n, const int64_t *row_ptr, const int32_t *col,
                     const void *w, int32_t w_is_fp32, cudaStream_t s) {
    const lamg_options &o = h->opt;
    int64_t nnz = 0;
    LAMG_CUDA(cudaMemcpyAsync(&nnz, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LAMG_CUDA(cudaStreamSynchronize(s));
    LAMG_REQUIRE(nnz >= 0 && nnz < ((int64_t)1 << 31), LAMG_ERR_ARG, "row_ptr[n] must be < 2^31");
    LAMG_REQUIRE(nnz == 0 || (col && w), LAMG_ERR_ARG, "NULL col or w");
    h->sl.clear();
    h->sl.reserve(128);
    h->sl.emplace_back();
    {
        SetupLevel &L0 = h->sl[0];
        L0.n = (int32_t)n;
        L0.nnz = nnz;
        L0.rp.alloc(n + 1);
        L0.col.alloc(nnz);
        L0.w.alloc(nnz);
        k_rp64_to_32<<<ceil_div(n + 1, 256), 256, 0, s>>>(row_ptr, L0.rp.get(), n + 1);
        LAMG_CHECK_LAUNCH();
        if (nnz) {
            LAMG_CUDA(cudaMemcpyAsync(L0.col.get(), col, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, s));
            k_w_to_64<<<ceil_div(nnz, 256), 256, 0, s>>>(w, w_is_fp32, L0.w.get(), nnz);
            LAMG_CHECK_LAUNCH();
        }
    }
    const int maxl = std::min(o.max_levels, 128);
    int32_t nxl = o.lgmg_nx;   // Lean Geometric MG: the current grid side
    LAMG_REQUIRE(nxl >= 0 && (nxl == 0 || (int64_t)nxl * nxl == n), LAMG_ERR_ARG,
                 "lgmg_nx * lgmg_nx must equal n");
    int nagg = 0;   // aggregation levels so far (the TV count grows with them)
    for (int l = 0;; l++) {
        SetupLevel &L = h->sl[l];
        const int32_t nl = L.n;
        h->L = l + 1;
        Tiers T(nl, s);
        build_tiers(L.rp.get(), nl, T, s);
        Tmp<double> diag(nl, s), adiag(nl, s), maxw(nl, s);
        L.hub.alloc(nl);
        LAUNCH3(k_node_stats, nl, (const int32_t *)nullptr, T.w.get(), T.nw, T.b.get(), T.nb, s, L.rp.get(),
                L.col.get(), L.w.get(), o.hub_factor, diag.get(), adiag.get(), maxw.get(), L.hub.get());
        if (nl < o.n_coarsest || l + 1 >= maxl || (nxl > 0 && (nxl % 2 != 0 || nxl < 6))) {
            colour_level(h, L, l, T, nxl, s);
            L.coarsest = 1;
            L.stop_reason = nl < o.n_coarsest ? 1 : 4;
            break;
        }
        if (o.elim && nxl == 0) {   // low-degree elimination before aggregating (Sec. 3.2)
            L.nF = select_elim(h, L, l, s);
            if (L.nF >= 1 && (double)L.nF >= o.elim_min_frac * (double)nl) {
                colour_level(h, L, l, T, 0, s, false);   // no relaxation on this level: one colour
                L.elim = 1;
                L.nc = (int32_t)(nl - L.nF);
                Tmp<int32_t> erow(L.nnz, s);
                LAUNCH3(k_entry_rows, nl, (const int32_t *)nullptr, T.w.get(), T.nw, T.b.get(), T.nb, s,
                        L.rp.get(), erow.get());
                h->sl.emplace_back();   // capacity reserved: references stay valid
                eliminate_level(h->sl[l], h->sl[l + 1], erow.get(), diag.get(), s);
                continue;
            }
            L.nF = 0;
            L.cidx.release();
        }
        colour_level(h, L, l, T, nxl, s);
        if (nxl > 0) {   // Lean Geometric MG: 1:2 coarsening in both directions, 2x2 aggregates
            L.agg.alloc(nl);
            L.state.alloc(nl);
            k_geo_agg<<<ceil_div(nl, 256), 256, 0, s>>>(nl, nxl, L.agg.get(), L.state.get());
            LAMG_CHECK_LAUNCH();
            LAMG_CUDA(cudaMemsetAsync(L.hub.get(), 0, (size_t)nl, s));
            L.nc = (nxl / 2) * (nxl / 2);
            L.alpha = (double)L.nc / (double)nl;
            Tmp<int32_t> erow(L.nnz, s);
            LAUNCH3(k_entry_rows, nl, (const int32_t *)nullptr, T.w.get(), T.nw, T.b.get(), T.nb, s, L.rp.get(),
                    erow.get());
            h->sl.emplace_back();
            galerkin_level(h->sl[l], h->sl[l + 1], erow.get(), s);
            nxl /= 2;
            continue;
        }
        int K = o.k_finest + o.k_step * nagg;
        if (K > o.k_max) K = o.k_max;
        if (K > 16) K = 16;
        if (K < 1) K = 1;
        L.K = K;
        Tmp<double> X((size_t)nl * K, s);
        L.tv_ratio = relax_tvs(h, L, l, T, diag.get(), X.get(), s);
        if (o.keep_setup_data) {
            L.tv.alloc((size_t)nl * K);
            LAMG_CUDA(cudaMemcpyAsync(L.tv.get(), X.get(), sizeof(double) * nl * K, cudaMemcpyDeviceToDevice, s));
        }
        if (L.tv_ratio <= o.relax_fast_ratio) {
            L.coarsest = 1;
            L.stop_reason = 2;
            break;
        }
        // per-node TV quantities, then per-entry affinity / energy ratio / score
        Tmp<double> XX(nl, s), ystar((size_t)nl * K, s), emin((size_t)nl * K, s);
        LAUNCH3(k_node_pre, nl, (const int32_t *)nullptr, T.w.get(), T.nw, T.b.get(), T.nb, s, L.rp.get(),
                L.col.get(), L.w.get(), adiag.get(), K, X.get(), XX.get(), ystar.get(), emin.get());
        Tmp<int32_t> erow(L.nnz, s);
        LAUNCH3(k_entry_rows, nl, (const int32_t *)nullptr, T.w.get(), T.nw, T.b.get(), T.nb, s, L.rp.get(),
                erow.get());
        Tmp<double> score(L.nnz, s);
        if (o.keep_setup_data) {
            L.aff.alloc(L.nnz);
            L.q.alloc(L.nnz);
            L.score.alloc(L.nnz);
        }
        if (L.nnz) {
            k_scores<<<ceil_div(L.nnz, 256), 256, 0, s>>>(L.nnz, erow.get(), L.col.get(), L.w.get(), K, X.get(),
                                                         XX.get(), ystar.get(), emin.get(), adiag.get(),
                                                         maxw.get(), o.q_max, o.weak_tol, L.aff.get(),
                                                         L.q.get(), score.get());
            LAMG_CHECK_LAUNCH();
            if (o.keep_setup_data)
                LAMG_CUDA(cudaMemcpyAsync(L.score.get(), score.get(), sizeof(double) * L.nnz,
                                          cudaMemcpyDeviceToDevice, s));
        }
        aggregate_level(h, L, l, T, score.get(), maxw.get(), s);
        if (L.alpha > o.alpha_stall) {
            L.coarsest = 1;
            L.stop_reason = 3;
            break;
        }
        h->sl.emplace_back();
        galerkin_level(h->sl[l], h->sl[l + 1], erow.get(), s);
        nagg++;
    }
    cycle_indices(h);
    LAMG_CUDA(cudaStreamSynchronize(s));
}

}  // namespace lamg
