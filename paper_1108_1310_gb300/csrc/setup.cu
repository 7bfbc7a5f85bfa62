// setup.cu -- the LAMG setup phase on the GPU (Sec. 4.1 of Livne & Brandt,
// arXiv 1108.1310): colouring, test-vector relaxation (Sec. 3.3.1), affinity
// (Eq. (3.5)) and energy ratio (Eq. (3.12)) per edge, hubs (Sec. 3.4.1),
// aggregation stages (Sec. 3.4.2), Galerkin coarse operator (Eq. (2.5)).
//
// Every floating-point value that feeds an integer decision is computed in
// FP64 with a fixed operation order (this translation unit is compiled with
// -fmad=false, so no multiply-add is contracted):
//  * row sums of up to kLongRow terms: one thread, left to right from +0.0;
//  * longer sums: one warp, lane j sums terms j, j+32, ... left to right, then
//    p_j += p_{j+h} for h = 16, 8, 4, 2, 1 (shfl_down); the result is lane 0's.
// Rows are therefore processed by a thread-per-row kernel (short rows) and a
// warp-per-row kernel (the list of long rows).
#include <cmath>
#include <cstdio>

#include "lamg_internal.cuh"

namespace lamg {

constexpr unsigned kFull = 0xffffffffu;
enum { ST_U = 0, ST_S = 1, ST_A = 2, ST_D = 3 };

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

__device__ __forceinline__ double warp_tree(double p) {
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) p = p + __shfl_down_sync(kFull, p, h);
    return __shfl_sync(kFull, p, 0);
}

// Row addressing: thread variant covers rows [0, n) and skips long rows;
// warp variant takes its rows from the long-row list.
template <bool WARP>
__device__ __forceinline__ bool get_row(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                                        int32_t &row, int &lane) {
    if (!WARP) {
        int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (i >= n) return false;
        row = (int32_t)i;
        lane = 0;
        return true;
    }
    int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wg >= nlist) return false;
    row = list[wg];
    lane = threadIdx.x & 31;
    return true;
}

template <bool WARP>
static void grid_for(int64_t count, int &blocks, int &threads) {
    threads = 256;
    int64_t t = WARP ? count * 32 : count;
    blocks = (int)std::max<int64_t>(1, (t + threads - 1) / threads);
}

#define LAUNCH_ROWS(KERNEL, N, LIST, NLIST, S, ...)                                       \
    do {                                                                                  \
        int b_, t_;                                                                       \
        if ((N) > 0) {                                                                    \
            grid_for<false>((N), b_, t_);                                                 \
            KERNEL<false><<<b_, t_, 0, (S)>>>((N), (LIST), (NLIST), __VA_ARGS__);         \
            LAMG_CHECK_LAUNCH();                                                          \
        }                                                                                 \
        if ((NLIST) > 0) {                                                                \
            grid_for<true>((NLIST), b_, t_);                                              \
            KERNEL<true><<<b_, t_, 0, (S)>>>((N), (LIST), (NLIST), __VA_ARGS__);          \
            LAMG_CHECK_LAUNCH();                                                          \
        }                                                                                 \
    } while (0)

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

__global__ void k_validate_rows(int64_t n, const int64_t *__restrict__ rp,
                                const int32_t *__restrict__ col, const double *__restrict__ w,
                                int32_t *flags) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    int64_t s = rp[u], e = rp[u + 1];
    int f = 0;
    if (e < s) f |= VF_ARG;
    for (int64_t i = s; i < e && !(f & VF_ARG); i++) {
        int32_t v = col[i];
        if (v < 0 || v >= n || v == u) f |= VF_ARG;
        if (i > s && v <= col[i - 1]) f |= VF_ARG;
        double x = w[i];
        if (!(x > 0.0) || !isfinite(x)) f |= VF_WEIGHT;
    }
    if (f) atomicOr(flags, f);
}

__global__ void k_validate_sym(int64_t n, const int64_t *__restrict__ rp,
                               const int32_t *__restrict__ col, const double *__restrict__ w,
                               int32_t *flags) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    for (int64_t i = rp[u]; i < rp[u + 1]; i++) {
        int32_t v = col[i];
        int64_t lo = rp[v], hi = rp[v + 1] - 1, f = -1;
        while (lo <= hi) {
            int64_t mid = (lo + hi) >> 1;
            int32_t c = col[mid];
            if (c == u) { f = mid; break; }
            if (c < u) lo = mid + 1; else hi = mid - 1;
        }
        if (f < 0 || __double_as_longlong(w[f]) != __double_as_longlong(w[i])) {
            atomicOr(flags, VF_SYM);
            return;
        }
    }
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

__global__ void k_uf_union(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                           int32_t *parent) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    for (int64_t i = rp[u]; i < rp[u + 1]; i++) {
        int32_t v = col[i];
        if (v <= u) continue;
        int32_t a = (int32_t)u, b = v;
        // hook the larger root under the smaller; retry until both share a root
        for (int it = 0; it < (1 << 20); it++) {
            int32_t ra = uf_find(parent, a), rb = uf_find(parent, b);
            if (ra == rb) break;
            int32_t hi = ra > rb ? ra : rb, lo = ra > rb ? rb : ra;
            if (atomicCAS(&parent[hi], hi, lo) == hi) break;
            a = ra; b = rb;
        }
    }
}

__global__ void k_uf_roots(int32_t *parent, int64_t n, unsigned long long *roots) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c = 0;
    if (i < n) c = (uf_find(parent, (int32_t)i) == i) ? 1ull : 0ull;
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(roots, c);
}

void validate_graph(int64_t n, const int64_t *row_ptr, const int32_t *col, const void *w,
                    int32_t w_is_fp32, cudaStream_t s) {
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
    k_validate_rows<<<ceil_div(n, 256), 256, 0, s>>>(n, row_ptr, col, w64.get(), flags.get());
    LAMG_CHECK_LAUNCH();
    int32_t f = read_scalar(flags.get(), s);
    LAMG_REQUIRE(!(f & VF_ARG), LAMG_ERR_ARG,
                 "malformed CSR: columns must be in range, strictly increasing, no self loops");
    LAMG_REQUIRE(!(f & VF_WEIGHT), LAMG_ERR_BAD_WEIGHT, "weights must be positive and finite");
    k_validate_sym<<<ceil_div(n, 256), 256, 0, s>>>(n, row_ptr, col, w64.get(), flags.get());
    LAMG_CHECK_LAUNCH();
    f = read_scalar(flags.get(), s);
    LAMG_REQUIRE(!(f & VF_SYM), LAMG_ERR_NOT_SYMMETRIC, "CSR is not symmetric (w_uv != w_vu)");
    Tmp<int32_t> parent(n, s);
    Tmp<unsigned long long> roots(1, s);
    LAMG_CUDA(cudaMemsetAsync(roots.get(), 0, sizeof(unsigned long long), s));
    k_uf_init<<<ceil_div(n, 256), 256, 0, s>>>(parent.get(), n);
    LAMG_CHECK_LAUNCH();
    k_uf_union<<<ceil_div(n, 256), 256, 0, s>>>(n, row_ptr, col, parent.get());
    LAMG_CHECK_LAUNCH();
    k_uf_roots<<<ceil_div(n, 256), 256, 0, s>>>(parent.get(), n, roots.get());
    LAMG_CHECK_LAUNCH();
    unsigned long long r = read_scalar(roots.get(), s);
    LAMG_REQUIRE(r == 1, LAMG_ERR_DISCONNECTED, "graph is not connected");
}

// ---------------------------------------------------------------------------
// Per-node statistics: a_uu, max|w|, hub test (Sec. 3.4.1 footnote)
// ---------------------------------------------------------------------------

template <bool WARP>
__global__ void k_node_stats(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                             const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                             const double *__restrict__ w, double hub_factor,
                             double *__restrict__ diag, double *__restrict__ maxw,
                             uint8_t *__restrict__ hub) {
    int32_t u; int lane;
    if (!get_row<WARP>(n, list, nlist, u, lane)) return;
    const int32_t s = rp[u], e = rp[u + 1], deg = e - s;
    if (!WARP && deg > kLongRow) return;
    double d = 0.0, m = 0.0, s1 = 0.0, s2 = 0.0;
    for (int32_t i = s + lane; i < e; i += (WARP ? 32 : 1)) {
        const double wi = w[i];
        const int32_t v = col[i];
        const double a = fabs(wi);
        d = d + wi;
        m = fmax(m, a);
        s1 = s1 + a;
        s2 = s2 + a * (double)(rp[v + 1] - rp[v]);
    }
    if (WARP) {
        d = warp_tree(d);
        s1 = warp_tree(s1);
        s2 = warp_tree(s2);
        for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
        if (lane) return;
    }
    diag[u] = d;
    maxw[u] = m;
    const double lhs = (double)deg * s1;
    const double rhs = hub_factor * s2;
    hub[u] = (deg > 0 && lhs >= rhs) ? 1 : 0;
}

// Initial aggregation state (Sec. 3.4.2): nodes without strong edges form the
// dummy aggregate (D), hubs are seeds (S), the rest undecided (U).
template <bool WARP>
__global__ void k_node_state(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                             const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                             const double *__restrict__ w, const double *__restrict__ maxw,
                             double weak_tol, const uint8_t *__restrict__ hub,
                             int32_t *__restrict__ state) {
    int32_t u; int lane;
    if (!get_row<WARP>(n, list, nlist, u, lane)) return;
    const int32_t s = rp[u], e = rp[u + 1];
    if (!WARP && e - s > kLongRow) return;
    bool strong = false;
    const double mu = maxw[u];
    for (int32_t i = s + lane; i < e; i += (WARP ? 32 : 1)) {
        const double mw = fmax(mu, maxw[col[i]]);
        if (fabs(w[i]) >= weak_tol * mw) strong = true;
    }
    if (WARP) {
        strong = __any_sync(kFull, strong);
        if (lane) return;
    }
    state[u] = !strong ? ST_D : (hub[u] ? ST_S : ST_U);
}

// ---------------------------------------------------------------------------
// Jones-Plassmann colouring
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool beats(uint64_t pu, int32_t u, uint64_t pv, int32_t v) {
    return pu > pv || (pu == pv && u < v);
}

template <bool WARP>
__global__ void k_jp_select(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                            const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                            const int32_t *__restrict__ colour, uint64_t key,
                            uint8_t *__restrict__ sel) {
    int32_t u; int lane;
    if (!get_row<WARP>(n, list, nlist, u, lane)) return;
    const int32_t s = rp[u], e = rp[u + 1];
    if (!WARP && e - s > kLongRow) return;
    if (colour[u] >= 0) {
        if (lane == 0) sel[u] = 0;
        return;
    }
    const uint64_t pu = splitmix64(key + (uint64_t)u);
    bool is_max = true;
    for (int32_t i = s + lane; i < e; i += (WARP ? 32 : 1)) {
        const int32_t v = col[i];
        if (colour[v] < 0 && beats(splitmix64(key + (uint64_t)v), v, pu, u)) { is_max = false; break; }
    }
    if (WARP) {
        is_max = __all_sync(kFull, is_max);
        if (lane) return;
    }
    sel[u] = is_max ? 1 : 0;
}

template <bool WARP>
__global__ void k_jp_assign(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                            const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                            const uint8_t *__restrict__ sel, int32_t *__restrict__ colour,
                            int32_t *__restrict__ remaining) {
    int32_t u; int lane;
    if (!get_row<WARP>(n, list, nlist, u, lane)) return;
    const int32_t s = rp[u], e = rp[u + 1];
    if (!WARP && e - s > kLongRow) return;
    if (!sel[u]) return;
    // smallest colour not used by a neighbour, searched in windows of 64
    for (int32_t base = 0;; base += 64) {
        unsigned long long mask = 0ull;
        for (int32_t i = s + lane; i < e; i += (WARP ? 32 : 1)) {
            const int32_t c = colour[col[i]];
            if (c >= base && c < base + 64) mask |= 1ull << (c - base);
        }
        if (WARP)
            for (int o = 16; o; o >>= 1) mask |= __shfl_xor_sync(kFull, mask, o);
        if (mask != ~0ull) {
            if (lane == 0) {
                colour[u] = base + __ffsll((long long)~mask) - 1;
                atomicSub(remaining, 1);
            }
            return;
        }
    }
}

__global__ void k_fill_i32(int32_t *a, int64_t n, int32_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

__global__ void k_iota(int32_t *a, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = (int32_t)i;
}

__global__ void k_to_u32(const int32_t *__restrict__ a, uint32_t *__restrict__ o, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) o[i] = (uint32_t)a[i];
}

__global__ void k_hist_i32(const int32_t *__restrict__ a, int64_t n, int32_t *__restrict__ cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&cnt[a[i]], 1);
}

__global__ void k_long_flags(const int32_t *__restrict__ rp, const int32_t *__restrict__ order,
                             int64_t n, uint8_t *__restrict__ f) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t u = order ? order[i] : (int32_t)i;
    f[i] = (rp[u + 1] - rp[u]) > kLongRow ? 1 : 0;
}

__global__ void k_gather_i32(const int32_t *__restrict__ idx, const int32_t *__restrict__ src,
                             int32_t *__restrict__ dst, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

static int bits_for(uint64_t maxval) {
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) b++;
    return b;
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

// One colour of a TV sweep: rows order[lo..hi) (thread variant skips long rows;
// warp variant takes the colour's long rows from `list`).
template <bool WARP>
__global__ void k_tv_sweep(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                           const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                           const double *__restrict__ w, const double *__restrict__ diag,
                           int32_t K, double *__restrict__ X) {
    int32_t i; int lane;
    if (!get_row<WARP>(n, list, nlist, i, lane)) return;
    const int32_t u = WARP ? i : list[i];  // thread variant: list = colour order slice
    const int32_t s = rp[u], e = rp[u + 1];
    if (!WARP && e - s > kLongRow) return;
    const double du = diag[u];
    for (int k = 0; k < K; k++) {
        double acc = 0.0;
        for (int32_t j = s + lane; j < e; j += (WARP ? 32 : 1))
            acc = acc + w[j] * X[(int64_t)col[j] * K + k];
        if (WARP) acc = warp_tree(acc);
        if (lane == 0) X[(int64_t)u * K + k] = acc / du;
        if (WARP) __syncwarp();
    }
}

// Nodal energy E_u = 1/2 sum_v w_uv (x_u - x_v)^2 of TV k (Eq. (3.11a)).
template <bool WARP>
__global__ void k_tv_energy(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                            const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                            const double *__restrict__ w, int32_t K, int32_t k,
                            const double *__restrict__ X, double *__restrict__ eu) {
    int32_t u; int lane;
    if (!get_row<WARP>(n, list, nlist, u, lane)) return;
    const int32_t s = rp[u], e = rp[u + 1];
    if (!WARP && e - s > kLongRow) return;
    const double xu = X[(int64_t)u * K + k];
    double acc = 0.0;
    for (int32_t j = s + lane; j < e; j += (WARP ? 32 : 1)) {
        const double d = xu - X[(int64_t)col[j] * K + k];
        acc = acc + w[j] * (d * d);
    }
    if (WARP) acc = warp_tree(acc);
    if (lane == 0) eu[u] = 0.5 * acc;
}

// Canonical sum of chunks of 4096 terms, one warp per chunk.
__global__ void k_canon_chunks(const double *__restrict__ t, int64_t len, double *__restrict__ out) {
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t lo = c * 4096;
    if (lo >= len) return;
    const int64_t cnt = (len - lo) < 4096 ? (len - lo) : 4096;
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
    Tmp<double> a((size_t)std::max<int64_t>(1, (len + 4095) / 4096), s);
    Tmp<double> b((size_t)std::max<int64_t>(1, (len + 4095) / 4096), s);
    const double *src = t;
    double *dst = a.get(), *other = b.get();
    while (true) {
        int64_t nch = (len + 4095) / 4096;
        if (nch < 1) nch = 1;
        k_canon_chunks<<<ceil_div(nch * 32, 256), 256, 0, s>>>(src, len, dst);
        LAMG_CHECK_LAUNCH();
        if (len <= 4096) break;
        len = nch;
        src = dst;
        std::swap(dst, other);
    }
    return read_scalar(dst, s);
}

// ---------------------------------------------------------------------------
// Affinity and energy ratio (Eqs. (3.5), (3.12)); see the oracle for the
// reading of Eq. (3.12): q_us = max_k E_u(x^k; x^k_s) / min_y E_u(x^k; y).
// ---------------------------------------------------------------------------

template <bool WARP>
__global__ void k_node_pre(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                           const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                           const double *__restrict__ w, const double *__restrict__ diag,
                           int32_t K, const double *__restrict__ X, double *__restrict__ XX,
                           double *__restrict__ ystar, double *__restrict__ emin) {
    int32_t u; int lane;
    if (!get_row<WARP>(n, list, nlist, u, lane)) return;
    const int32_t s = rp[u], e = rp[u + 1];
    if (!WARP && e - s > kLongRow) return;
    if (lane == 0) {
        double xx = 0.0;
        for (int k = 0; k < K; k++) {
            const double x = X[(int64_t)u * K + k];
            xx = xx + x * x;
        }
        XX[u] = xx;
    }
    const double du = diag[u];
    for (int k = 0; k < K; k++) {
        double B = 0.0;
        for (int32_t j = s + lane; j < e; j += (WARP ? 32 : 1))
            B = B + w[j] * X[(int64_t)col[j] * K + k];
        if (WARP) B = warp_tree(B);
        const double y = B / du;
        double E = 0.0;
        for (int32_t j = s + lane; j < e; j += (WARP ? 32 : 1)) {
            const double d = y - X[(int64_t)col[j] * K + k];
            E = E + w[j] * (d * d);
        }
        if (WARP) E = warp_tree(E);
        if (lane == 0) {
            ystar[(int64_t)u * K + k] = y;
            emin[(int64_t)u * K + k] = 0.5 * E;
        }
    }
}

template <bool WARP>
__global__ void k_entry_rows(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                             const int32_t *__restrict__ rp, int32_t *__restrict__ erow) {
    int32_t u; int lane;
    if (!get_row<WARP>(n, list, nlist, u, lane)) return;
    const int32_t s = rp[u], e = rp[u + 1];
    if (!WARP && e - s > kLongRow) return;
    for (int32_t j = s + lane; j < e; j += (WARP ? 32 : 1)) erow[j] = u;
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
    for (int k = 0; k < K; k++) dot = dot + xu[k] * xv[k];
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

template <bool WARP>
__global__ void k_best(int32_t n, const int32_t *__restrict__ list, int32_t nlist,
                       const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                       const double *__restrict__ score, const int32_t *__restrict__ state,
                       int32_t *__restrict__ best) {
    int32_t u; int lane;
    if (!get_row<WARP>(n, list, nlist, u, lane)) return;
    const int32_t s = rp[u], e = rp[u + 1];
    if (!WARP && e - s > kLongRow) return;
    if (state[u] != ST_U) {
        if (lane == 0) best[u] = -1;
        return;
    }
    double bs = -1.0;
    int32_t bv = -1;
    for (int32_t j = s + lane; j < e; j += (WARP ? 32 : 1)) {
        const int32_t v = col[j];
        const double sc = score[j];
        if (sc < 0.0 || state[v] == ST_A) continue;
        if (sc > bs || (sc == bs && v < bv)) { bs = sc; bv = v; }
    }
    if (WARP) {
        for (int o = 16; o; o >>= 1) {
            const double os = __shfl_xor_sync(kFull, bs, o);
            const int32_t ov = __shfl_xor_sync(kFull, bv, o);
            if (ov >= 0 && (os > bs || (os == bs && (bv < 0 || ov < bv)))) { bs = os; bv = ov; }
        }
        if (lane) return;
    }
    best[u] = bv;
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

__global__ void k_seg_long(int64_t P, const int32_t *__restrict__ start, int64_t M,
                           uint8_t *__restrict__ f) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int64_t e = (p + 1 < P) ? start[p + 1] : M;
    f[p] = (e - start[p]) > kLongRow ? 1 : 0;
}

// Segment sums: thread variant for short segments, warp variant for the long list.
template <bool WARP>
__global__ void k_seg_sum(int32_t P, const int32_t *__restrict__ list, int32_t nlist,
                          const int32_t *__restrict__ start, int64_t M,
                          const double *__restrict__ val, double *__restrict__ W) {
    int32_t p; int lane;
    if (!get_row<WARP>(P, list, nlist, p, lane)) return;
    const int64_t s = start[p], e = (p + 1 < P) ? start[p + 1] : M;
    if (!WARP && e - s > kLongRow) return;
    double acc = 0.0;
    for (int64_t j = s + lane; j < e; j += (WARP ? 32 : 1)) acc = acc + val[j];
    if (WARP) acc = warp_tree(acc);
    if (lane == 0) W[p] = acc;
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
// Driver
// ---------------------------------------------------------------------------

struct LongList {
    int32_t n = 0;
    Tmp<int32_t> *buf = nullptr;
};

static int32_t build_long_rows(const int32_t *rp, int32_t n, Tmp<int32_t> &out, cudaStream_t s) {
    Tmp<uint8_t> f(n, s);
    k_long_flags<<<ceil_div(n, 256), 256, 0, s>>>(rp, nullptr, n, f.get());
    LAMG_CHECK_LAUNCH();
    return (int32_t)compact_indices(f.get(), out.get(), n, s);
}

static void colour_level(lamg_ctx *h, SetupLevel &L, int level, const int32_t *longrows,
                         int32_t nlong, cudaStream_t s) {
    const int32_t n = L.n;
    L.colour.alloc(n);
    Tmp<uint8_t> sel(n, s);
    Tmp<int32_t> remaining(1, s);
    k_fill_i32<<<ceil_div(n, 256), 256, 0, s>>>(L.colour.get(), n, -1);
    LAMG_CHECK_LAUNCH();
    LAMG_CUDA(cudaMemcpyAsync(remaining.get(), &n, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    const uint64_t key = colour_key(h->opt.seed, level);
    int rounds = 0;
    for (int32_t left = n; left > 0; rounds++) {
        LAMG_REQUIRE(rounds < 100000, LAMG_ERR_CUDA, "colouring did not terminate");
        LAUNCH_ROWS(k_jp_select, n, longrows, nlong, s, L.rp.get(), L.col.get(), L.colour.get(), key,
                    sel.get());
        LAUNCH_ROWS(k_jp_assign, n, longrows, nlong, s, L.rp.get(), L.col.get(), sel.get(),
                    L.colour.get(), remaining.get());
        left = read_scalar(remaining.get(), s);
    }
    L.jp_rounds = rounds;
    L.ncolours = reduce_max_i32(L.colour.get(), n, s) + 1;
    // nodes sorted by (colour, id) and the colour ranges
    L.corder.alloc(n);
    Tmp<uint32_t> keys(n, s), ktmp(n, s);
    Tmp<int32_t> vtmp(n, s), cnt(L.ncolours + 1, s), cst(L.ncolours + 1, s);
    k_to_u32<<<ceil_div(n, 256), 256, 0, s>>>(L.colour.get(), keys.get(), n);
    LAMG_CHECK_LAUNCH();
    k_iota<<<ceil_div(n, 256), 256, 0, s>>>(L.corder.get(), n);
    LAMG_CHECK_LAUNCH();
    radix_sort_pairs<uint32_t, int32_t>(keys.get(), L.corder.get(), ktmp.get(), vtmp.get(), n,
                                        bits_for((uint64_t)L.ncolours - 1), s);
    LAMG_CUDA(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t) * (L.ncolours + 1), s));
    k_hist_i32<<<ceil_div(n, 256), 256, 0, s>>>(L.colour.get(), n, cnt.get());
    LAMG_CHECK_LAUNCH();
    exclusive_scan_i32(cnt.get(), cst.get(), L.ncolours + 1, s);
    L.cstart.resize(L.ncolours + 1);
    LAMG_CUDA(cudaMemcpyAsync(L.cstart.data(), cst.get(), sizeof(int32_t) * (L.ncolours + 1),
                              cudaMemcpyDeviceToHost, s));
    LAMG_CUDA(cudaStreamSynchronize(s));
}

// TVs and their sweeps; returns the largest per-TV energy ratio of the last
// sweep when the relaxation-speed test is enabled (else +inf).
static double relax_tvs(lamg_ctx *h, SetupLevel &L, int level, const double *diag, double *X,
                        cudaStream_t s) {
    const int32_t n = L.n, K = L.K;
    const lamg_options &o = h->opt;
    k_tv_init<<<ceil_div((int64_t)n * K, 256), 256, 0, s>>>(X, (int64_t)n * K, tv_key(o.seed, level));
    LAMG_CHECK_LAUNCH();
    // long rows in colour order, with per-colour ranges
    Tmp<uint8_t> f(n, s);
    Tmp<int32_t> pos(n, s), lorder(n, s);
    k_long_flags<<<ceil_div(n, 256), 256, 0, s>>>(L.rp.get(), L.corder.get(), n, f.get());
    LAMG_CHECK_LAUNCH();
    int32_t nl = (int32_t)compact_indices(f.get(), pos.get(), n, s);
    std::vector<int32_t> lstart(L.ncolours + 1, 0);
    if (nl > 0) {
        k_gather_i32<<<ceil_div(nl, 256), 256, 0, s>>>(pos.get(), L.corder.get(), lorder.get(), nl);
        LAMG_CHECK_LAUNCH();
        std::vector<int32_t> hpos(nl);
        LAMG_CUDA(cudaMemcpyAsync(hpos.data(), pos.get(), sizeof(int32_t) * nl, cudaMemcpyDeviceToHost, s));
        LAMG_CUDA(cudaStreamSynchronize(s));
        // positions in corder are sorted; colour c covers corder [cstart[c], cstart[c+1])
        int32_t j = 0;
        for (int c = 0; c <= L.ncolours; c++) {
            while (j < nl && hpos[j] < L.cstart[c]) j++;
            lstart[c] = j;
        }
        lstart[L.ncolours] = nl;
    }
    const bool test = o.relax_fast_ratio > 0.0 && o.nu_tv >= 2;
    Tmp<double> eu(test ? n : 0, s);
    Tmp<int32_t> noneL(0, s);
    double eprev[16], ecur[16];
    for (int sw = 1; sw <= o.nu_tv; sw++) {
        for (int c = 0; c < L.ncolours; c++) {
            const int32_t c0 = L.cstart[c], c1 = L.cstart[c + 1];
            if (c1 > c0) {
                int b, t;
                grid_for<false>(c1 - c0, b, t);
                k_tv_sweep<false><<<b, t, 0, s>>>(c1 - c0, L.corder.get() + c0, 0, L.rp.get(),
                                                 L.col.get(), L.w.get(), diag, K, X);
                LAMG_CHECK_LAUNCH();
            }
            const int32_t l0 = lstart[c], l1 = lstart[c + 1];
            if (l1 > l0) {
                int b, t;
                grid_for<true>(l1 - l0, b, t);
                k_tv_sweep<true><<<b, t, 0, s>>>(0, lorder.get() + l0, l1 - l0, L.rp.get(),
                                                L.col.get(), L.w.get(), diag, K, X);
                LAMG_CHECK_LAUNCH();
            }
        }
        if (test && sw >= o.nu_tv - 1) {
            Tmp<int32_t> lr(n, s);
            int32_t nlr = build_long_rows(L.rp.get(), n, lr, s);
            for (int k = 0; k < K; k++) {
                LAUNCH_ROWS(k_tv_energy, n, lr.get(), nlr, s, L.rp.get(), L.col.get(), L.w.get(), K, k,
                            X, eu.get());
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
static void aggregate_level(lamg_ctx *h, SetupLevel &L, const int32_t *longrows, int32_t nlong,
                            const double *score, const double *maxw, cudaStream_t s) {
    const int32_t n = L.n;
    const lamg_options &o = h->opt;
    Tmp<int32_t> state(n, s), seed(n, s), best(n, s), nstate(n, s), nseed(n, s), bseed(n, s);
    L.state.alloc(n);
    L.agg.alloc(n);
    LAUNCH_ROWS(k_node_state, n, longrows, nlong, s, L.rp.get(), L.col.get(), L.w.get(), maxw,
                o.weak_tol, L.hub.get(), state.get());
    LAMG_CUDA(cudaMemsetAsync(seed.get(), 0xFF, sizeof(int32_t) * n, s));
    const int64_t nd = count_equal_i32(state.get(), n, ST_D, s);
    const double amax = 0.7 / o.gamma;
    double best_alpha = INFINITY;
    int best_round = 0, r;
    Tmp<int32_t> changed(1, s);
    Tmp<unsigned long long> cnt(1, s);
    for (r = 1; r <= o.max_rounds; r++) {
        LAUNCH_ROWS(k_best, n, longrows, nlong, s, L.rp.get(), L.col.get(), score, state.get(), best.get());
        LAMG_CUDA(cudaMemcpyAsync(nstate.get(), state.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
        LAMG_CUDA(cudaMemcpyAsync(nseed.get(), seed.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
        LAMG_CUDA(cudaMemsetAsync(changed.get(), 0, sizeof(int32_t), s));
        k_resolve<<<ceil_div(n, 256), 256, 0, s>>>(n, state.get(), best.get(), nstate.get(), nseed.get(),
                                                  changed.get());
        LAMG_CHECK_LAUNCH();
        LAMG_CUDA(cudaMemcpyAsync(state.get(), nstate.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
        LAMG_CUDA(cudaMemcpyAsync(seed.get(), nseed.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
        LAMG_CUDA(cudaMemsetAsync(cnt.get(), 0, sizeof(unsigned long long), s));
        k_count_su<<<ceil_div(n, 256), 256, 0, s>>>(state.get(), n, cnt.get());
        LAMG_CHECK_LAUNCH();
        const int32_t ch = read_scalar(changed.get(), s);
        const unsigned long long su = read_scalar(cnt.get(), s);
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
    L.rounds = r > o.max_rounds ? o.max_rounds : r;
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
    Tmp<uint8_t> lf(P, s);
    Tmp<int32_t> lsegs(P, s);
    Tmp<double> W(P, s);
    int64_t nls = 0;
    if (P) {
        k_seg_long<<<ceil_div(P, 256), 256, 0, s>>>(P, start.get(), M, lf.get());
        LAMG_CHECK_LAUNCH();
        nls = compact_indices(lf.get(), lsegs.get(), P, s);
        LAUNCH_ROWS(k_seg_sum, (int32_t)P, lsegs.get(), (int32_t)nls, s, start.get(), M, val.get(), W.get());
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
        const double ml = (double)h->sl[l].nnz / 2.0, mn = (double)h->sl[l + 1].nnz / 2.0;
        double g = mn > 0.0 ? 0.7 * ml / mn : 2.0;
        const double gmax = ml > 0.1 * m1 ? h->opt.gamma : 2.0;
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
    for (int l = 0;; l++) {
        SetupLevel &L = h->sl[l];
        const int32_t nl = L.n;
        h->L = l + 1;
        Tmp<int32_t> longrows(nl, s);
        const int32_t nlong = build_long_rows(L.rp.get(), nl, longrows, s);
        Tmp<double> diag(nl, s), maxw(nl, s);
        L.hub.alloc(nl);
        LAUNCH_ROWS(k_node_stats, nl, longrows.get(), nlong, s, L.rp.get(), L.col.get(), L.w.get(),
                    o.hub_factor, diag.get(), maxw.get(), L.hub.get());
        colour_level(h, L, l, longrows.get(), nlong, s);
        if (nl < o.n_coarsest || l + 1 >= maxl) {
            L.coarsest = 1;
            L.stop_reason = nl < o.n_coarsest ? 1 : 4;
            break;
        }
        int K = o.k_finest + o.k_step * l;
        if (K > o.k_max) K = o.k_max;
        if (K > 16) K = 16;
        if (K < 1) K = 1;
        L.K = K;
        Tmp<double> X((size_t)nl * K, s);
        L.tv_ratio = relax_tvs(h, L, l, diag.get(), X.get(), s);
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
        LAUNCH_ROWS(k_node_pre, nl, longrows.get(), nlong, s, L.rp.get(), L.col.get(), L.w.get(),
                    diag.get(), K, X.get(), XX.get(), ystar.get(), emin.get());
        Tmp<int32_t> erow(L.nnz, s);
        LAUNCH_ROWS(k_entry_rows, nl, longrows.get(), nlong, s, L.rp.get(), erow.get());
        Tmp<double> score(L.nnz, s);
        if (o.keep_setup_data) {
            L.aff.alloc(L.nnz);
            L.q.alloc(L.nnz);
            L.score.alloc(L.nnz);
        }
        if (L.nnz) {
            k_scores<<<ceil_div(L.nnz, 256), 256, 0, s>>>(L.nnz, erow.get(), L.col.get(), L.w.get(), K, X.get(),
                                                         XX.get(), ystar.get(), emin.get(), diag.get(),
                                                         maxw.get(), o.q_max, o.weak_tol, L.aff.get(),
                                                         L.q.get(), score.get());
            LAMG_CHECK_LAUNCH();
            if (o.keep_setup_data)
                LAMG_CUDA(cudaMemcpyAsync(L.score.get(), score.get(), sizeof(double) * L.nnz,
                                          cudaMemcpyDeviceToDevice, s));
        }
        aggregate_level(h, L, longrows.get(), nlong, score.get(), maxw.get(), s);
        if (L.alpha > o.alpha_stall) {
            L.coarsest = 1;
            L.stop_reason = 3;
            break;
        }
        h->sl.emplace_back();
        galerkin_level(h->sl[l], h->sl[l + 1], erow.get(), s);
    }
    cycle_indices(h);
    LAMG_CUDA(cudaStreamSynchronize(s));
}

}  // namespace lamg
